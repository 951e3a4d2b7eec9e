"""CPU checks of the launch schedule (hs_plan_schedule, host only).

The register sweep may apply a factor ahead of earlier ones when they commute.
These tests check, from the Pauli masks alone, that the schedule applies
every factor of every step exactly once, in the product formula's order up
to swaps of factors whose terms commute pairwise (Pauli strings (x1, z1) and
(x2, z2) commute iff |x1 & z2| + |z1 & x2| is even), that each sweep's
flipped qubits fit a tile, and that it never takes more sweeps than the
in-order schedule; and, with the oracle's direct rotations applied in the
schedule's order, that the evolution is the formula-order one to rounding."""
from collections import Counter, defaultdict

import numpy as np
import pytest

from paper_2606_16959_gb300 import hs, workloads as W


@pytest.fixture(scope="module")
def lib():
    from paper_2606_16959_gb300 import _build
    _build.build()
    return hs.lib()


def _commute(x, z, i, j):
    return bin((int(x[i]) & int(z[j])) ^ (int(z[i]) & int(x[j]))).count("1") % 2 == 0


def _check_schedule(x, z, n, budget, order, steps, tile_bits, low_bits, max_fuse=0):
    groups, _ = hs.hs_plan_factors(x, z, n, budget)
    G = len(groups)
    ref = hs.hs_plan_schedule(x, z, n, budget, steps, tile_bits, low_bits, order=order, max_fuse=max_fuse,
                              commuting=False)
    got = hs.hs_plan_schedule(x, z, n, budget, steps, tile_bits, low_bits, order=order, max_fuse=max_fuse,
                              commuting=True)
    rf, rs, rw = ref
    gf, gs, gw = got
    # every application once
    assert Counter(zip(rf.tolist(), rs.tolist())) == Counter(zip(gf.tolist(), gs.tolist()))
    assert np.all(np.diff(rs) >= 0) and np.all(np.diff(rw) >= 0) and np.all(np.diff(gw) >= 0)
    # position of each formula-order application in the new order (k-th copy of
    # (factor, step) matched with its k-th copy)
    seen = defaultdict(list)
    for k, key in enumerate(zip(gf.tolist(), gs.tolist())):
        seen[key].append(k)
    used = Counter()
    pos = []
    for key in zip(rf.tolist(), rs.tolist()):
        pos.append(seen[key][used[key]])
        used[key] += 1
    pos = np.array(pos)
    terms = [range(groups[g % G][0], groups[g % G][1]) for g in range(int(rf.max()) + 1)]
    memo = {}

    def factors_commute(a, b):
        k = (min(a, b), max(a, b))
        if k not in memo:
            memo[k] = all(_commute(x, z, i, j) for i in terms[a] for j in terms[b])
        return memo[k]

    swaps = 0
    for i in range(len(pos)):
        later = np.nonzero(pos[i + 1:] < pos[i])[0] + i + 1
        for j in later:
            swaps += 1
            assert factors_commute(int(rf[i]), int(rf[j])), (i, j)
    # each sweep's flips fit a tile
    for s in np.unique(gw):
        span = 0
        for g in gf[gw == s]:
            for t in terms[g]:
                span |= int(x[t])
        if (gw == s).sum() > 1:
            assert bin(span).count("1") <= tile_bits
    n_ref, n_got = int(rw.max()) + 1, int(gw.max()) + 1
    assert n_got <= n_ref
    return n_ref, n_got, swaps


def test_schedule_families(oracle, lib):
    cases = [(W.maxcut_3regular(24, 1003), 4), (W.tfim_chain(15, 1.0, 0.8), 4), (W.heisenberg_chain(14, np.ones(14)), 8),
             (W.tsp_onehot(4, 5), 4), (W.tfim_chain(20, 1.0, 0.5, periodic=True), 4)]
    for ham, budget in cases:
        x, z, n = oracle.parse_terms(ham.labels)
        for order in (1, 2, 4):
            for tb, lb in ((13, 2), (10, 3), (8, 1)):
                _check_schedule(x, z, n, budget, order, 5, min(tb, n), min(lb, n))


def test_schedule_driven_and_random(oracle, lib):
    ham = W.anneal_maxcut(16, seed=78)
    x, z, n = oracle.parse_terms(ham.labels)
    _check_schedule(x, z, n, 4, 1, 12, 13, 2)
    rng = np.random.default_rng(2024)
    for trial in range(40):
        n = int(rng.integers(4, 13))
        m = int(rng.integers(2, 24))
        labels = ["".join(rng.choice(list("IXYZ"), p=[0.6, 0.15, 0.1, 0.15], size=n)) for _ in range(m)]
        x, z, _ = oracle.parse_terms(labels)
        tb = int(rng.integers(3, n + 1))
        _check_schedule(x, z, n, int(rng.integers(1, 9)), int(rng.choice([1, 2, 4])), int(rng.integers(1, 5)), tb,
                        int(rng.integers(1, tb + 1)), max_fuse=int(rng.choice([0, 3, 8])))


def test_schedule_maxcut24_one_sweep_per_step(oracle, lib):
    """MaxCut on 24 qubits (mixer on), 2^13-row tiles keeping 2 low bits: the
    in-order schedule needs two sweeps per step (each X_i must be local, 24 >
    13); commuting the mixer's X factors lets each sweep finish one step and
    start the next, one sweep per step."""
    x, z, n = oracle.parse_terms(W.maxcut_3regular(24, 1003, 0.5).labels)  # the maxcut24 Hamiltonian
    n_ref, n_got, swaps = _check_schedule(x, z, n, 4, 1, 12, 13, 2)
    assert n_ref >= 24 and n_got <= 13 and swaps > 0
    fac, st, sw = hs.hs_plan_schedule(x, z, n, 4, 50, 13, 2)
    assert int(sw.max()) + 1 <= 51


def test_schedule_rejects_bad_input(lib):
    with pytest.raises(hs.HSError):
        hs.hs_plan_schedule([1], [0], 4, 4, 2, 0, 0)
    with pytest.raises(hs.HSError):
        hs.hs_plan_schedule([1], [0], 4, 4, 2, 3, 4)  # low bits above tile bits
    with pytest.raises(hs.HSError):
        hs.hs_plan_schedule([1], [0], 4, 4, -1, 3, 1)


def test_commuting_schedule_evolves_like_the_formula_on_the_oracle(oracle, lib):
    """The register sweep's schedule, each factor application expanded into its
    terms (first term first) and applied by the oracle's direct rotations, gives
    the formula-order evolution to rounding; swapping one non-commuting pair
    instead changes it (the check is sensitive)."""
    rng = np.random.default_rng(31)
    t, steps = 0.8, 4
    dt = t / steps
    for ham in (W.maxcut_3regular(10, 5, 0.5), W.tfim_chain(10, 1.0, 0.7), W.tfim_chain(9, 0.8, 1.1, periodic=True)):
        x, z, n = oracle.parse_terms(ham.labels)
        c = np.asarray(ham.coeffs, dtype=np.float64)
        groups, _ = hs.hs_plan_factors(x, z, n, 4)
        fac, st, sw = hs.hs_plan_schedule(x, z, n, 4, steps, 6, 1)  # tiles of 6 of the 9-10 qubits
        ref, _, rsw = hs.hs_plan_schedule(x, z, n, 4, steps, 6, 1, commuting=False)
        assert int(sw.max()) < int(rsw.max())  # the schedule does reorder here, and saves sweeps
        psi = W.gaussian_state(n, rng)
        want = oracle.evolve_direct(x, z, c, t, steps, psi)

        def run(seq):
            out = np.array(psi, dtype=np.complex128)
            for g in seq:
                a, b = groups[g][:2]
                out = oracle.evolve_direct(x[a:b], z[a:b], c[a:b], dt, 1, out)
            return out

        assert np.max(np.abs(run(ref) - want)) <= 1e-12
        assert np.max(np.abs(run(fac) - want)) <= 1e-12
        # negative control: move the first factor holding an X term ahead of the
        # factor before it when that one holds a term it anticommutes with
        seq = list(ref)
        for k in range(1, len(seq)):
            a0, b0 = groups[seq[k - 1]][:2]
            a1, b1 = groups[seq[k]][:2]
            if not all(_commute(x, z, i, j) for i in range(a0, b0) for j in range(a1, b1)):
                seq[k - 1], seq[k] = seq[k], seq[k - 1]
                break
        assert np.max(np.abs(run(seq) - want)) > 1e-6
