"""Batched evolution: one graph launch for many uneven jobs.

Each job of a batch follows the schedule hs_evolve_ex would give it (same
sweeps, same per-row arithmetic), so the batch must reproduce evolving every
job alone with the same tile_bits / low_bits and one state per tile bit for
bit; small jobs are also checked against the FP64 oracle.
"""
import numpy as np
import pytest

import oracle as O
from paper_2606_16959_gb300 import hs, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_16959_gb300 import _build
    _build.build()
    O.build()
    hs.lib()


def _tdt(dt):
    return torch.complex64 if dt == "c64" else torch.complex128


def _jobs(rng, dt, count, n_lo, n_hi, steps_hi):
    out = []
    for k in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        kind = k % 3
        if kind == 0:
            ham = W.tfim_chain(n, float(rng.uniform(0.5, 1.5)), float(rng.uniform(0, 2)), periodic=False)
        elif kind == 1:
            ham = W.heisenberg_chain(n, rng.uniform(0.5, 1.5, n), periodic=True)
        else:
            labels = ["".join(rng.choice(list("IXYZ"), p=[0.6, 0.14, 0.13, 0.13], size=n)) for _ in range(6)]
            ham = W.Hamiltonian("random", n, labels, rng.uniform(-1, 1, 6))
        steps = int(rng.integers(0, steps_hi + 1))
        budget = int(rng.integers(1, 17))
        n_rhs = 1 + (k % 4 == 3)
        psi0 = np.stack([W.gaussian_state(n, rng) for _ in range(n_rhs)])
        f = hs.hs_build_factors(ham.labels, ham.coeffs, 0.8, max(steps, 1), budget, dt)
        out.append((ham, f, psi0, steps))
    return out


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_batch_equals_jobs_alone_bitwise(dt):
    rng = np.random.default_rng(900)
    jobs = _jobs(rng, dt, 14, 7, 13, 9)
    lb = 2 if dt == "c64" else 1
    states = [torch.from_numpy(p).to("cuda", _tdt(dt)) for _, _, p, _ in jobs]
    b = hs.hs_batch_create([(f, s, st) for (_, f, _, st), s in zip(jobs, states)], tile_bits=9, low_bits=lb)
    assert b.n_separate >= 1  # the jobs below 9 qubits run with their own launches
    hs.hs_batch_launch(b)
    torch.cuda.synchronize()
    for (ham, f, p0, steps), got in zip(jobs, states):
        ref = torch.from_numpy(p0).to("cuda", _tdt(dt))
        if ham.n_qubits >= 9:
            hs.hs_evolve_ex(f, ref, steps, method=hs.HS_METHOD_FUSED, tile_bits=9, rhs_block=1, low_bits=lb)
        else:
            hs.hs_evolve(f, ref, steps)
        assert torch.equal(got, ref), (ham.family, ham.n_qubits, steps)
    b.close()


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_batch_matches_oracle_and_relaunch(dt):
    rng = np.random.default_rng(901)
    jobs = _jobs(rng, dt, 6, 9, 11, 5)
    states = [torch.from_numpy(p).to("cuda", _tdt(dt)) for _, _, p, _ in jobs]
    b = hs.hs_batch_create([(f, s, st) for (_, f, _, st), s in zip(jobs, states)])
    hs.hs_batch_launch(b)
    hs.hs_batch_launch(b)  # a second launch evolves by the same steps again
    torch.cuda.synchronize()
    tol = 1e-12 if dt == "c128" else 1e-5
    for (ham, f, p0, steps), got in zip(jobs, states):
        x, z, _ = O.parse_terms(ham.labels)
        want = O.evolve_direct(x, z, ham.coeffs, 0.8 / max(steps, 1) * 2 * steps, 2 * steps, p0) if steps else p0
        assert np.max(np.abs(got.cpu().numpy() - want)) <= tol
    b.close()


def test_batch_uneven_heisenberg_tfim_mix():
    """A reduced copy of the 256-instance mix: n 12..15, 20..40 steps, budgets 4..16."""
    jobs = W.batch256(n_jobs=24, n_lo=12, n_hi=15, seed=77)
    facs, states, refs = [], [], []
    for j in jobs:
        j.n_steps = min(j.n_steps, 40)
        f = hs.hs_build_factors(j.ham.labels, j.ham.coeffs, j.t, j.n_steps, j.budget, "c64")
        facs.append(f)
        states.append(torch.from_numpy(j.psi0).to("cuda", torch.complex64))
        r = torch.from_numpy(j.psi0).to("cuda", torch.complex64)
        hs.hs_evolve_ex(f, r, j.n_steps, method=hs.HS_METHOD_FUSED, tile_bits=9, rhs_block=1, low_bits=2)
        refs.append(r)
    b = hs.hs_batch_create([(f, s, j.n_steps) for f, s, j in zip(facs, states, jobs)], tile_bits=9, low_bits=2)
    assert b.n_separate == 0
    assert b.n_updates == sum(j.n_steps * f.n_factors * (1 << j.ham.n_qubits) for f, j in zip(facs, jobs))
    hs.hs_batch_launch(b)
    torch.cuda.synchronize()
    for s, r in zip(states, refs):
        assert torch.equal(s, r)
        assert abs((s.abs().double() ** 2).sum().item() - 1.0) < 1e-4
    b.close()


def test_batch_rejects_mixed_dtypes():
    f1 = hs.hs_build_factors(["XX", "ZZ"], [1.0, 1.0], 1.0, 2, 4, "c64")
    f2 = hs.hs_build_factors(["XX", "ZZ"], [1.0, 1.0], 1.0, 2, 4, "c128")
    s1 = torch.zeros(4, dtype=torch.complex64, device="cuda")
    s2 = torch.zeros(4, dtype=torch.complex128, device="cuda")
    with pytest.raises(hs.HSError) as e:
        hs.hs_batch_create([(f1, s1, 1), (f2, s2, 1)])
    assert e.value.code == hs.HS_EDTYPE


def test_batch_value_tables_bitwise_equal_to_staged_diagonals():
    jobs = W.batch256(n_jobs=12, n_lo=12, n_hi=15, seed=78)
    facs, s1, s2 = [], [], []
    for j in jobs:
        j.n_steps = min(j.n_steps, 30)
        facs.append(hs.hs_build_factors(j.ham.labels, j.ham.coeffs, j.t, j.n_steps, j.budget, "c64"))
        s1.append(torch.from_numpy(j.psi0).to("cuda", torch.complex64))
        s2.append(torch.from_numpy(j.psi0).to("cuda", torch.complex64))
    b1 = hs.hs_batch_create([(f, s, j.n_steps) for f, s, j in zip(facs, s1, jobs)])
    b2 = hs.hs_batch_create([(f, s, j.n_steps) for f, s, j in zip(facs, s2, jobs)], no_tables=True)
    hs.hs_batch_launch(b1)
    hs.hs_batch_launch(b2)
    torch.cuda.synchronize()
    for a, b in zip(s1, s2):
        assert torch.equal(a, b)
    b1.close()
    b2.close()
