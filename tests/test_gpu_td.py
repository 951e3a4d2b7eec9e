"""GPU parity of time-dependent evolution under H(t) = H0 + f(t) H1 against the
oracle's term-by-term evolution with the same per-step drive samples; factor
values after a drive rebuild against a static build of H0 + f H1 (bitwise);
graph replays with new drive samples; argument errors."""
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


def _drive(s):
    return np.cos(2.3 * s) + 0.4 * s


def _random_driven(rng, n):
    """Heisenberg chain whose YY terms and a random subset of the others are
    driven (a_j and b_j both nonzero on some terms)."""
    base = W.heisenberg_chain(n, rng.uniform(0.5, 1.5, n), periodic=True)
    m = len(base.labels)
    a = base.coeffs.copy()
    b = np.where(rng.uniform(size=m) < 0.4, rng.uniform(-1, 1, m), 0.0)
    b[1::3] = rng.uniform(0.2, 0.8, m // 3)
    return W.DrivenHamiltonian("heis_driven", n, list(base.labels), a, b)


def _hams(rng):
    return [("tfim11", W.driven_tfim(11, 1.0, 0.9), 4),
            ("anneal12", W.anneal_maxcut(12, seed=77), 4),
            ("heis10", _random_driven(rng, 10), 8)]


def _close(got, want, dt):
    if dt == "c128":
        return np.max(np.abs(got - want)) <= 1e-12
    ok = np.max(np.abs(got - want)) <= 1e-5
    return ok and max(1 - O.fidelity(got[k], want[k]) for k in range(got.shape[0])) <= 1e-6


@pytest.mark.parametrize("order", [1, 2, 4])
@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_td_matches_oracle(order, dt):
    rng = np.random.default_rng(700 + order)
    tdt = torch.complex128 if dt == "c128" else torch.complex64
    t, steps = 0.9, 6
    fv = W.midpoint_samples(_drive, t, steps)
    for name, ham, budget in _hams(rng):
        x, z, n = O.parse_terms(ham.labels)
        psi = np.stack([W.gaussian_state(n, rng) for _ in range(2)])
        want = O.evolve_direct_td(x, z, ham.a, ham.b, fv, t, psi, order)
        f = hs.hs_build_factors_td(x, z, ham.a, ham.b, n, t, steps, budget, dt, order=order)
        # register sweeps first: they leave the stored diagonals to be rebuilt
        # on first read, which the schedules after them do
        for kw in (dict(method=hs.HS_METHOD_REG), dict(method=hs.HS_METHOD_REG, use_graph=True),
                   dict(), dict(method=hs.HS_METHOD_PLAIN), dict(use_graph=True), dict(no_tables=True),
                   dict(method=hs.HS_METHOD_FUSED, tile_bits=8, rhs_block=1, low_bits=1)):
            pd = torch.from_numpy(psi).to("cuda", tdt)
            hs.hs_evolve_td(f, pd, fv, **kw)
            got = pd.cpu().numpy().astype(np.complex128)
            assert _close(got, want, dt), (name, kw, np.max(np.abs(got - want)))
        f.close()


def _values(f):
    return [f.factor(g)[3] for g in range(f.n_factors)]


@pytest.mark.parametrize("order", [1, 2])
def test_drive_rebuild_equals_static_build_bitwise(order):
    """Values rebuilt for a drive value f equal those of a static build with
    coefficients a + f b (same rounding of the angles), for every factor."""
    rng = np.random.default_rng(31)
    for name, ham, budget in _hams(rng):
        x, z, n = O.parse_terms(ham.labels)
        for dt in ("c128", "c64"):
            f = hs.hs_build_factors_td(x, z, ham.a, ham.b, n, 1.3, 7, budget, dt, order=order)
            s0 = hs.hs_build_factors_masks(x, z, ham.a, n, 1.3, 7, budget, dt, order=order)
            for a, b in zip(_values(f), _values(s0)):
                assert np.array_equal(a, b), name
            fval = -0.8125
            hs.hs_factors_set_drive(f, fval)
            s1 = hs.hs_build_factors_masks(x, z, ham.a + fval * ham.b, n, 1.3, 7, budget, dt, order=order)
            for a, b in zip(_values(f), _values(s1)):
                assert np.array_equal(a, b), name
            # after an evolution, the values are those of the last drive sample
            psi = torch.from_numpy(W.gaussian_state(n, rng)).to("cuda", torch.complex128 if dt == "c128"
                                                                  else torch.complex64)
            fv = np.array([0.3, 1.7, -0.4, 2.25])
            hs.hs_evolve_td(f, psi, fv)
            s2 = hs.hs_build_factors_masks(x, z, ham.a + fv[-1] * ham.b, n, 1.3, 7, budget, dt, order=order)
            for a, b in zip(_values(f), _values(s2)):
                assert np.array_equal(a, b), name
            for o in (f, s0, s1, s2):
                o.close()


def test_constant_drive_matches_static_evolution():
    rng = np.random.default_rng(5)
    ham = W.driven_tfim(13, 1.0, 1.1)
    x, z, n = O.parse_terms(ham.labels)
    psi = np.stack([W.gaussian_state(n, rng) for _ in range(3)])
    fval = 0.55
    f = hs.hs_build_factors_td(x, z, ham.a, ham.b, n, 1.0, 9, 4, "c128")
    s = hs.hs_build_factors_masks(x, z, ham.a + fval * ham.b, n, 1.0, 9, 4, "c128")
    p1 = torch.from_numpy(psi).to("cuda")
    p2 = torch.from_numpy(psi).to("cuda")
    hs.hs_evolve_td(f, p1, np.full(9, fval))
    hs.hs_evolve(s, p2, 9)
    assert torch.max(torch.abs(p1 - p2)).item() <= 1e-13
    f.close()
    s.close()


def test_graph_replay_reads_new_drive():
    rng = np.random.default_rng(9)
    ham = W.anneal_maxcut(14, seed=3)
    x, z, n = O.parse_terms(ham.labels)
    psi = np.stack([W.plus_state(n), W.gaussian_state(n, rng)])
    t = 1.2
    f = hs.hs_build_factors_td(x, z, ham.a, ham.b, n, t, 8, 4, "c64")
    pd = torch.empty((2, 1 << n), dtype=torch.complex64, device="cuda")
    for ramp in (lambda s: s / t, lambda s: 1.0 - s / t, _drive):
        fv = W.midpoint_samples(ramp, t, 8)
        pd.copy_(torch.from_numpy(psi))
        hs.hs_evolve_td(f, pd, fv, use_graph=True)
        want = O.evolve_direct_td(x, z, ham.a, ham.b, fv, t, psi)
        assert _close(pd.cpu().numpy().astype(np.complex128), want, "c64")
    # more steps than the drive buffer held: it grows and the graphs are
    # re-captured; each step keeps the factor set's dt = t / 8, so 80 steps span 10 t
    fv = W.midpoint_samples(_drive, 10 * t, 80)
    pd.copy_(torch.from_numpy(psi))
    hs.hs_evolve_td(f, pd, fv, use_graph=True)
    want = O.evolve_direct_td(x, z, ham.a, ham.b, fv, 10 * t, psi)
    assert _close(pd.cpu().numpy().astype(np.complex128), want, "c64")
    f.close()


def test_anneal_norm_at_size():
    """MaxCut annealing at 22 qubits, 8 states, complex64: the state norms stay
    1 (FP64 reduction) and state 0 matches the oracle on 3 steps."""
    ham = W.anneal_maxcut(22, seed=1003)
    x, z, n = O.parse_terms(ham.labels)
    rng = np.random.default_rng(4)
    psi = np.stack([W.plus_state(n)] + [W.gaussian_state(n, rng) for _ in range(7)])
    t = 2.0
    f = hs.hs_build_factors_td(x, z, ham.a, ham.b, n, t, 3, 4, "c64")
    fv = W.midpoint_samples(lambda s: s / t, t, 3)
    pd = torch.from_numpy(psi).to("cuda", torch.complex64)
    hs.hs_evolve_td(f, pd, fv)
    for k in range(8):
        _, na, _ = hs.hs_fidelity(pd[k], pd[k])
        assert abs(na - 1.0) < 1e-5
    want = O.evolve_direct_td(x, z, ham.a, ham.b, fv, t, psi[0])
    got = pd[0].cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(got - want)) <= 1e-5 and 1 - O.fidelity(got, want) <= 1e-6
    f.close()


def test_td_errors():
    ham = W.driven_tfim(8)
    x, z, n = O.parse_terms(ham.labels)
    s = hs.hs_build_factors_masks(x, z, ham.a, n, 1.0, 4, 4, "c64")
    psi = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    with pytest.raises(hs.HSError):
        hs.hs_evolve_td(s, psi, np.zeros(4))
    with pytest.raises(hs.HSError):
        hs.hs_factors_set_drive(s, 0.5)
    bad = ham.b.copy()
    bad[2] = np.nan
    with pytest.raises(hs.HSError):
        hs.hs_build_factors_td(x, z, ham.a, bad, n, 1.0, 4, 4, "c64")
    f = hs.hs_build_factors_td(x, z, ham.a, ham.b, n, 1.0, 4, 4, "c64")
    with pytest.raises(hs.HSError):
        hs.hs_evolve_td(f, psi, np.array([0.1, np.inf]))
    with pytest.raises(hs.HSError):
        hs.hs_factors_set_drive(f, np.nan)
    hs.hs_evolve_td(f, psi, np.zeros(0))  # zero steps: no-op
    s.close()
    f.close()
