"""GPU parity of the single-factor Taylor mode (include/hs_dia.h) against the
FP64 oracle (oracle/taylor.py): H in the compact layout (offsets and values
bit-exact), SpGEMM, the truncated Taylor exponential of Alg. 2, the budgeted
step search of Eq. 5, SpMV and the Alg. 3 evolution, plus edge cases."""
import numpy as np
import pytest

import oracle as O
from oracle import taylor as OT
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


def _odia(ham):
    x, z, n = O.parse_terms(ham.labels)
    return OT.ham_dia(x, z, ham.coeffs, n)


def _same_structure(g, o):
    offs, vals = g.get()
    assert list(offs) == o.offsets
    return vals


def _max_rel(vals, o):
    top = max(float(np.max(np.abs(v))) for v in o.diags.values())
    return max(float(np.max(np.abs(vals[d] - o.diags[d]))) for d in o.diags) / max(top, 1e-300)


def _random_labels(rng, n, m):
    return ["".join(rng.choice(list("IXYZ"), p=[0.4, 0.2, 0.2, 0.2], size=n)) for _ in range(m)]


# ---------------------------------------------------------------------------
# H in the compact layout: bit-exact
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(8))
def test_h_from_terms_bit_exact(seed):
    rng = np.random.default_rng(3000 + seed)
    n = int(rng.integers(1, 11))
    labels = _random_labels(rng, n, int(rng.integers(1, 14)))
    labels += labels[: int(rng.integers(0, 3))]           # duplicate terms compose
    coeffs = rng.uniform(-1, 1, len(labels))
    if len(labels) > 1:
        coeffs[-1] = -coeffs[0] if labels[-1] == labels[0] else coeffs[-1]
    ham = W.Hamiltonian("random", n, labels, coeffs)
    g = hs.hs_dia_from_terms(labels, coeffs)
    o = _odia(ham)
    vals = _same_structure(g, o)
    for d in o.diags:
        assert np.array_equal(vals[d], o.diags[d]), d
    assert g.nnz == o.nnz()


@pytest.mark.parametrize("n,periodic", [(12, True), (13, False), (16, True)])
def test_h_chains_counts_and_values(n, periodic):
    J = np.linspace(0.5, 1.5, n if periodic else n - 1)
    for ham in (W.heisenberg_chain(n, J, periodic=periodic), W.tfim_chain(n, 1.0, 0.7, periodic=periodic)):
        g = hs.hs_dia_from_terms(ham.labels, ham.coeffs)
        o = _odia(ham)
        vals = _same_structure(g, o)
        assert all(np.array_equal(vals[d], o.diags[d]) for d in o.diags)
        # Tab. 3 closed forms: Heisenberg 1 + 2 * bonds (XX+YY cancel on +-3*2^i), TFIM 2n + 1
        bonds = n if periodic else n - 1
        want = 1 + 2 * bonds if ham.family == "heisenberg" else 2 * n + 1
        assert g.n_diags == want


def test_dia_create_roundtrip_and_convert():
    rng = np.random.default_rng(11)
    N = 1 << 7
    diags = {d: rng.normal(size=N - abs(d)) + 1j * rng.normal(size=N - abs(d)) for d in (5, -1, 0, 127, -64)}
    a = hs.hs_dia_create(7, diags)
    offs, vals = a.get()
    assert list(offs) == [0, -1, 5, -64, 127]
    assert all(np.array_equal(vals[d], diags[d]) for d in diags)
    b = hs.hs_dia_convert(a, "c64")
    assert b.dtype == "c64"
    _, v64 = b.get()
    for d in diags:
        assert np.array_equal(v64[d], diags[d].astype(np.complex64).astype(np.complex128))


# ---------------------------------------------------------------------------
# SpGEMM and the Taylor exponential
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_spgemm_matches_oracle(seed):
    rng = np.random.default_rng(4000 + seed)
    n = int(rng.integers(2, 11))
    N = 1 << n
    def rand():
        k = int(rng.integers(1, min(2 * N - 1, 12) + 1))
        offs = rng.choice(np.arange(-(N - 1), N), size=k, replace=False)
        return {int(d): rng.normal(size=N - abs(int(d))) + 1j * rng.normal(size=N - abs(int(d))) for d in offs}
    da, db = rand(), rand()
    C, fro = hs.hs_spgemm(hs.hs_dia_create(n, da), hs.hs_dia_create(n, db))
    oc = OT.spgemm(OT.Dia(N, da), OT.Dia(N, db))
    vals = _same_structure(C, oc)
    assert _max_rel(vals, oc) <= 1e-13
    assert fro == pytest.approx(OT.fro(oc), rel=1e-12)


def test_spgemm_heisenberg_square_drops_cancelled_diagonals():
    ham = W.heisenberg_chain(12, np.linspace(0.5, 1.5, 12), periodic=True)
    H = hs.hs_dia_from_terms(ham.labels, ham.coeffs)
    H2, _ = hs.hs_spgemm(H, H)
    o = _odia(ham)
    o2 = OT.spgemm(o, o)
    vals = _same_structure(H2, o2)
    assert _max_rel(vals, o2) <= 1e-13


SPME_CASES = [
    ("tfim8", lambda: W.tfim_chain(8, 1.0, 0.7, periodic=False), 0.3),
    ("tfim10", lambda: W.tfim_chain(10, 1.0, 1.0, periodic=True), 0.05),
    ("heis8", lambda: W.heisenberg_chain(8, np.linspace(0.5, 1.5, 8), periodic=True), 0.2),
    ("heis11", lambda: W.heisenberg_chain(11, np.linspace(0.5, 1.5, 10), periodic=False), 0.1),
]


@pytest.mark.parametrize("name,make,t", SPME_CASES, ids=[c[0] for c in SPME_CASES])
def test_spme_matches_oracle(name, make, t):
    ham = make()
    U, K, ok = hs.hs_spme(hs.hs_dia_from_terms(ham.labels, ham.coeffs), t)
    oU, oK, ook = OT.expm_taylor(_odia(ham), t)
    assert (K, ok) == (oK, ook)
    vals = _same_structure(U, oU)
    assert _max_rel(vals, oU) <= 1e-12


def test_spme_diagonal_is_exact():
    ham = W.maxcut(10, W.random_regular_graph(10, 3, np.random.default_rng(77)),
                   np.random.default_rng(5).uniform(0, 1, 15), mixer=0.0)
    U, K, ok = hs.hs_spme(hs.hs_dia_from_terms(ham.labels, ham.coeffs), 1.3)
    assert K == 0 and ok and U.n_diags == 1
    oU, _, _ = OT.expm(_odia(ham), 1.3)
    _, vals = U.get()
    assert np.max(np.abs(vals[0] - oU.diags[0])) <= 1e-14


def test_spme_not_converged_reports_it():
    ham = W.tfim_chain(6, 1.0, 1.0)
    U, K, ok = hs.hs_spme(hs.hs_dia_from_terms(ham.labels, ham.coeffs), 2.0, 1e-6, 3)
    oU, oK, ook = OT.expm_taylor(_odia(ham), 2.0, 1e-6, 3)
    assert (K, ok) == (oK, ook) == (3, False)
    _same_structure(U, oU)


# ---------------------------------------------------------------------------
# Step search (Eq. 5)
# ---------------------------------------------------------------------------

STEP_CASES = [
    ("tfim4", lambda: W.tfim_chain(4, 1.0, 0.7, periodic=False), 1.0, 29),
    ("heis4_one_step", lambda: W.heisenberg_chain(4, np.array([0.6, 1.1, 1.4, 0.9]), periodic=True), 1.0, 17),
    ("heis6_open", lambda: W.heisenberg_chain(6, np.ones(5), periodic=False), 1.0, 85),
    ("tfim6", lambda: W.tfim_chain(6, 1.0, 1.0, periodic=False), 1.0, 125),
    ("heis9", lambda: W.heisenberg_chain(9, np.linspace(0.5, 1.5, 9), periodic=True), 1.0, 200),
]


@pytest.mark.parametrize("name,make,t,budget", STEP_CASES, ids=[c[0] for c in STEP_CASES])
def test_estimate_timesteps_matches_oracle(name, make, t, budget):
    ham = make()
    r = hs.hs_estimate_timesteps(hs.hs_dia_from_terms(ham.labels, ham.coeffs), t, budget)
    assert r == OT.estimate_timesteps(_odia(ham), t, budget)


def test_estimate_timesteps_diagonal_and_infeasible():
    zz = W.Hamiltonian("zz", 3, ["ZZI", "IZZ"], np.array([0.5, -1.0]))
    assert hs.hs_estimate_timesteps(hs.hs_dia_from_terms(zz.labels, zz.coeffs), 5.0, 1) == 1
    ham = W.tfim_chain(5, 1.0, 1.0)
    with pytest.raises(hs.HSError) as e:
        hs.hs_estimate_timesteps(hs.hs_dia_from_terms(ham.labels, ham.coeffs), 1.0, 3, max_steps=64)
    assert e.value.code == hs.HS_EINVAL


# ---------------------------------------------------------------------------
# SpMV and the Alg. 3 evolution
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n_rhs", [1, 2, 3, 5])
@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_spmv_matches_oracle(n_rhs, dt):
    ham = W.heisenberg_chain(11, np.linspace(0.5, 1.5, 11), periodic=True)
    H = hs.hs_dia_from_terms(ham.labels, ham.coeffs)
    A = H if dt == "c128" else hs.hs_dia_convert(H, "c64")
    rng = np.random.default_rng(n_rhs)
    x = np.stack([W.gaussian_state(11, rng) for _ in range(n_rhs)])
    tdt = torch.complex128 if dt == "c128" else torch.complex64
    xd = torch.from_numpy(x).to("cuda", tdt)
    yd = torch.empty_like(xd)
    hs.hs_spmv(A, xd, yd)
    want = OT.spmv(_odia(ham), x)
    got = yd.cpu().numpy().astype(np.complex128)
    tol = 1e-12 if dt == "c128" else 1e-5
    assert np.max(np.abs(got - want)) <= tol * max(1.0, np.max(np.abs(want)))


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_taylor_evolution_matches_oracle(dt):
    """Alg. 3: r from the budget, U = SpME(H, t/r), psi <- U^r psi."""
    ham = W.heisenberg_chain(9, np.linspace(0.5, 1.5, 9), periodic=True)
    H = hs.hs_dia_from_terms(ham.labels, ham.coeffs)
    t, budget = 1.0, 200
    r = hs.hs_estimate_timesteps(H, t, budget)
    U, K, ok = hs.hs_spme(H, t / r)
    assert ok
    Ue = U if dt == "c128" else hs.hs_dia_convert(U, "c64")
    rng = np.random.default_rng(9)
    psi = np.stack([W.gaussian_state(9, rng) for _ in range(3)])
    tdt = torch.complex128 if dt == "c128" else torch.complex64
    pd = torch.from_numpy(psi).to("cuda", tdt)
    hs.hs_dia_evolve(Ue, pd, r)
    oU, _, _ = OT.expm_taylor(_odia(ham), t / r)
    want = OT.evolve(oU, psi, r)
    got = pd.cpu().numpy().astype(np.complex128)
    if dt == "c128":
        assert np.max(np.abs(got - want)) <= 1e-12
    else:
        assert np.max(np.abs(got - want)) <= 1e-5
        for k in range(3):
            assert 1.0 - O.fidelity(got[k], want[k]) <= 1e-6


@pytest.mark.parametrize("steps", [0, 1, 4, 7])
def test_dia_evolve_diagonal_in_place(steps):
    ham = W.maxcut(8, W.random_regular_graph(8, 3, np.random.default_rng(5)), np.linspace(0.1, 0.9, 12), mixer=0.0)
    U, _, _ = hs.hs_spme(hs.hs_dia_from_terms(ham.labels, ham.coeffs), 0.7)
    psi = W.gaussian_state(8, np.random.default_rng(1))
    pd = torch.from_numpy(psi).to("cuda", torch.complex128)
    hs.hs_dia_evolve(U, pd, steps)
    oU, _, _ = OT.expm(_odia(ham), 0.7)
    assert np.max(np.abs(pd.cpu().numpy() - OT.evolve(oU, psi, steps))) <= 1e-13


def test_taylor_argument_errors():
    with pytest.raises(hs.HSError) as e:
        hs.hs_dia_from_terms([], [])
    assert e.value.code == hs.HS_EINVAL
    with pytest.raises(hs.HSError) as e:
        hs.hs_dia_from_terms(["XQ"], [1.0])
    assert e.value.code == hs.HS_EINVAL
    a = hs.hs_dia_from_terms(["XX", "ZZ"], [1.0, 0.5])
    b = hs.hs_dia_from_terms(["XXX"], [1.0])
    with pytest.raises(hs.HSError) as e:
        hs.hs_spgemm(a, b)
    assert e.value.code == hs.HS_EINVAL
    with pytest.raises(hs.HSError) as e:
        hs.hs_spme(hs.hs_dia_convert(a, "c64"), 1.0)
    assert e.value.code == hs.HS_EDTYPE
    with pytest.raises(hs.HSError) as e:
        hs.hs_spme(a, 1.0, 0.0)
    assert e.value.code == hs.HS_EINVAL


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_expectation_matches_oracle_and_is_conserved(dt):
    """<psi|H|psi> against the oracle; the exact-Taylor evolution of Alg. 3
    conserves it to the propagator's accuracy."""
    ham = W.heisenberg_chain(10, np.linspace(0.5, 1.5, 10), periodic=True)
    H = hs.hs_dia_from_terms(ham.labels, ham.coeffs)
    Hd = H if dt == "c128" else hs.hs_dia_convert(H, "c64")
    rng = np.random.default_rng(12)
    psi = np.stack([W.gaussian_state(10, rng) for _ in range(3)])
    tdt = torch.complex128 if dt == "c128" else torch.complex64
    pd = torch.from_numpy(psi).to("cuda", tdt)
    vals, norms = hs.hs_expectation(Hd, pd)
    x = psi if dt == "c128" else psi.astype(np.complex64).astype(np.complex128)
    want = OT.expectation(_odia(ham), x)
    tol = 1e-12 if dt == "c128" else 1e-5
    assert np.max(np.abs(vals - want)) <= tol * max(1.0, np.max(np.abs(want)))
    assert np.max(np.abs(norms - 1.0)) <= (1e-12 if dt == "c128" else 1e-6)
    # conservation under the evolution by a propagator accurate to ~1e-13 per step
    U, _, ok = hs.hs_spme(H, 0.01, 1e-13, 200)
    assert ok
    p2 = torch.from_numpy(psi).to("cuda", torch.complex128)
    hs.hs_dia_evolve(U, p2, 50)
    v2, n2 = hs.hs_expectation(H, p2)
    e0 = OT.expectation(_odia(ham), psi) / np.sum(np.abs(psi) ** 2, axis=1)
    assert np.max(np.abs(v2 / n2 - e0)) < 1e-9
