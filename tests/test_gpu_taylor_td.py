"""GPU parity of time-dependent evolution in the single-factor Taylor mode
(hs_dia_evolve_td) against the oracle's evolve_td with the same drive samples:
complex128 at 1e-12, complex64 at 1e-5 with infidelity <= 1e-6, the exact
diagonal path, and argument errors."""
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


def _drive(s):
    return np.cos(2.3 * s) + 0.4 * s


def _cases():
    rng = np.random.default_rng(77)
    heis = W.heisenberg_chain(5, rng.uniform(0.5, 1.5, 5), periodic=True)
    b = np.zeros(len(heis.labels))
    b[2::3] = rng.uniform(0.3, 0.9, len(b[2::3]))  # the ZZ terms are driven
    return [("tfim6", W.driven_tfim(6, 1.0, 0.9)),
            ("heis5", W.DrivenHamiltonian("heis_driven", 5, list(heis.labels), heis.coeffs.copy(), b))]


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_dia_evolve_td_matches_oracle(dt):
    rng = np.random.default_rng(5)
    t, steps = 0.6, 5
    fv = W.midpoint_samples(_drive, t, steps)
    tdt = torch.complex128 if dt == "c128" else torch.complex64
    for name, ham in _cases():
        x, z, n = O.parse_terms(ham.labels)
        psi = np.stack([W.gaussian_state(n, rng) for _ in range(2)])
        want = np.stack([OT.evolve_td(x, z, ham.a, ham.b, fv, n, t, psi[r]) for r in range(2)])
        pd = torch.from_numpy(psi).to("cuda", tdt)
        hs.hs_dia_evolve_td(x, z, ham.a, ham.b, n, t, fv, pd)
        got = pd.cpu().numpy().astype(np.complex128)
        if dt == "c128":
            assert np.max(np.abs(got - want)) <= 1e-12, name
        else:
            assert np.max(np.abs(got - want)) <= 1e-5, name
            assert max(1 - O.fidelity(got[k], want[k]) for k in range(2)) <= 1e-6, name


def test_dia_evolve_td_diagonal_exact():
    labels = ["IIIIZ", "IIZZI", "ZIIIZ", "IZZII", "IIIII", "ZZIII"]
    a = np.array([0.4, -0.7, 0.0, 1.2, 0.3, 0.0])
    b = np.array([0.0, 0.5, -0.9, 0.0, 0.1, 0.35])
    x, z, n = O.parse_terms(labels)
    psi = W.gaussian_state(n, np.random.default_rng(8))
    t = 1.7
    fv = W.midpoint_samples(_drive, t, 4)
    want = OT.evolve_td(x, z, a, b, fv, n, t, psi)
    pd = torch.from_numpy(psi).to("cuda")
    hs.hs_dia_evolve_td(x, z, a, b, n, t, fv, pd)
    assert np.max(np.abs(pd.cpu().numpy() - want)) <= 1e-12


def test_dia_evolve_td_errors():
    ham = W.driven_tfim(4)
    x, z, n = O.parse_terms(ham.labels)
    psi = torch.zeros(1 << n, dtype=torch.complex128, device="cuda")
    with pytest.raises(hs.HSError):
        hs.hs_dia_evolve_td(x, z, ham.a, ham.b, n, 1.0, np.array([0.1, np.nan]), psi)
    with pytest.raises(hs.HSError):
        hs.hs_dia_evolve_td(x, z, ham.a, ham.b, n, -1.0, np.array([0.1]), psi)
    with pytest.raises(hs.HSError):
        hs.hs_dia_evolve_td(x, z, ham.a, ham.b, n, 1.0, np.array([0.1]), psi, tol=0.0)
    hs.hs_dia_evolve_td(x, z, ham.a, ham.b, n, 1.0, np.zeros(0), psi)  # zero steps: no-op
    assert torch.count_nonzero(psi).item() == 0
