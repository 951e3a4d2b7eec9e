"""Pins of the oracle's higher-order product formulas (second-order Strang and
fourth-order Suzuki, the paper's future-work formulas): dense products of scipy
exponentials in the stated stage order, the dt^2 / dt^4 error scaling against
eigh-exact evolution, time-reversal symmetry, and the first-order special case."""
import numpy as np
import pytest
import scipy.linalg

import oracle as O
from paper_2606_16959_gb300 import workloads as W
from test_oracle_pins import dense_h, dense_pauli


def _exact(H, t, psi):
    w, V = np.linalg.eigh(H)
    return (V * np.exp(-1j * t * w)) @ (V.conj().T @ psi)


def _dense_step(labels, coeffs, dt, order):
    """The step operator built from scipy expm of each term (rightmost acts first)."""
    N = 2 ** len(labels[0])
    U = np.eye(N, dtype=complex)
    for h, direction in O.step_stages(order, dt):
        idx = range(len(labels)) if direction > 0 else range(len(labels) - 1, -1, -1)
        for j in idx:
            U = scipy.linalg.expm(-1j * (coeffs[j] * h) * dense_pauli(labels[j])) @ U
    return U


HAMS = [
    ("heis4", lambda: W.heisenberg_chain(4, np.array([0.6, 1.1, 1.4, 0.9]), periodic=True)),
    ("tfim5", lambda: W.tfim_chain(5, 1.0, 0.8, periodic=False)),
    ("rand4", lambda: W.Hamiltonian("r", 4, ["XYZI", "IZXY", "YYII", "ZIIZ", "XIIX"],
                                    np.array([0.3, -0.8, 0.5, 1.1, -0.4]))),
]


@pytest.mark.parametrize("name,make", HAMS, ids=[h[0] for h in HAMS])
@pytest.mark.parametrize("order", [1, 2, 4])
def test_order_matches_dense_stage_product(name, make, order):
    ham = make()
    x, z, n = O.parse_terms(ham.labels)
    psi = W.gaussian_state(n, np.random.default_rng(4))
    t, steps = 0.9, 3
    got = O.evolve_direct_order(x, z, ham.coeffs, t, steps, psi, order)
    U = np.linalg.matrix_power(_dense_step(ham.labels, ham.coeffs, t / steps, order), steps)
    assert np.max(np.abs(got - U @ psi)) < 1e-12


def test_order_one_is_first_order():
    ham = W.tfim_chain(6, 1.0, 0.7)
    x, z, n = O.parse_terms(ham.labels)
    psi = W.gaussian_state(n, np.random.default_rng(2))
    a = O.evolve_direct_order(x, z, ham.coeffs, 1.0, 4, psi, 1)
    b = O.evolve_direct(x, z, ham.coeffs, 1.0, 4, psi)
    assert np.max(np.abs(a - b)) < 1e-14


@pytest.mark.parametrize("order,ratio", [(2, 4.0), (4, 16.0)])
def test_error_scaling(order, ratio):
    """Doubling the step count divides the error by ~2^order."""
    ham = W.heisenberg_chain(5, np.array([0.7, 1.2, 0.9, 1.3, 0.8]), periodic=True)
    x, z, n = O.parse_terms(ham.labels)
    H = dense_h(ham.labels, ham.coeffs)
    psi = W.gaussian_state(n, np.random.default_rng(9))
    t = 1.0
    want = _exact(H, t, psi)
    errs = [np.linalg.norm(O.evolve_direct_order(x, z, ham.coeffs, t, s, psi, order) - want) for s in (8, 16, 32)]
    for a, b in zip(errs, errs[1:]):
        assert 0.8 * ratio < a / b < 1.2 * ratio, errs
    # a first-order step count with the same cost is far less accurate
    e1 = np.linalg.norm(O.evolve_direct(x, z, ham.coeffs, t, 32, psi) - want)
    assert errs[-1] < e1


@pytest.mark.parametrize("order", [2, 4])
def test_time_reversal_symmetry(order):
    """Symmetric formulas satisfy S(dt) S(-dt) = I."""
    ham = W.heisenberg_chain(5, np.array([0.7, 1.2, 0.9, 1.3]), periodic=False)
    x, z, n = O.parse_terms(ham.labels)
    psi = W.gaussian_state(n, np.random.default_rng(1))
    fwd = O.evolve_direct_order(x, z, ham.coeffs, 0.6, 1, psi, order)
    back = O.evolve_direct_order(x, z, ham.coeffs, -0.6, 1, fwd, order)
    assert np.max(np.abs(back - psi)) < 1e-13
    # the first-order formula is not symmetric
    f1 = O.evolve_direct_order(x, z, ham.coeffs, 0.6, 1, psi, 1)
    b1 = O.evolve_direct_order(x, z, ham.coeffs, -0.6, 1, f1, 1)
    assert np.max(np.abs(b1 - psi)) > 1e-4
