"""Pins of the oracle's time-dependent evolution H(t) = H0 + f(t) H1 (the
paper's outlook on time-dependent Hamiltonians): the constant-drive special
case, dense per-step products of scipy exponentials, exact phases for diagonal
H0 and H1, convergence to the time-ordered exponential from an independent ODE
solver with the step-count scaling of each order, and norm preservation."""
import numpy as np
import pytest
import scipy.integrate
import scipy.linalg

import oracle as O
from paper_2606_16959_gb300 import workloads as W
from test_oracle_pins import dense_h, dense_pauli


def _drive(t):
    return np.cos(2.3 * t) + 0.4 * t


def _dense_td(labels, a, b, fvals, t, order):
    """Product over steps of the order's stage products of scipy expm, step s
    with coefficients a_j + f_s b_j (rightmost factor acts first)."""
    N = 2 ** len(labels[0])
    dt = t / len(fvals)
    U = np.eye(N, dtype=complex)
    for f in fvals:
        for h, direction in O.step_stages(order, dt):
            idx = range(len(labels)) if direction > 0 else range(len(labels) - 1, -1, -1)
            for j in idx:
                c = a[j] + f * b[j]
                U = scipy.linalg.expm(-1j * (c * h) * dense_pauli(labels[j])) @ U
    return U


def _tfim_drive(n=4):
    return W.driven_tfim(n, 1.0, 0.9, periodic=False)


@pytest.mark.parametrize("order", [1, 2, 4])
def test_td_matches_dense_per_step_product(order):
    ham = W.DrivenHamiltonian("r", 4, ["XYZI", "IZXY", "YYII", "ZIIZ", "XIIX", "IIXZ"],
                              np.array([0.3, 0.0, 0.5, 1.1, -0.4, 0.2]),
                              np.array([0.0, -0.8, 0.25, 0.0, 0.6, -0.3]))
    x, z, n = O.parse_terms(ham.labels)
    psi = W.gaussian_state(n, np.random.default_rng(3))
    fv = np.array([0.2, -1.3, 0.7, 2.1])
    got = O.evolve_direct_td(x, z, ham.a, ham.b, fv, 0.8, psi, order)
    want = _dense_td(ham.labels, ham.a, ham.b, fv, 0.8, order) @ psi
    assert np.max(np.abs(got - want)) < 1e-12


@pytest.mark.parametrize("order", [1, 2, 4])
def test_td_constant_drive_is_static_evolution(order):
    ham = _tfim_drive(6)
    x, z, n = O.parse_terms(ham.labels)
    psi = W.gaussian_state(n, np.random.default_rng(5))
    f = 0.65
    got = O.evolve_direct_td(x, z, ham.a, ham.b, np.full(5, f), 1.1, psi, order)
    want = O.evolve_direct_order(x, z, ham.a + f * ham.b, 1.1, 5, psi, order)
    assert np.max(np.abs(got - want)) < 1e-14


def test_td_diagonal_exact_phases():
    """Diagonal H0 and H1 commute at all times: the evolution is the phase
    exp(-i (t E0(b) + dt sum_s f_s E1(b))) per basis state b, for any step count."""
    n = 5
    labels = ["IIIIZ", "IIZZI", "ZIIIZ", "IZZII", "IIIII", "ZZIII"]
    a = np.array([0.4, -0.7, 0.0, 1.2, 0.3, 0.0])
    b = np.array([0.0, 0.5, -0.9, 0.0, 0.1, 0.35])
    x, z, _ = O.parse_terms(labels)
    psi = W.gaussian_state(n, np.random.default_rng(8))
    E0 = np.real(np.diag(dense_h(labels, a)))
    E1 = np.real(np.diag(dense_h(labels, b)))
    t = 1.7
    for steps in (1, 3, 7):
        fv = W.midpoint_samples(_drive, t, steps)
        want = np.exp(-1j * (t * E0 + (t / steps) * np.sum(fv) * E1)) * psi
        for order in (1, 2):
            got = O.evolve_direct_td(x, z, a, b, fv, t, psi, order)
            assert np.max(np.abs(got - want)) < 1e-12


def _time_ordered(labels, a, b, t, psi):
    """i dpsi/dt = (H0 + f(t) H1) psi by an 8th-order Runge-Kutta solver."""
    H0, H1 = dense_h(labels, a), dense_h(labels, b)
    sol = scipy.integrate.solve_ivp(lambda s, y: -1j * ((H0 + _drive(s) * H1) @ y), (0.0, t),
                                    psi.astype(complex), method="DOP853", rtol=1e-12, atol=1e-13)
    return sol.y[:, -1]


@pytest.mark.parametrize("order,ratio", [(1, 2.0), (2, 4.0)])
def test_td_converges_to_time_ordered_exponential(order, ratio):
    """With midpoint samples, doubling the step count divides the error against
    the time-ordered exponential by ~2 (first order) or ~4 (Strang)."""
    ham = _tfim_drive(4)
    x, z, n = O.parse_terms(ham.labels)
    psi = W.gaussian_state(n, np.random.default_rng(11))
    t = 1.0
    want = _time_ordered(ham.labels, ham.a, ham.b, t, psi)
    errs = []
    for steps in (16, 32, 64):
        fv = W.midpoint_samples(_drive, t, steps)
        errs.append(np.linalg.norm(O.evolve_direct_td(x, z, ham.a, ham.b, fv, t, psi, order) - want))
    for e1, e2 in zip(errs, errs[1:]):
        assert 0.75 * ratio < e1 / e2 < 1.25 * ratio, errs
    # ignoring the drive (f frozen at its t=0 value) does not converge
    fv0 = np.full(64, _drive(0.0))
    e_frozen = np.linalg.norm(O.evolve_direct_td(x, z, ham.a, ham.b, fv0, t, psi, order) - want)
    assert e_frozen > 20 * errs[-1]


def test_td_preserves_norm_and_multi_rhs():
    ham = W.anneal_maxcut(8, seed=21)
    x, z, n = O.parse_terms(ham.labels)
    rng = np.random.default_rng(2)
    psi = np.stack([W.plus_state(n), W.gaussian_state(n, rng)])
    fv = W.midpoint_samples(lambda s: s / 1.5, 1.5, 6)
    out = O.evolve_direct_td(x, z, ham.a, ham.b, fv, 1.5, psi)
    assert np.allclose(np.linalg.norm(out, axis=1), 1.0, atol=1e-13)
    for r in range(2):
        one = O.evolve_direct_td(x, z, ham.a, ham.b, fv, 1.5, psi[r])
        assert np.max(np.abs(one - out[r])) == 0.0


def test_anneal_endpoints():
    """The annealing family is the mixer at s = 0 and MaxCut's H_C at s = 1."""
    ham = W.anneal_maxcut(6, seed=4, mixer=0.5)
    mc = W.maxcut_3regular(6, 4, mixer=0.0)
    H0 = dense_h(ham.labels, ham.a)
    H1 = dense_h(ham.labels, ham.a + ham.b)
    mix = sum(0.5 * dense_pauli(W.label_of(6, {i: "X"})) for i in range(6))
    assert np.allclose(H0, mix)
    assert np.allclose(H1, dense_h(mc.labels, mc.coeffs))
