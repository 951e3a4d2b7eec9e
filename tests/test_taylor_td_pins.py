"""Pins of the Taylor-mode oracle for time-dependent H(t) = H0 + f(t) H1:
H(f) against dense Kronecker sums, per-step evolution against eigh
exponentials, exact phases for diagonal H0 and H1, second-order convergence of
the midpoint samples to an independent ODE solution, and the shared step count
against a brute-force scan of dense Taylor sums."""
import numpy as np
import pytest
import scipy.integrate

import oracle as O
from oracle import taylor as OT
from paper_2606_16959_gb300 import workloads as W
from test_oracle_pins import dense_h
from test_taylor_pins import _dense_diag_count


def _drive(s):
    return np.cos(2.3 * s) + 0.4 * s


def _exact_expm(H, t):
    w, V = np.linalg.eigh(H)
    return (V * np.exp(-1j * t * w)) @ V.conj().T


def _ham():
    return W.driven_tfim(4, 1.0, 0.9, periodic=False)


def test_ham_dia_td_equals_kronecker_sum():
    ham = W.DrivenHamiltonian("r", 4, ["XYZI", "IZXY", "YYII", "ZIIZ", "XIIX", "IIXZ"],
                              np.array([0.3, 0.0, 0.5, 1.1, -0.4, 0.2]),
                              np.array([0.0, -0.8, 0.25, 0.0, 0.6, -0.3]))
    x, z, n = O.parse_terms(ham.labels)
    for f in (0.0, -1.25, 0.7):
        A = OT.ham_dia_td(x, z, ham.a, ham.b, f, n)
        assert np.array_equal(OT.to_dense(A), dense_h(ham.labels, ham.a + f * ham.b))


def test_drive_that_cancels_terms_drops_their_diagonals():
    labels = ["ZZ", "XI"]
    x, z, n = O.parse_terms(labels)
    a, b = np.array([1.0, 0.5]), np.array([0.0, 1.0])
    assert OT.ham_dia_td(x, z, a, b, 0.0, n).offsets == [0, -2, 2]
    assert OT.ham_dia_td(x, z, a, b, -0.5, n).offsets == [0]


@pytest.mark.parametrize("tol", [1e-15, 1e-6])
def test_evolve_td_matches_dense_per_step(tol):
    ham = _ham()
    x, z, n = O.parse_terms(ham.labels)
    psi = W.gaussian_state(n, np.random.default_rng(3))
    fv = np.array([0.2, -1.3, 0.7, 2.1])
    t = 0.8
    got = OT.evolve_td(x, z, ham.a, ham.b, fv, n, t, psi, tol=tol)
    want = psi.copy()
    for f in fv:
        want = _exact_expm(dense_h(ham.labels, ham.a + f * ham.b), t / len(fv)) @ want
    # each step's truncation error is below tol / (1 - ||X|| / (K + 1)) < 2 tol here
    assert np.linalg.norm(got - want) <= len(fv) * 2 * tol + 1e-12


def test_evolve_td_diagonal_exact_phases():
    labels = ["IIIIZ", "IIZZI", "ZIIIZ", "IZZII", "IIIII", "ZZIII"]
    a = np.array([0.4, -0.7, 0.0, 1.2, 0.3, 0.0])
    b = np.array([0.0, 0.5, -0.9, 0.0, 0.1, 0.35])
    x, z, n = O.parse_terms(labels)
    psi = W.gaussian_state(n, np.random.default_rng(8))
    E0 = np.real(np.diag(dense_h(labels, a)))
    E1 = np.real(np.diag(dense_h(labels, b)))
    t = 1.7
    for steps in (1, 3, 7):
        fv = W.midpoint_samples(_drive, t, steps)
        want = np.exp(-1j * (t * E0 + (t / steps) * np.sum(fv) * E1)) * psi
        got = OT.evolve_td(x, z, a, b, fv, n, t, psi)
        assert np.max(np.abs(got - want)) < 1e-12


def test_evolve_td_midpoint_is_second_order():
    """With the exponential of each frozen step exact (tight tolerance), midpoint
    samples converge to the time-ordered solution with error ratio ~4 per
    halved step (an independent 8th-order Runge-Kutta solution)."""
    ham = _ham()
    x, z, n = O.parse_terms(ham.labels)
    psi = W.gaussian_state(n, np.random.default_rng(11))
    H0, H1 = dense_h(ham.labels, ham.a), dense_h(ham.labels, ham.b)
    t = 1.0
    sol = scipy.integrate.solve_ivp(lambda s, y: -1j * ((H0 + _drive(s) * H1) @ y), (0.0, t),
                                    psi.astype(complex), method="DOP853", rtol=1e-12, atol=1e-13)
    want = sol.y[:, -1]
    errs = [np.linalg.norm(OT.evolve_td(x, z, ham.a, ham.b, W.midpoint_samples(_drive, t, s), n, t, psi,
                                        tol=1e-15) - want) for s in (8, 16, 32)]
    for e1, e2 in zip(errs, errs[1:]):
        assert 3.0 < e1 / e2 < 5.0, errs
    # left-endpoint samples are only first order
    left = [np.linalg.norm(OT.evolve_td(x, z, ham.a, ham.b, [_drive(k * t / s) for k in range(s)], n, t, psi,
                                        tol=1e-15) - want) for s in (16, 32)]
    assert 1.6 < left[0] / left[1] < 2.4


@pytest.mark.parametrize("budget", [25, 29])
def test_estimate_timesteps_td_brute_force(budget):
    """The shared step count is the smallest r whose U(t/r) meets the budget for
    every distinct drive sample, each checked by dense Taylor sums."""
    ham = _ham()
    x, z, n = O.parse_terms(ham.labels)
    fv = np.array([0.3, 1.0, 1.6, 1.0])
    t = 1.0
    r = OT.estimate_timesteps_td(x, z, ham.a, ham.b, fv, n, t, budget)
    per_sample = []
    for f in sorted(set(fv)):
        H = dense_h(ham.labels, ham.a + f * ham.b)
        per_sample.append(next(s for s in range(1, 1 << 12)
                               if (c := _dense_diag_count(H, t / s, 1e-6)) is not None and c <= budget))
    assert r == max(per_sample)
