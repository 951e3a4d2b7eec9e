"""Oracle for the single-factor Taylor mode -- TEST INFRASTRUCTURE ONLY.

Plain, slow FP64 numpy statement of the paper's original pipeline (Alg. 3):
H converted to the compact diagonal layout (Eq. 6) with identically-zero
diagonals dropped (the numeric counts of Tab. 3), the diagonal-pair product of
two such matrices (SpGEMM paragraph, Sec. 3.3), the truncated Taylor
exponential (Alg. 2), the diagonal-budget step search (Eq. 5 and the adaptive
timestep flowchart of Sec. 3.1), and the repeated diagonal-times-vector
evolution (Alg. 1 inside Alg. 3), plus expectation values <psi|A|psi> on the
compact layout.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline leg may use it; the product package never does.

A matrix is a ``Dia``: N and {offset d: values}, the value of entry
(row i, col i+d) stored at element index min(i, i+d), offsets kept in the
canonical order of Tab. 1 (0, then |d| ascending, negative first).

Readings of the paper used here (it is silent or ambiguous on each):
  * T.norm() in Alg. 2 is the Frobenius norm; the loop stops before adding the
    first term whose norm is below the tolerance (default 1e-6, as Alg. 2's
    input list states); no scaling and squaring in the budgeted mode, since
    squaring would grow the diagonal count past the cap;
  * a product keeps the diagonals its diagonal pairs can reach, minus those
    whose every entry is at most DROP_REL times the largest entry magnitude of
    that product (cancellation residue; H itself drops only exact zeros);
  * a purely diagonal matrix is exponentiated exactly, element by element
    (SpME paragraph), and needs one step (flowchart's first test);
  * step search: l = n_min = 1, the upper bound doubles from l until the budget
    is met, then a binary search between the last failing and first passing
    counts; r is feasible iff the Taylor loop converges within max_iter terms
    and num_diags(U(t/r)) <= D_max (Eq. 5).

Time-dependent H0 + f(t) H1 (ham_dia_td, estimate_timesteps_td, evolve_td)
is pinned by tests/test_taylor_td_pins.py.

Parity status: every function is pinned by tests/test_taylor_pins.py (dense
Kronecker sums, numpy matrix products, eigh-based exponentials with the Taylor
remainder bound, elementwise exponentials, brute-force step scans, Tab. 3,
dense quadratic forms and a closed-form eigenstate energy).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import numpy as np

from . import canonical_order, ham_diagonals

DROP_REL = 2.0 ** -46


@dataclass
class Dia:
    N: int
    diags: Dict[int, np.ndarray] = field(default_factory=dict)

    @property
    def offsets(self) -> List[int]:
        return canonical_order(self.diags.keys())

    @property
    def n_diags(self) -> int:
        return len(self.diags)

    def nnz(self) -> int:
        return int(sum(np.count_nonzero(v) for v in self.diags.values()))


def identity(N: int) -> Dia:
    return Dia(N, {0: np.ones(N, dtype=np.complex128)})


def ham_dia(x, z, coeffs, n_qubits: int) -> Dia:
    """H = sum_j c_j P_j in the compact layout, exactly-zero diagonals dropped."""
    d = ham_diagonals(x, z, coeffs, n_qubits)
    return Dia(1 << n_qubits, {k: v for k, v in d.items() if np.any(v != 0)})


def to_dense(A: Dia) -> np.ndarray:
    M = np.zeros((A.N, A.N), dtype=np.complex128)
    for d, v in A.diags.items():
        i = np.arange(A.N - abs(d))
        r = i - min(0, d)
        M[r, r + d] = v
    return M


def from_dense(M) -> Dia:
    """Every diagonal of a dense matrix with a nonzero entry."""
    M = np.asarray(M, dtype=np.complex128)
    N = M.shape[0]
    return Dia(N, {d: np.diagonal(M, d).copy() for d in range(-(N - 1), N) if np.any(np.diagonal(M, d) != 0)})


def drop_negligible(A: Dia, rel: float = DROP_REL) -> Dia:
    """Remove the diagonals whose entries are all <= rel * (largest |entry| of A)."""
    if not A.diags:
        return A
    top = max(float(np.max(np.abs(v))) if v.size else 0.0 for v in A.diags.values())
    thr = rel * top
    return Dia(A.N, {d: v for d, v in A.diags.items() if v.size and float(np.max(np.abs(v))) > thr})


def spgemm(A: Dia, B: Dia) -> Dia:
    """C = A B by diagonal pairs (SpGEMM paragraph): result diagonal dc collects
    every pair (da, db) with da + db = dc, entry (i, i+dc) += A(i, i+da) * B(i+da, i+dc)
    over the rows where all three entries exist.  Pairs in A-major canonical order."""
    N = A.N
    C: Dict[int, np.ndarray] = {}
    for da in A.offsets:
        va = A.diags[da]
        for db in B.offsets:
            vb = B.diags[db]
            dc = da + db
            if abs(dc) >= N:
                continue
            lo, hi = max(0, -da, -dc), min(N, N - da, N - dc)
            if lo >= hi:
                continue
            i = np.arange(lo, hi)
            acc = C.setdefault(dc, np.zeros(N - abs(dc), dtype=np.complex128))
            acc[np.minimum(i, i + dc)] += va[np.minimum(i, i + da)] * vb[np.minimum(i + da, i + dc)]
    return drop_negligible(Dia(N, C))


def add(A: Dia, B: Dia) -> Dia:
    """A + B on the union of the two diagonal sets (matrix addition, Sec. 3.3)."""
    out = {d: v.copy() for d, v in A.diags.items()}
    for d, v in B.diags.items():
        if d in out:
            out[d] = out[d] + v
        else:
            out[d] = v.copy()
    return Dia(A.N, out)


def scale(A: Dia, s: complex) -> Dia:
    return Dia(A.N, {d: v * s for d, v in A.diags.items()})


def fro(A: Dia) -> float:
    return float(np.sqrt(sum(float(np.sum(np.abs(v) ** 2)) for v in A.diags.values())))


def is_diagonal(A: Dia) -> bool:
    return all(d == 0 for d in A.diags)


def expm_diag(A: Dia, t: float) -> Dia:
    """exp(-i t A) of a diagonal A, entry by entry (SpME fast path)."""
    v = A.diags.get(0, np.zeros(A.N, dtype=np.complex128))
    return Dia(A.N, {0: np.exp(-1j * t * v)})


def expm_taylor(A: Dia, t: float, tol: float = 1e-6, max_iter: int = 100,
                max_diags: Optional[int] = None) -> Tuple[Dia, int, bool]:
    """Alg. 2: X = -i t A; U = T = I; for k = 1..max_iter: T = (T X) / k; stop
    when ||T||_F < tol, else U += T.  Returns (U, k at the stop, converged).
    With max_diags, also stops (not converged) once U holds more diagonals."""
    X = scale(A, -1j * t)
    U = identity(A.N)
    T = identity(A.N)
    for k in range(1, max_iter + 1):
        T = scale(spgemm(T, X), 1.0 / k)
        if fro(T) < tol:
            return U, k, True
        U = add(U, T)
        if max_diags is not None and U.n_diags > max_diags:
            return U, k, False
    return U, max_iter, False


def expm(A: Dia, t: float, tol: float = 1e-6, max_iter: int = 100) -> Tuple[Dia, int, bool]:
    """SpME: exact for a diagonal matrix, truncated Taylor otherwise."""
    if is_diagonal(A):
        return expm_diag(A, t), 0, True
    return expm_taylor(A, t, tol, max_iter)


def feasible(A: Dia, t: float, r: int, budget: int, tol: float = 1e-6, max_iter: int = 100) -> bool:
    """Eq. 5 for r steps: the Taylor loop converges and U(t/r) has <= budget diagonals."""
    U, _, ok = expm_taylor(A, t / r, tol, max_iter, max_diags=budget)
    return ok and U.n_diags <= budget


def estimate_timesteps(A: Dia, t: float, budget: int, tol: float = 1e-6, max_iter: int = 100,
                       max_steps: int = 1 << 20) -> int:
    """Smallest r with num_diags(exp(-i A t/r)) <= budget (adaptive timestep
    flowchart, Sec. 3.1).  Raises ValueError if no r <= max_steps passes."""
    if is_diagonal(A):
        return 1
    lo = 0
    hi = 1
    while not feasible(A, t, hi, budget, tol, max_iter):
        lo = hi
        hi *= 2
        if hi > max_steps:
            raise ValueError("diagonal budget not met within max_steps")
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if feasible(A, t, mid, budget, tol, max_iter):
            hi = mid
        else:
            lo = mid
    return hi


def spmv(A: Dia, x) -> np.ndarray:
    """y = A x: y[i] = sum_d A(i, i+d) x[i+d] (Alg. 1)."""
    x = np.asarray(x, dtype=np.complex128)
    y = np.zeros_like(x)
    N = A.N
    for d in A.offsets:
        v = A.diags[d]
        lo, hi = max(0, -d), min(N, N - d)
        i = np.arange(lo, hi)
        y[..., i] += v[np.minimum(i, i + d)] * x[..., i + d]
    return y


def expectation(A: Dia, psi) -> np.ndarray:
    """<psi|A|psi> per state (rows of psi): the plain definition, conj(psi) . (A psi)."""
    x = np.atleast_2d(np.asarray(psi, dtype=np.complex128))
    y = spmv(A, x)
    return np.array([np.vdot(x[k], y[k]) for k in range(x.shape[0])])


def evolve(U: Dia, psi, n_steps: int) -> np.ndarray:
    """Alg. 3's loop: psi <- U psi, n_steps times."""
    x = np.asarray(psi, dtype=np.complex128).copy()
    for _ in range(n_steps):
        x = spmv(U, x)
    return x


# ----------------------------------------------------------------------------
# Time-dependent H(t) = H0 + f(t) H1 in the single-factor mode (the outlook on
# time-dependent Hamiltonians).  Readings: step k freezes the drive at the
# caller's sample f_k; H(f_k) is formed from the terms with c_j = a_j + f_k b_j
# (product rounded before the sum) and exactly-zero diagonals dropped, then
# exponentiated by SpME at dt = t / (number of samples) and applied once.  One
# step count serves every step: the smallest r meeting Eq. 5 for each distinct
# sample (each searched as for a static H), so the search runs once before the
# evolution and not per step.
# ----------------------------------------------------------------------------

def ham_dia_td(x, z, a, b, f: float, n_qubits: int) -> Dia:
    """H0 + f H1 in the compact layout."""
    c = np.asarray(a, dtype=np.float64) + float(f) * np.asarray(b, dtype=np.float64)
    return ham_dia(x, z, c, n_qubits)


def estimate_timesteps_td(x, z, a, b, drive, n_qubits: int, t: float, budget: int, tol: float = 1e-6,
                          max_iter: int = 100, max_steps: int = 1 << 20) -> int:
    """Steps r over [0, t] such that U(t/r) of every sampled H(f_k) has at most
    budget diagonals: the largest of the static searches over distinct samples."""
    r = 1
    for f in sorted(set(float(v) for v in np.asarray(drive, dtype=np.float64).ravel())):
        r = max(r, estimate_timesteps(ham_dia_td(x, z, a, b, f, n_qubits), t, budget, tol, max_iter, max_steps))
    return r


def evolve_td(x, z, a, b, drive, n_qubits: int, t: float, psi, tol: float = 1e-6,
              max_iter: int = 100) -> np.ndarray:
    """One step per drive sample, dt = t / len(drive): psi <- U_k psi with
    U_k = SpME(H(f_k), dt) (exact for a diagonal H(f_k))."""
    fv = np.asarray(drive, dtype=np.float64).ravel()
    dt = float(t) / len(fv)
    out = np.asarray(psi, dtype=np.complex128).copy()
    for f in fv:
        U, _, ok = expm(ham_dia_td(x, z, a, b, f, n_qubits), dt, tol, max_iter)
        if not ok:
            raise ValueError("Taylor series did not converge within max_iter terms")
        out = spmv(U, out)
    return out
