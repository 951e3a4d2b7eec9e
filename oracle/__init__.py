"""Oracle for diagonal-budgeted Trotterization -- TEST INFRASTRUCTURE ONLY.

Plain, slow FP64 CPU implementation of what the GPU path computes.  Only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import it; the product package never does, and the two share no code.

Python half (this file): Pauli-label parsing, the budgeted next-fit grouping
with its structural offset sets (the structural dry run of the diagonal-set
estimation paragraph, Sec. 3.2), and the canonical diagonal order of Tab. 1.
Numeric half (``hs_oracle.c``, loaded through ctypes): Pauli rotations,
direct Trotter evolution (Eq. 4) and, in Python over the same rotations, the
second- and fourth-order product formulas and time-dependent evolution under
H0 + f(t) H1, factor materialisation into the compact
layout (Eq. 6), the diagonal-times-vector product (Alg. 1), pairwise sums.

Readings of the paper used here (the paper is silent or ambiguous on each):
  * label character p acts on qubit n-1-p (rightmost character = qubit 0 =
    bit 0 of the basis index);
  * first-order product: term 1 acts first (Eq. 4 read left-to-right in time);
  * a group admits term j iff it is empty, or its offset count after adding
    j stays within the budget, or adding j leaves the offset set unchanged;
  * stored offsets are structural (all of O(X), even if a value is zero);
  * canonical offset order: 0, then |d| ascending, negative before positive
    (reproduces Tab. 1's [0, -3, 3]);
  * fidelity = |<a|b>|^2 / (|a|^2 |b|^2) (evaluation section, Metrics).

Parity status: every function here is pinned by tests/test_oracle_pins.py
(dense Kronecker products, scipy expm, numpy eigh, closed forms, Tab. 1,
Tab. 3 and the appendix quick-start example), the product formulas by
tests/test_order_pins.py and the time-dependent evolution by
tests/test_td_pins.py (per-step scipy exponentials, exact diagonal phases, an
independent ODE solver); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

_lib_handle = None


def build(force: bool = False) -> str:
    """Compile the C half with gcc (plain -O2, no target-specific flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _lib_handle
    if _lib_handle is None:
        lib = ctypes.CDLL(build())
        i64, u64p, dp, i64p = ctypes.c_int64, ctypes.POINTER(ctypes.c_uint64), ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)
        lib.orc_pauli_apply.argtypes = [i64, ctypes.c_uint64, ctypes.c_uint64, dp, dp]
        lib.orc_rotate.argtypes = [i64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double, dp]
        lib.orc_evolve_direct.argtypes = [i64, ctypes.c_int, ctypes.c_int, u64p, u64p, dp,
                                          ctypes.c_double, ctypes.c_int, dp]
        lib.orc_build_factor.argtypes = [i64, ctypes.c_int, u64p, u64p, dp, ctypes.c_int, u64p,
                                         ctypes.c_int, i64p, i64p, dp]
        lib.orc_build_factor.restype = ctypes.c_int
        lib.orc_dia_apply.argtypes = [i64, ctypes.c_int, i64p, i64p, dp, dp, dp]
        lib.orc_norm2.argtypes = [i64, dp]
        lib.orc_norm2.restype = ctypes.c_double
        lib.orc_inner.argtypes = [i64, dp, dp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        _lib_handle = lib
    return _lib_handle


def _u64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint64))


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


# ----------------------------------------------------------------------------
# Pauli labels (terms are Pauli strings with real coefficients, Sec. 4.4)
# ----------------------------------------------------------------------------

def parse_label(label: str) -> Tuple[int, int]:
    """Label over {I,X,Y,Z} -> (x_mask, z_mask).  Character p acts on qubit n-1-p.
    X sets x, Z sets z, Y sets both."""
    n = len(label)
    x = z = 0
    for p, ch in enumerate(label):
        q = n - 1 - p
        if ch == "I":
            continue
        if ch == "X":
            x |= 1 << q
        elif ch == "Z":
            z |= 1 << q
        elif ch == "Y":
            x |= 1 << q
            z |= 1 << q
        else:
            raise ValueError(f"invalid Pauli character {ch!r} in {label!r}")
    return x, z


def parse_terms(labels: Sequence[str]) -> Tuple[np.ndarray, np.ndarray, int]:
    if not labels:
        raise ValueError("no terms")
    n = len(labels[0])
    if any(len(l) != n for l in labels):
        raise ValueError("labels differ in length")
    xz = [parse_label(l) for l in labels]
    return _u64([a for a, _ in xz]), _u64([b for _, b in xz]), n


# ----------------------------------------------------------------------------
# Structural grouping (diagonal budget, Eq. 5 used as a cap per factor)
# ----------------------------------------------------------------------------

def offsets_of_mask(x: int) -> set:
    """Diagonal offsets d = col - row of the entries of a Pauli with flip mask x:
    row r and column r xor x differ by +2^k where r has bit k clear and -2^k where
    it is set, so offs(x) = { sum_{k in x} +-2^k } (2^|x| values)."""
    offs = {0}
    k = 0
    while x >> k:
        if (x >> k) & 1:
            offs = {o + s * (1 << k) for o in offs for s in (1, -1)}
        k += 1
    return offs


def offsets_of_set(X: set) -> set:
    out = set()
    for u in X:
        out |= offsets_of_mask(u)
    return out


def canonical_order(offsets) -> List[int]:
    """0 first, then |d| ascending, negative before positive (Tab. 1: [0, -3, 3])."""
    return sorted(offsets, key=lambda d: (abs(d), d))


@dataclass
class Group:
    first: int          # first term index (inclusive)
    last: int           # last term index (exclusive)
    X: List[int]        # the group's x-mask set, closed under xor, sorted
    offsets: List[int]  # canonical order


def group_terms(x_masks: Sequence[int], budget: int) -> List[Group]:
    """Next-fit grouping in input order.  A group keeps its x-mask set X (starting
    at {0}; adding x gives X | {u ^ x : u in X}) and O(X) = union of offs(u).
    Term j joins the open group iff the group is empty, |O(X')| <= budget, or
    O(X') == O(X); otherwise the group closes and j opens the next one."""
    if budget < 1:
        raise ValueError("budget must be >= 1")
    groups: List[Group] = []
    first = 0
    X, O = {0}, {0}
    for j, xj in enumerate(int(v) for v in x_masks):
        Xn = X | {u ^ xj for u in X}
        On = offsets_of_set(Xn)
        if j == first or len(On) <= budget or On == O:
            X, O = Xn, On
        else:
            groups.append(Group(first, j, sorted(X), canonical_order(O)))
            first = j
            X = {0, xj}
            O = offsets_of_set(X)
    groups.append(Group(first, len(x_masks), sorted(X), canonical_order(O)))
    return groups


def starts_of(offsets: Sequence[int], N: int) -> np.ndarray:
    """Storage start of each diagonal: prefix sums of N - |d| (no padding)."""
    st = np.zeros(len(offsets), dtype=np.int64)
    acc = 0
    for k, d in enumerate(offsets):
        st[k] = acc
        acc += N - abs(d)
    return st


# ----------------------------------------------------------------------------
# Numeric parts (C core)
# ----------------------------------------------------------------------------

@dataclass
class Factor:
    first: int
    last: int
    X: List[int]
    offsets: List[int]
    starts: np.ndarray
    values: np.ndarray = field(repr=False)  # complex128, unpadded compact layout


def step_angles(coeffs, t: float, n_steps: int) -> np.ndarray:
    """theta_j = c_j * dt with dt = t / n_steps (one FP64 rounding each)."""
    dt = float(t) / float(n_steps)
    return np.asarray([float(c) * dt for c in coeffs], dtype=np.float64)


def build_factors(x, z, coeffs, n_qubits: int, t: float, n_steps: int, budget: int) -> List[Factor]:
    """Group the terms, fix each group's offsets and starts, and materialise its
    numeric values column by column (FP64)."""
    x, z = _u64(x), _u64(z)
    N = 1 << n_qubits
    theta = step_angles(coeffs, t, n_steps)
    lib = _lib()
    out = []
    for g in group_terms(x, budget):
        offs = _i64(g.offsets)
        st = starts_of(g.offsets, N)
        total = int(st[-1] + N - abs(g.offsets[-1]))
        vals = np.zeros(total, dtype=np.complex128)
        gx, gz = _u64(x[g.first:g.last]), _u64(z[g.first:g.last])
        th = np.ascontiguousarray(theta[g.first:g.last])
        Xa = _u64(g.X)
        rc = lib.orc_build_factor(N, g.last - g.first, _ptr(gx, ctypes.c_uint64), _ptr(gz, ctypes.c_uint64),
                                  th.ctypes.data, len(g.X), _ptr(Xa, ctypes.c_uint64), len(g.offsets),
                                  _ptr(offs, ctypes.c_int64), _ptr(st, ctypes.c_int64), vals.ctypes.data)
        if rc != 0:
            raise RuntimeError("structural entry outside the factor's offset set")
        out.append(Factor(g.first, g.last, list(g.X), list(g.offsets), st, vals))
    return out


def pauli_apply(x: int, z: int, psi) -> np.ndarray:
    psi = _c128(psi)
    out = np.empty_like(psi)
    _lib().orc_pauli_apply(psi.size, int(x), int(z), psi.ctypes.data, out.ctypes.data)
    return out


def evolve_direct(x, z, coeffs, t: float, n_steps: int, psi) -> np.ndarray:
    """Direct first-order Trotter evolution; psi is (N,) or (n_rhs, N); returns a copy."""
    psi = _c128(psi).copy()
    shape = psi.shape
    psi2 = psi.reshape(-1, shape[-1])
    x, z = _u64(x), _u64(z)
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
    _lib().orc_evolve_direct(shape[-1], psi2.shape[0], len(x), _ptr(x, ctypes.c_uint64),
                             _ptr(z, ctypes.c_uint64), c.ctypes.data, float(t), int(n_steps), psi2.ctypes.data)
    return psi2.reshape(shape)


# ----------------------------------------------------------------------------
# Higher-order product formulas (the paper's future-work passage on second-
# and fourth-order formulas; readings: symmetric Strang splitting and Suzuki's
# fourth-order recursion of it)
# ----------------------------------------------------------------------------

SUZUKI_P = 1.0 / (4.0 - 4.0 ** (1.0 / 3.0))


def step_stages(order: int, dt: float):
    """One step of the product formula of the given order as a list of
    (angle scale h, direction): every term j is applied as exp(-i c_j h P_j),
    terms in input order for direction +1 and in reverse order for -1.
      order 1: [(dt, +1)]
      order 2 (Strang): [(dt/2, +1), (dt/2, -1)]
      order 4 (Suzuki): S2(p dt) S2(p dt) S2((1-4p) dt) S2(p dt) S2(p dt), p = 1/(4 - 4^(1/3))."""
    if order == 1:
        return [(dt, 1)]
    if order == 2:
        return [(dt * 0.5, 1), (dt * 0.5, -1)]
    if order == 4:
        hp = (SUZUKI_P * dt) * 0.5
        hq = ((1.0 - 4.0 * SUZUKI_P) * dt) * 0.5
        out = []
        for h in (hp, hp, hq, hp, hp):
            out += [(h, 1), (h, -1)]
        return out
    raise ValueError("order must be 1, 2 or 4")


def evolve_direct_order(x, z, coeffs, t: float, n_steps: int, psi, order: int) -> np.ndarray:
    """Direct evolution by the product formula of the given order (term by term,
    FP64); psi is (N,) or (n_rhs, N); returns a copy."""
    psi = _c128(psi).copy()
    shape = psi.shape
    rows = psi.reshape(-1, shape[-1])
    x, z = _u64(x), _u64(z)
    c = np.asarray(coeffs, dtype=np.float64)
    dt = float(t) / float(n_steps)
    lib = _lib()
    stages = step_stages(order, dt)
    for r in range(rows.shape[0]):
        row = np.ascontiguousarray(rows[r])
        for _ in range(n_steps):
            for h, direction in stages:
                js = range(len(x)) if direction > 0 else range(len(x) - 1, -1, -1)
                for j in js:
                    lib.orc_rotate(row.size, int(x[j]), int(z[j]), float(c[j]) * h, row.ctypes.data)
        rows[r] = row
    return rows.reshape(shape)


# ----------------------------------------------------------------------------
# Time-dependent Hamiltonians H(t) = H0 + f(t) H1 (the paper's outlook on
# time-dependent Hamiltonians).  Readings: term j carries two real
# coefficients, a_j in H0 and b_j in H1 (either may be zero); step s freezes
# H at the caller's sample f_s of f for that step, so every term uses
# c_j(s) = a_j + f_s b_j (the product rounded before the sum), and the step is
# the product formula of the given order with those coefficients.  Sampling f
# at the step midpoints gives the exponential midpoint rule.
# ----------------------------------------------------------------------------

def td_coeffs(a, b, f: float) -> np.ndarray:
    """c_j = a_j + f b_j for one frozen value f of the drive."""
    return np.asarray(a, dtype=np.float64) + float(f) * np.asarray(b, dtype=np.float64)


def evolve_direct_td(x, z, a, b, f_values, t: float, psi, order: int = 1) -> np.ndarray:
    """Direct evolution under H(t) = H0 + f(t) H1 with one step per entry of
    f_values (dt = t / len(f_values)); psi is (N,) or (n_rhs, N); returns a copy."""
    psi = _c128(psi).copy()
    shape = psi.shape
    rows = psi.reshape(-1, shape[-1])
    x, z = _u64(x), _u64(z)
    fv = np.asarray(f_values, dtype=np.float64).ravel()
    n_steps = len(fv)
    dt = float(t) / float(n_steps)
    lib = _lib()
    stages = step_stages(order, dt)
    coeffs = [td_coeffs(a, b, fv[s]) for s in range(n_steps)]
    for r in range(rows.shape[0]):
        row = np.ascontiguousarray(rows[r])
        for s in range(n_steps):
            c = coeffs[s]
            for h, direction in stages:
                js = range(len(x)) if direction > 0 else range(len(x) - 1, -1, -1)
                for j in js:
                    lib.orc_rotate(row.size, int(x[j]), int(z[j]), float(c[j]) * h, row.ctypes.data)
        rows[r] = row
    return rows.reshape(shape)


def dia_apply(offsets, starts, values, xvec) -> np.ndarray:
    """y = A x for A in the compact diagonal layout (Alg. 1)."""
    offs, st, vals, xv = _i64(offsets), _i64(starts), _c128(values), _c128(xvec)
    y = np.empty_like(xv)
    _lib().orc_dia_apply(xv.size, len(offs), _ptr(offs, ctypes.c_int64), _ptr(st, ctypes.c_int64),
                         vals.ctypes.data, xv.ctypes.data, y.ctypes.data)
    return y


def evolve_factors(factors: Sequence[Factor], psi, n_steps: int) -> np.ndarray:
    """psi <- (F_G ... F_1)^n_steps psi through the diagonal layout (Alg. 3 loop)."""
    psi = _c128(psi)
    shape = psi.shape
    rows = [r.copy() for r in psi.reshape(-1, shape[-1])]
    for s in range(n_steps):
        for f in factors:
            rows = [dia_apply(f.offsets, f.starts, f.values, r) for r in rows]
    return np.stack(rows).reshape(shape)


def norm2(a) -> float:
    a = _c128(a)
    return float(_lib().orc_norm2(a.size, a.ctypes.data))


def inner(a, b) -> complex:
    a, b = _c128(a), _c128(b)
    re, im = ctypes.c_double(), ctypes.c_double()
    _lib().orc_inner(a.size, a.ctypes.data, b.ctypes.data, ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def fidelity(a, b) -> float:
    """|<a|b>|^2 / (|a|^2 |b|^2)."""
    ip = inner(a, b)
    return (ip.real * ip.real + ip.imag * ip.imag) / (norm2(a) * norm2(b))


# ----------------------------------------------------------------------------
# Dense <-> compact layout (used by the layout pins; Tab. 1 and Eq. 6)
# ----------------------------------------------------------------------------

def dia_from_dense(M, offsets=None, tol: float = 0.0):
    """Compact layout of a dense matrix.  offsets=None keeps every diagonal with an
    entry of magnitude > tol (numeric count), in canonical order."""
    M = np.asarray(M)
    N = M.shape[0]
    if offsets is None:
        offsets = [d for d in range(-(N - 1), N) if np.any(np.abs(np.diagonal(M, d)) > tol)]
        offsets = canonical_order(offsets)
    st = starts_of(offsets, N)
    vals = np.concatenate([np.diagonal(M, d) for d in offsets]).astype(np.complex128)
    return list(offsets), st, vals


def ham_diagonals(x, z, coeffs, n_qubits: int) -> dict:
    """Every diagonal of H = sum_j c_j P_j that some term touches, as
    {offset d: values indexed by min(row, col)} (Eq. 6 element index).  Entry
    (row b xor x_j, col b) of P_j is i^{y_j} (-1)^{popcount(z_j & b)}; terms are
    accumulated in input order, so cancelling terms leave exact zeros."""
    N = 1 << n_qubits
    b = np.arange(N, dtype=np.uint64)
    diags = {}
    for xj, zj, c in zip(_u64(x), _u64(z), coeffs):
        xj, zj = int(xj), int(zj)
        y = bin(xj & zj).count("1")
        par = np.zeros(N, dtype=np.int64)
        zb = b & np.uint64(zj)
        for k in range(n_qubits):
            par ^= ((zb >> np.uint64(k)) & np.uint64(1)).astype(np.int64)
        phase = (1j ** y) * np.where(par == 1, -1.0, 1.0)
        row = (b ^ np.uint64(xj)).astype(np.int64)
        col = b.astype(np.int64)
        d_all = col - row
        for d in np.unique(d_all):
            sel = d_all == d
            arr = diags.setdefault(int(d), np.zeros(N - abs(int(d)), dtype=np.complex128))
            idx = np.minimum(row[sel], col[sel])
            np.add.at(arr, idx, c * phase[sel])
    return diags


def hamiltonian_structure(x, z, coeffs, n_qubits: int, tol: float = 0.0):
    """Numeric diagonal count and nonzero count of H = sum c_j P_j (zeros dropped),
    the two structural columns of Tab. 3."""
    diags = ham_diagonals(x, z, coeffs, n_qubits)
    nz = {d: int(np.count_nonzero(np.abs(v) > tol)) for d, v in diags.items()}
    kept = [d for d, k in nz.items() if k > 0]
    return len(kept), sum(nz.values())
