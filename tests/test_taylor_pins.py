"""Pins of the Taylor-mode oracle (Alg. 2, Alg. 3, Eq. 5) against things other
than itself: dense Kronecker sums of the 2x2 Pauli matrices, numpy matrix
products and powers, eigh-based exponentials with the Taylor remainder bound,
elementwise exponentials of diagonal energies evaluated on bitstrings, a
brute-force step scan on dense matrices, and the Tab. 3 diagonal counts.
"""
import math

import numpy as np
import pytest

import oracle as O
from conftest import read_golden
from oracle import taylor as OT
from paper_2606_16959_gb300 import workloads as W
from test_oracle_pins import dense_h, random_labels


def _dia(ham):
    x, z, n = O.parse_terms(ham.labels)
    return OT.ham_dia(x, z, ham.coeffs, n)


def _exact_expm(H, t):
    w, V = np.linalg.eigh(H)
    return (V * np.exp(-1j * t * w)) @ V.conj().T


def _random_dia(rng, N, n_diags):
    offs = rng.choice(np.arange(-(N - 1), N), size=n_diags, replace=False)
    return OT.Dia(N, {int(d): rng.normal(size=N - abs(int(d))) + 1j * rng.normal(size=N - abs(int(d)))
                      for d in offs})


# ---------------------------------------------------------------------------
# H in the compact layout
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_ham_dia_equals_kronecker_sum(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 6))
    labels = random_labels(rng, n, int(rng.integers(1, 9)))
    coeffs = rng.uniform(-1, 1, len(labels))
    x, z, _ = O.parse_terms(labels)
    A = OT.ham_dia(x, z, coeffs, n)
    M = dense_h(labels, coeffs)
    assert np.array_equal(OT.to_dense(A), M)
    # kept diagonals are exactly the nonzero diagonals of the dense sum
    assert sorted(A.diags) == sorted(d for d in range(-(M.shape[0] - 1), M.shape[0]) if np.any(np.diagonal(M, d)))


def test_heisenberg_bond_cancellation():
    """XX + YY cancels on 00 <-> 11: a bond keeps offsets 0, +-2^i only (Tab. 3)."""
    A = _dia(W.Hamiltonian("bond", 2, ["XX", "YY", "ZZ"], np.array([1.0, 1.0, 1.0])))
    assert A.offsets == [0, -1, 1]
    assert A.nnz() == 4 + 2  # diagonal (ZZ) + the two flip-flop entries


@pytest.mark.parametrize("row", read_golden("tab3_structure.txt")["rows"], ids=lambda r: r[0])
def test_tab3_counts_through_ham_dia(row):
    label, fam, n, bc, ndiag, sp = row[0], row[1], int(row[2]), row[3], int(row[4]), row[5]
    if n > 14:
        pytest.skip("kept to n <= 14 for the CPU suite (n = 16 rows are covered by test_oracle_pins)")
    if fam == "tfim":
        ham = W.tfim_chain(n, 1.0, 1.0, periodic=(bc == "pbc"))
    elif fam == "heisenberg":
        ham = W.heisenberg_chain(n, np.ones(n if bc == "pbc" else n - 1), periodic=(bc == "pbc"))
    else:
        pytest.skip("TSP rows: diagonal Hamiltonian, covered by the oracle pins")
    A = _dia(ham)
    assert A.n_diags == ndiag
    if sp != "-":
        assert round(100.0 * (1.0 - A.nnz() / float(A.N) ** 2), 4) == pytest.approx(float(sp), abs=1e-9)


# ---------------------------------------------------------------------------
# SpGEMM, addition, SpMV
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(8))
def test_spgemm_equals_dense_product(seed):
    rng = np.random.default_rng(100 + seed)
    N = int(2 ** rng.integers(1, 7))
    A = _random_dia(rng, N, int(rng.integers(1, min(2 * N - 1, 9) + 1)))
    B = _random_dia(rng, N, int(rng.integers(1, min(2 * N - 1, 9) + 1)))
    C = OT.spgemm(A, B)
    P = OT.to_dense(A) @ OT.to_dense(B)
    assert np.max(np.abs(OT.to_dense(C) - P)) <= 1e-13 * max(1.0, np.max(np.abs(P)))
    # the kept diagonals are the reachable ones with a nonzero entry
    reach = {a + b for a in A.diags for b in B.diags if abs(a + b) < N}
    assert set(C.diags) == {d for d in reach if np.any(np.abs(np.diagonal(P, d)) > 0)}


def test_spgemm_drops_cancellation_residue():
    """(XX+YY)^2 on one bond: the +-3 and +-2 diagonals cancel exactly in the
    product of the matrices, and the product is 2 (I - ZZ) restricted there."""
    A = _dia(W.Hamiltonian("bond", 2, ["XX", "YY"], np.array([1.0, 1.0])))
    C = OT.spgemm(A, A)
    M = dense_h(["XX", "YY"], [1.0, 1.0])
    assert np.allclose(OT.to_dense(C), M @ M, atol=1e-15)
    assert C.offsets == [0]


@pytest.mark.parametrize("seed", range(4))
def test_add_and_spmv_dense(seed):
    rng = np.random.default_rng(200 + seed)
    N = 32
    A, B = _random_dia(rng, N, 5), _random_dia(rng, N, 4)
    assert np.allclose(OT.to_dense(OT.add(A, B)), OT.to_dense(A) + OT.to_dense(B), atol=0)
    x = rng.normal(size=(3, N)) + 1j * rng.normal(size=(3, N))
    assert np.allclose(OT.spmv(A, x), x @ OT.to_dense(A).T, atol=1e-13)
    assert np.allclose(OT.evolve(A, x[0], 3), np.linalg.matrix_power(OT.to_dense(A), 3) @ x[0], rtol=1e-12)


# ---------------------------------------------------------------------------
# Truncated Taylor exponential (Alg. 2)
# ---------------------------------------------------------------------------

CASES = [
    ("tfim4", lambda: W.tfim_chain(4, 1.0, 0.7, periodic=False)),
    ("heis4", lambda: W.heisenberg_chain(4, np.array([0.6, 1.1, 1.4, 0.9]), periodic=True)),
    ("rand3", lambda: W.Hamiltonian("random", 3, ["XYZ", "IZX", "YYI", "ZIZ"], np.array([0.3, -0.8, 0.5, 1.1]))),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("t", [0.05, 0.3, 1.0])
def test_taylor_remainder_bound(name, make, t):
    """||U - exp(-iHt)||_F <= sum of the dropped terms <= tol / (1 - ||X||_2/(K+1))."""
    ham = make()
    H = dense_h(ham.labels, ham.coeffs)
    A = _dia(ham)
    tol = 1e-6
    U, K, ok = OT.expm_taylor(A, t, tol, 200)
    assert ok
    nx = t * np.linalg.norm(H, 2)
    assert nx < K + 1
    err = np.linalg.norm(OT.to_dense(U) - _exact_expm(H, t))
    assert err <= tol / (1.0 - nx / (K + 1)) + 1e-12
    # K is the first power whose term falls under the tolerance (dense brute force)
    k, T = 0, np.eye(H.shape[0], dtype=complex)
    while True:
        k += 1
        T = T @ (-1j * t * H) / k
        if np.linalg.norm(T) < tol:
            break
    assert K == k


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_taylor_tight_tolerance_is_exact(name, make):
    ham = make()
    H = dense_h(ham.labels, ham.coeffs)
    U, _, ok = OT.expm_taylor(_dia(ham), 0.4, 1e-15, 200)
    assert ok
    assert np.max(np.abs(OT.to_dense(U) - _exact_expm(H, 0.4))) < 1e-13


def test_diagonal_exponential_from_bitstring_energies():
    """MaxCut without the mixer: U = diag(exp(-i t E(b))), E(b) = sum_edges w (1 - s_i s_j)/2
    evaluated on bitstrings, independently of the Pauli expansion."""
    n = 6
    edges = [(0, 1, 0.3), (1, 2, 0.9), (2, 3, 0.4), (3, 4, 0.7), (4, 5, 0.2), (5, 0, 0.6), (0, 3, 0.5)]
    labels, coeffs = ["I" * n], [sum(w for *_, w in edges) / 2]
    for i, j, w in edges:
        lab = ["I"] * n
        lab[n - 1 - i] = lab[n - 1 - j] = "Z"
        labels.append("".join(lab))
        coeffs.append(-w / 2)
    x, z, _ = O.parse_terms(labels)
    A = OT.ham_dia(x, z, np.array(coeffs), n)
    b = np.arange(1 << n)
    E = np.zeros(1 << n)
    for i, j, w in edges:
        E += w * (((b >> i) & 1) != ((b >> j) & 1))
    t = 1.7
    U, K, ok = OT.expm(A, t)
    assert ok and K == 0 and U.offsets == [0]
    assert np.max(np.abs(U.diags[0] - np.exp(-1j * t * E))) < 1e-14
    Ut, _, ok = OT.expm_taylor(A, t, 1e-15, 200)
    assert ok and np.max(np.abs(Ut.diags[0] - np.exp(-1j * t * E))) < 1e-12


# ---------------------------------------------------------------------------
# Step search (Eq. 5)
# ---------------------------------------------------------------------------

def _dense_diag_count(H, dt, tol, max_iter=200):
    """num_diags of the truncated Taylor sum, from dense powers: the union of the
    diagonals of the terms kept before the first term under tol."""
    N = H.shape[0]
    T = np.eye(N, dtype=complex)
    keep = {0}
    for k in range(1, max_iter + 1):
        T = T @ (-1j * dt * H) / k
        if np.linalg.norm(T) < tol:
            return len(keep)
        top = np.max(np.abs(T))
        keep |= {d for d in range(-(N - 1), N) if np.max(np.abs(np.diagonal(T, d))) > OT.DROP_REL * top}
    return None


@pytest.mark.parametrize("name,make,t,budget", [
    ("tfim4", lambda: W.tfim_chain(4, 1.0, 0.7, periodic=False), 1.0, 29),
    ("tfim4_tight", lambda: W.tfim_chain(4, 1.0, 0.7, periodic=False), 1.0, 12),
    ("heis4_one_step", lambda: W.heisenberg_chain(4, np.array([0.6, 1.1, 1.4, 0.9]), periodic=True), 1.0, 17),
    ("heis6_open", lambda: W.heisenberg_chain(6, np.ones(5), periodic=False), 1.0, 85),
    ("tfim6", lambda: W.tfim_chain(6, 1.0, 1.0, periodic=False), 1.0, 125),
])
def test_estimate_timesteps_brute_force(name, make, t, budget):
    ham = make()
    H = dense_h(ham.labels, ham.coeffs)
    r = OT.estimate_timesteps(_dia(ham), t, budget)
    scan = next(s for s in range(1, 1 << 16) if (c := _dense_diag_count(H, t / s, 1e-6)) is not None and c <= budget)
    assert r == scan
    if name == "heis4_one_step":
        assert r == 1
    assert r == 1 or _dense_diag_count(H, t / (r - 1), 1e-6) is None or _dense_diag_count(H, t / (r - 1), 1e-6) > budget


def test_estimate_timesteps_diagonal_is_one():
    A = _dia(W.Hamiltonian("zz", 3, ["ZZI", "IZZ", "ZIZ"], np.array([0.5, -1.0, 2.0])))
    assert OT.estimate_timesteps(A, 10.0, 1) == 1


def test_taylor_evolution_tracks_exact():
    """r steps of U(t/r) (Alg. 3) approach exp(-iHt) psi within r times the per-step bound."""
    ham = W.heisenberg_chain(4, np.array([0.6, 1.1, 1.4, 0.9]), periodic=True)
    H = dense_h(ham.labels, ham.coeffs)
    A = _dia(ham)
    rng = np.random.default_rng(5)
    psi = W.gaussian_state(4, rng)
    r = OT.estimate_timesteps(A, 1.0, 17)
    U, K, ok = OT.expm_taylor(A, 1.0 / r)
    got = OT.evolve(U, psi, r)
    want = _exact_expm(H, 1.0) @ psi
    nx = np.linalg.norm(H, 2) / r
    assert np.linalg.norm(got - want) <= r * 1e-6 / (1 - nx / (K + 1)) + 1e-12
    # sensitivity: stopping four terms early (a truncation mistake) breaks the bound
    assert K > 4
    Ubad = OT.expm_taylor(A, 1.0 / r, 1e-6, K - 5)[0]
    assert np.linalg.norm(OT.evolve(Ubad, psi, r) - want) > r * 1e-6 / (1 - nx / (K + 1))


def test_expectation_dense_and_eigenstate():
    """<psi|H|psi> equals the dense quadratic form; a TFIM at h = 0 has |0...0> as
    an eigenstate with energy -J * (number of bonds)."""
    rng = np.random.default_rng(31)
    ham = W.heisenberg_chain(5, rng.uniform(0.5, 1.5, 5), periodic=True)
    H = dense_h(ham.labels, ham.coeffs)
    psi = np.stack([W.gaussian_state(5, rng) for _ in range(3)])
    got = OT.expectation(_dia(ham), psi)
    want = np.einsum("ri,ij,rj->r", psi.conj(), H, psi)
    assert np.max(np.abs(got - want)) < 1e-13
    assert np.max(np.abs(got.imag)) < 1e-13  # Hermitian
    tf = W.tfim_chain(6, 0.8, 0.0, periodic=False)
    e = OT.expectation(_dia(tf), W.basis_state(6))
    assert abs(e[0] - (-0.8 * 5)) < 1e-14
