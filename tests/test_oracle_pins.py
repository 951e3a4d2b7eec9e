"""Pins of the FP64 oracle against things other than itself.

Each test ties one part of the oracle to the paper (Tab. 1, Tab. 3, the
appendix quick-start example), to an independent library routine (Kronecker
products of the 2x2 Pauli matrices, scipy.linalg.expm, numpy.linalg.eigh,
math.fsum), to a closed form, or to brute force on tiny inputs.  The
"sensitivity" tests plant a plausible mistake in the oracle's inputs or
outputs and check that the corresponding pin would catch it.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from conftest import read_golden
from paper_2606_16959_gb300 import workloads as W

PAULI = {
    "I": np.eye(2, dtype=complex),
    "X": np.array([[0, 1], [1, 0]], dtype=complex),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=complex),
    "Z": np.array([[1, 0], [0, -1]], dtype=complex),
}


def dense_pauli(label):
    """Kronecker product, leftmost character = most significant qubit."""
    m = np.ones((1, 1), dtype=complex)
    for ch in label:
        m = np.kron(m, PAULI[ch])
    return m


def dense_h(labels, coeffs):
    return sum(c * dense_pauli(l) for l, c in zip(labels, coeffs))


def dense_trotter(labels, coeffs, t, n_steps):
    """(prod_j expm(-i c_j dt P_j))^r with term 1 acting first, via scipy expm."""
    dt = t / n_steps
    N = 2 ** len(labels[0])
    step = np.eye(N, dtype=complex)
    for l, c in zip(labels, coeffs):
        step = scipy.linalg.expm(-1j * (c * dt) * dense_pauli(l)) @ step
    return np.linalg.matrix_power(step, n_steps)


def random_labels(rng, n, m, alphabet="IXYZ"):
    return ["".join(rng.choice(list(alphabet), size=n)) for _ in range(m)]


def dense_from_dia(N, offsets, starts, vals):
    """Independent rebuild with numpy.diag: diagonal d holds N-|d| entries."""
    M = np.zeros((N, N), dtype=complex)
    for d, s in zip(offsets, starts):
        L = N - abs(d)
        M += np.diag(vals[s:s + L], d)
    return M


# ----------------------------------------------------------------------------
# Pauli action (brute force against Kronecker products)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_pauli_action_matches_kronecker(oracle, n):
    rng = np.random.default_rng(10 + n)
    for label in random_labels(rng, n, 12) + ["Y" * n, "X" * n, "Z" * n]:
        x, z = oracle.parse_label(label)
        P = dense_pauli(label)
        N = 2 ** n
        got = np.stack([oracle.pauli_apply(x, z, np.eye(N)[:, b]) for b in range(N)], axis=1)
        np.testing.assert_allclose(got, P, atol=0, rtol=0)


def test_parse_rejects_bad_labels(oracle):
    with pytest.raises(ValueError):
        oracle.parse_label("XQZ")
    with pytest.raises(ValueError):
        oracle.parse_terms(["XX", "XYZ"])


def test_quickstart_matrix_and_spmv(oracle):
    """Appendix quick start: H @ e0; the same H is XX + YY + ZZ on 2 qubits."""
    g = read_golden("quickstart_spmv.txt")
    H = np.array(g["matrix"], dtype=complex)
    psi = np.array(g["psi"], dtype=complex)
    y = np.array(g["y"], dtype=complex)
    # H from the oracle's Pauli action
    labels = ["XX", "YY", "ZZ"]
    Hp = np.zeros((4, 4), dtype=complex)
    for l in labels:
        x, z = oracle.parse_label(l)
        Hp += np.stack([oracle.pauli_apply(x, z, np.eye(4)[:, b]) for b in range(4)], axis=1)
    np.testing.assert_array_equal(Hp, H)
    offs, st, vals = oracle.dia_from_dense(H)
    assert offs == [0, -1, 1]
    np.testing.assert_array_equal(oracle.dia_apply(offs, st, vals, psi), y)
    # numeric structure: the +-3 diagonals of XX and YY cancel exactly
    x, z, _ = oracle.parse_terms(labels)
    ndiag, nnz = oracle.hamiltonian_structure(x, z, [1.0, 1.0, 1.0], 2)
    assert (ndiag, nnz) == (3, 6)


# ----------------------------------------------------------------------------
# Layout (Tab. 1) and the diagonal-times-vector product (Alg. 1)
# ----------------------------------------------------------------------------

def test_tab1_layout(oracle):
    g = read_golden("tab1_layout.txt")
    M = np.array(g["matrix"], dtype=complex)
    offs, st, vals = oracle.dia_from_dense(M)
    assert offs == [int(v) for v in g["offsets"]]
    np.testing.assert_array_equal(vals.real, g["values"])
    assert list(st) == [0, 4, 5]
    v = np.array([1 + 2j, -3j, 0.5, 7.0])
    np.testing.assert_allclose(oracle.dia_apply(offs, st, vals, v), M @ v, rtol=0, atol=1e-14)


def test_dia_apply_random_against_dense(oracle):
    rng = np.random.default_rng(3)
    N = 64
    for _ in range(10):
        offs = oracle.canonical_order(set(rng.choice(np.arange(-(N - 1), N), size=7, replace=False)) | {0})
        st = oracle.starts_of(offs, N)
        total = int(st[-1] + N - abs(offs[-1]))
        vals = rng.standard_normal(total) + 1j * rng.standard_normal(total)
        x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        M = dense_from_dia(N, offs, st, vals)
        np.testing.assert_allclose(oracle.dia_apply(offs, st, vals, x), M @ x, rtol=0, atol=1e-12)


def test_dia_apply_sensitivity_transposed_operand(oracle):
    """A transposed operand (reading x[i-d] instead of x[i+d]) must be visible."""
    rng = np.random.default_rng(4)
    N = 32
    offs = [0, -3, 3, 5]
    st = oracle.starts_of(offs, N)
    vals = rng.standard_normal(int(st[-1] + N - 5)) + 0j
    x = rng.standard_normal(N) + 0j
    M = dense_from_dia(N, offs, st, vals)
    assert np.max(np.abs(M.T @ x - oracle.dia_apply(offs, st, vals, x))) > 1e-3


# ----------------------------------------------------------------------------
# Grouping and structural offsets (closed forms, brute force, Tab. 3)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("k", [0, 1, 5, 9])
def test_single_x_offsets(oracle, k):
    g = oracle.group_terms([1 << k], budget=1)
    assert len(g) == 1 and g[0].offsets == [0, -(1 << k), 1 << k]


@pytest.mark.parametrize("i", [0, 3, 7])
def test_xx_bond_offsets(oracle, i):
    x = (1 << i) | (1 << (i + 1))
    g = oracle.group_terms([x], budget=1)  # over budget: a single term still forms a factor
    assert g[0].offsets == [0, -(1 << i), 1 << i, -3 * (1 << i), 3 * (1 << i)]


def test_offsets_brute_force(oracle):
    """O(X) equals the set of col-row over all (row, col) with row^col in X."""
    rng = np.random.default_rng(5)
    n = 6
    N = 2 ** n
    for _ in range(20):
        masks = [int(v) for v in rng.integers(0, N, size=3)]
        g = oracle.group_terms(masks, budget=10 ** 9)[0]
        Xs = set(g.X)
        brute = {c - r for r in range(N) for c in range(N) if (r ^ c) in Xs}
        assert set(g.offsets) == brute
        assert g.offsets == sorted(brute, key=lambda d: (abs(d), d))


def test_grouping_of_benchmark_families(oracle):
    tf = W.tfim_chain(10, 1.0, 1.0, periodic=False)
    x, _, _ = oracle.parse_terms(tf.labels)
    g = oracle.group_terms(x, 4)
    assert [(a.first, a.last) for a in g] == [(0, 10)] + [(9 + k, 10 + k) for k in range(1, 10)]
    assert all(len(a.offsets) == 3 for a in g)
    hz = W.heisenberg_chain(16, np.ones(16), periodic=True)
    x, _, _ = oracle.parse_terms(hz.labels)
    g = oracle.group_terms(x, 8)
    assert [(a.first, a.last) for a in g] == [(3 * k, 3 * k + 3) for k in range(16)]
    assert [len(a.offsets) for a in g] == [5] * 15 + [5]
    # wrap-around bond (15, 0): x = 2^15 + 1 -> offsets +-2^15 +-1
    assert g[15].offsets == [0, -(2 ** 15 - 1), 2 ** 15 - 1, -(2 ** 15 + 1), 2 ** 15 + 1]
    assert g[0].offsets == [0, -1, 1, -3, 3]
    mc = W.maxcut_3regular(24, 1003)
    x, _, _ = oracle.parse_terms(mc.labels)
    g = oracle.group_terms(x, 4)
    assert len(g) == 24 and all(len(a.offsets) == 3 for a in g)
    assert (g[0].first, g[0].last) == (0, 1 + 36 + 1)
    ts = W.tsp_onehot(4, 7)
    x, _, _ = oracle.parse_terms(ts.labels)
    g = oracle.group_terms(x, 1)
    assert len(g) == 1 and g[0].offsets == [0]


def test_grouping_admit_rule(oracle):
    # same-mask terms never split a group; a diagonal term never splits a group
    g = oracle.group_terms([0b11, 0b11, 0, 0b11], budget=1)
    assert len(g) == 1
    # budget exactly met, then exceeded
    g = oracle.group_terms([1, 2], budget=7)
    assert len(g) == 1 and len(g[0].offsets) == 7
    g = oracle.group_terms([1, 2], budget=6)
    assert [(a.first, a.last) for a in g] == [(0, 1), (1, 2)]
    with pytest.raises(ValueError):
        oracle.group_terms([1], budget=0)


def _family(row):
    label, fam, n, bc = row[0], row[1], int(row[2]), row[3]
    if fam == "tfim":
        return W.tfim_chain(n, 1.0, 1.0, periodic=(bc == "pbc"))
    if fam == "heisenberg":
        nb = n if bc == "pbc" else n - 1
        return W.heisenberg_chain(n, np.ones(nb), periodic=(bc == "pbc"))
    return W.tsp_onehot(4, 11)


@pytest.mark.parametrize("row", read_golden("tab3_structure.txt")["rows"], ids=lambda r: r[0])
def test_tab3_structure(oracle, row):
    ham = _family(row)
    x, z, n = oracle.parse_terms(ham.labels)
    assert n == int(row[2])
    ndiag, nnz = oracle.hamiltonian_structure(x, z, ham.coeffs, n)
    assert ndiag == int(row[4])
    if row[5] != "-":
        N = 2 ** n
        assert round(100.0 * (1.0 - nnz / (N * N)), 4) == pytest.approx(float(row[5]), abs=5e-5)


# ----------------------------------------------------------------------------
# Factor values (dense products through scipy expm)
# ----------------------------------------------------------------------------

def _check_factors_against_dense(oracle, labels, coeffs, t, steps, budget):
    x, z, n = oracle.parse_terms(labels)
    N = 2 ** n
    facs = oracle.build_factors(x, z, coeffs, n, t, steps, budget)
    dt = t / steps
    for f in facs:
        F = np.eye(N, dtype=complex)
        for j in range(f.first, f.last):
            F = scipy.linalg.expm(-1j * (coeffs[j] * dt) * dense_pauli(labels[j])) @ F
        # numeric entries lie on the structural offsets ...
        mask = np.zeros((N, N), dtype=bool)
        for d in f.offsets:
            mask |= np.eye(N, k=d, dtype=bool)
        assert np.max(np.abs(F[~mask]), initial=0.0) < 1e-14
        # ... and match the materialised layout
        np.testing.assert_allclose(dense_from_dia(N, f.offsets, f.starts, f.values), F, rtol=0, atol=1e-13)
    return facs


def test_factor_values_random_groups(oracle):
    rng = np.random.default_rng(6)
    for n in (2, 3, 5):
        for budget in (1, 3, 5, 9, 16):
            labels = random_labels(rng, n, 7)
            coeffs = rng.uniform(-1.5, 1.5, size=len(labels))
            _check_factors_against_dense(oracle, labels, coeffs, 0.7, 3, budget)


def test_factor_values_heisenberg_and_tfim(oracle):
    h = W.heisenberg_chain(6, [0.7, 1.1, 0.9, 1.3, 0.6, 1.0], periodic=True)
    _check_factors_against_dense(oracle, h.labels, h.coeffs, 1.0, 4, 8)
    t = W.tfim_chain(6, 1.0, 0.8, periodic=False)
    _check_factors_against_dense(oracle, t.labels, t.coeffs, 1.0, 4, 4)


def test_factor_sensitivity_order_and_sign(oracle):
    """Reversed product order or a flipped rotation sign would break the dense pin."""
    labels, coeffs = ["XY", "ZX", "YY"], np.array([0.9, -0.4, 1.2])
    x, z, n = oracle.parse_terms(labels)
    f = oracle.build_factors(x, z, coeffs, n, 1.0, 1, 64)[0]
    got = dense_from_dia(4, f.offsets, f.starts, f.values)
    rev = np.eye(4, dtype=complex)
    for l, c in list(zip(labels, coeffs))[::-1]:
        rev = scipy.linalg.expm(-1j * c * dense_pauli(l)) @ rev
    flip = np.eye(4, dtype=complex)
    for l, c in zip(labels, coeffs):
        flip = scipy.linalg.expm(+1j * c * dense_pauli(l)) @ flip
    assert np.max(np.abs(got - rev)) > 1e-2
    assert np.max(np.abs(got - flip)) > 1e-2


# ----------------------------------------------------------------------------
# Evolution: dense Trotter product, exact exponential, exact special cases
# ----------------------------------------------------------------------------

def test_direct_evolution_matches_dense_trotter(oracle):
    rng = np.random.default_rng(7)
    for n in (2, 4, 6):
        labels = random_labels(rng, n, 9)
        coeffs = rng.uniform(-1, 1, size=len(labels))
        x, z, _ = oracle.parse_terms(labels)
        psi0 = W.gaussian_state(n, rng)
        for steps in (1, 3):
            got = oracle.evolve_direct(x, z, coeffs, 0.8, steps, psi0)
            want = dense_trotter(labels, coeffs, 0.8, steps) @ psi0
            np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_direct_evolution_sensitivity_dropped_term(oracle):
    rng = np.random.default_rng(8)
    labels = random_labels(rng, 4, 6, "XYZ")
    coeffs = rng.uniform(0.5, 1, size=6)
    x, z, _ = oracle.parse_terms(labels)
    psi0 = W.gaussian_state(4, rng)
    got = oracle.evolve_direct(x[:-1], z[:-1], coeffs[:-1], 0.8, 2, psi0)
    want = dense_trotter(labels, coeffs, 0.8, 2) @ psi0
    assert np.max(np.abs(got - want)) > 1e-3


def _commutator_bound(labels, coeffs, t, r):
    """First-order Trotter bound (t^2 / 2r) sum_{j<k} ||[c_j P_j, c_k P_k]||;
    for Pauli strings the commutator norm is 2|c_j c_k| if they anticommute, else 0."""
    s = 0.0
    for j in range(len(labels)):
        for k in range(j + 1, len(labels)):
            Pj, Pk = dense_pauli(labels[j]), dense_pauli(labels[k])
            if not np.allclose(Pj @ Pk, Pk @ Pj):
                s += 2 * abs(coeffs[j] * coeffs[k])
    return t * t / (2 * r) * s


def test_trotter_error_against_exact_exponential(oracle):
    ham = W.tfim_chain(6, 1.0, 0.9, periodic=False)
    H = dense_h(ham.labels, ham.coeffs)
    w, V = np.linalg.eigh(H)
    psi0 = W.basis_state(6)
    t = 1.0
    exact = V @ (np.exp(-1j * w * t) * (V.conj().T @ psi0))
    x, z, _ = oracle.parse_terms(ham.labels)
    errs = []
    for r in (20, 40, 80):
        got = oracle.evolve_direct(x, z, ham.coeffs, t, r, psi0)
        err = np.linalg.norm(got - exact)
        assert err <= _commutator_bound(ham.labels, ham.coeffs, t, r)
        errs.append(err)
    # first order: halving dt halves the error
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2


def test_exact_for_commuting_terms_n10(oracle):
    """Dense exp(-iHt) on 10 qubits for a commuting H (diagonal ZZ + Z) equals the
    Trotter product for any step count."""
    rng = np.random.default_rng(9)
    n = 10
    labels = [W.label_of(n, {i: "Z", (i + 3) % n: "Z"}) for i in range(n)] + [W.label_of(n, {i: "Z"}) for i in range(n)]
    coeffs = rng.uniform(-1, 1, size=len(labels))
    H = dense_h(labels, coeffs)
    w, V = np.linalg.eigh(H)
    psi0 = W.gaussian_state(n, rng)
    exact = V @ (np.exp(-1j * w * 1.3) * (V.conj().T @ psi0))
    x, z, _ = oracle.parse_terms(labels)
    for steps in (1, 5):
        np.testing.assert_allclose(oracle.evolve_direct(x, z, coeffs, 1.3, steps, psi0), exact, rtol=0, atol=1e-12)


def _cut_value(edges, weights, b):
    return sum(w for (i, j), w in zip(edges, weights) if ((b >> i) & 1) != ((b >> j) & 1))


def test_maxcut_exact_phase(oracle):
    """Diagonal H: psi_T[b] = exp(-i t E(b)) psi_0[b], E = cut value on bitstrings."""
    ham = W.maxcut(10, *_graph_and_weights(10, 21), mixer=0.0)
    rng = np.random.default_rng(22)
    psi0 = W.gaussian_state(10, rng)
    E = np.array([_cut_value(ham.meta["edges"], ham.meta["weights"], b) for b in range(1 << 10)])
    x, z, _ = oracle.parse_terms(ham.labels)
    for steps in (1, 7):
        got = oracle.evolve_direct(x, z, ham.coeffs, 2.0, steps, psi0)
        np.testing.assert_allclose(got, np.exp(-2.0j * E) * psi0, rtol=0, atol=1e-12)
    facs = oracle.build_factors(x, z, ham.coeffs, 10, 2.0, 7, 4)
    assert len(facs) == 1 and facs[0].offsets == [0]
    np.testing.assert_allclose(oracle.evolve_factors(facs, psi0, 7), np.exp(-2.0j * E) * psi0, rtol=0, atol=1e-12)


def _graph_and_weights(n, seed):
    rng = np.random.default_rng(seed)
    edges = W.random_regular_graph(n, 3, rng)
    return edges, rng.uniform(0, 1, size=len(edges))


def test_random_regular_graph_is_simple_3_regular():
    edges = W.random_regular_graph(24, 3, np.random.default_rng(1003))
    deg = np.zeros(24, int)
    for a, b in edges:
        assert a < b
        deg[a] += 1
        deg[b] += 1
    assert len(edges) == 36 and len(set(edges)) == 36 and (deg == 3).all()


def _tsp_cost(ham, b):
    nc, d, A = ham.meta["n_cities"], ham.meta["dist"], ham.meta["A"]
    x = lambda v, p: (b >> W.tsp_qubit(v, p, nc)) & 1
    c = sum(A * (1 - sum(x(v, p) for p in range(nc))) ** 2 for v in range(nc))
    c += sum(A * (1 - sum(x(v, p) for v in range(nc))) ** 2 for p in range(nc))
    c += sum(d[u, v] * x(u, p) * x(v, (p + 1) % nc) for u in range(nc) for v in range(nc) if u != v for p in range(nc))
    return c


def test_tsp_exact_phase(oracle):
    ham = W.tsp_onehot(4, 31)
    N = 1 << 16
    E = np.array([_tsp_cost(ham, b) for b in range(N)])
    assert E.min() > 0  # cost positive everywhere: one diagonal, no zeros (Tab. 3 TSP rows)
    rng = np.random.default_rng(32)
    psi0 = W.gaussian_state(16, rng)
    x, z, _ = oracle.parse_terms(ham.labels)
    got = oracle.evolve_direct(x, z, ham.coeffs, 0.3, 2, psi0)
    np.testing.assert_allclose(got, np.exp(-0.3j * E) * psi0, rtol=0, atol=1e-11)


def test_tfim_free_spins_closed_form(oracle):
    """J = 0: H = -h sum X_i; |0> -> tensor_i (cos(ht)|0> + i sin(ht)|1>) for any r."""
    n, h, t = 8, 0.7, 1.4
    ham = W.tfim_chain(n, 0.0, h)
    x, z, _ = oracle.parse_terms(ham.labels)
    one = np.array([math.cos(h * t), 1j * math.sin(h * t)])
    want = np.ones(1, dtype=complex)
    for _ in range(n):
        want = np.kron(one, want)
    for steps in (1, 6):
        np.testing.assert_allclose(oracle.evolve_direct(x, z, ham.coeffs, t, steps, W.basis_state(n)), want,
                                   rtol=0, atol=1e-13)


def test_norm_preserved_every_step(oracle):
    rng = np.random.default_rng(12)
    ham = W.heisenberg_chain(8, rng.uniform(0.5, 1.5, size=8))
    x, z, _ = oracle.parse_terms(ham.labels)
    psi = W.gaussian_state(8, rng)
    for _ in range(5):
        psi = oracle.evolve_direct(x, z, ham.coeffs, 0.25, 1, psi)
        assert abs(oracle.norm2(psi) - 1.0) < 1e-13


def test_heisenberg_conserves_hamming_weight(oracle):
    rng = np.random.default_rng(13)
    n = 8
    ham = W.heisenberg_chain(n, rng.uniform(0.5, 1.5, size=n))
    x, z, _ = oracle.parse_terms(ham.labels)
    psi0 = W.gaussian_state(n, rng)
    psi = oracle.evolve_direct(x, z, ham.coeffs, 1.0, 9, psi0)
    wt = np.array([bin(b).count("1") for b in range(1 << n)])
    for k in range(n + 1):
        assert abs(np.sum(np.abs(psi[wt == k]) ** 2) - np.sum(np.abs(psi0[wt == k]) ** 2)) < 1e-13


# ----------------------------------------------------------------------------
# Grouping is fusion: the diagonal-layout path equals the direct path
# ----------------------------------------------------------------------------

def test_factor_path_equals_direct_tfim10(oracle):
    job = W.tfim10()
    x, z, n = oracle.parse_terms(job.ham.labels)
    facs = oracle.build_factors(x, z, job.ham.coeffs, n, job.t, job.n_steps, job.budget)
    assert len(facs) == 10
    a = oracle.evolve_factors(facs, job.psi0, job.n_steps)
    b = oracle.evolve_direct(x, z, job.ham.coeffs, job.t, job.n_steps, job.psi0)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-13)


def test_factor_path_equals_direct_random(oracle):
    rng = np.random.default_rng(14)
    for n in (3, 6):
        labels = random_labels(rng, n, 10)
        coeffs = rng.uniform(-1, 1, size=10)
        x, z, _ = oracle.parse_terms(labels)
        psi0 = np.stack([W.gaussian_state(n, rng) for _ in range(2)])
        for budget in (1, 4, 16):
            facs = oracle.build_factors(x, z, coeffs, n, 0.9, 3, budget)
            a = oracle.evolve_factors(facs, psi0, 3)
            b = oracle.evolve_direct(x, z, coeffs, 0.9, 3, psi0)
            np.testing.assert_allclose(a, b, rtol=0, atol=1e-13)


# ----------------------------------------------------------------------------
# Reductions (math.fsum is exactly rounded)
# ----------------------------------------------------------------------------

def test_norm_inner_fidelity(oracle):
    rng = np.random.default_rng(15)
    a = rng.standard_normal(1000) + 1j * rng.standard_normal(1000)
    b = rng.standard_normal(1000) + 1j * rng.standard_normal(1000)
    n2 = math.fsum((a.real ** 2 + a.imag ** 2).tolist())
    assert oracle.norm2(a) == pytest.approx(n2, rel=1e-15)
    p = np.conj(a) * b
    ip = oracle.inner(a, b)
    assert ip.real == pytest.approx(math.fsum(p.real.tolist()), rel=1e-14)
    assert ip.imag == pytest.approx(math.fsum(p.imag.tolist()), rel=1e-14)
    assert oracle.fidelity(a, a * np.exp(0.3j)) == pytest.approx(1.0, abs=1e-15)
    e0, e1 = np.eye(4)[0], np.eye(4)[1]
    assert oracle.fidelity(e0, e1) == 0.0
