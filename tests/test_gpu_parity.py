"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: complex128 amplitudes max-abs <= 1e-12; complex64 amplitudes
max-abs <= 1e-5 with infidelity <= 1e-6; grouping, offsets and term ranges
bit-exact; factor values 1e-13 (complex128) and 1e-7 (complex64: one FP32
rounding of numbers of magnitude <= 1).
"""
import numpy as np
import pytest

import oracle as O
from paper_2606_16959_gb300 import hs, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-12, "c64": 1e-5}
TDT = {"c128": None, "c64": None}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_16959_gb300 import _build
    _build.build()
    O.build()
    hs.lib()


def tdtype(dt):
    return torch.complex64 if dt == "c64" else torch.complex128


def to_dev(psi, dt):
    return torch.from_numpy(np.ascontiguousarray(psi)).to(device="cuda", dtype=tdtype(dt))


def infidelity(a, b):
    a, b = np.asarray(a, np.complex128).ravel(), np.asarray(b, np.complex128).ravel()
    return 1.0 - abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real)


def check_state(got, want, dt):
    got = np.asarray(got, np.complex128)
    err = float(np.max(np.abs(got - want)))
    assert err <= TOL[dt], f"max-abs {err:.3e} > {TOL[dt]}"
    if dt == "c64":
        rows = got.reshape(-1, got.shape[-1])
        wr = np.asarray(want).reshape(-1, got.shape[-1])
        for g, w in zip(rows, wr):
            assert infidelity(g, w) <= 1e-6
    return err


def gpu_evolve(labels, coeffs, t, steps, budget, dt, psi0, **kw):
    f = hs.hs_build_factors(labels, coeffs, t, steps, budget, dt)
    psi = to_dev(psi0, dt)
    if kw:
        hs.hs_evolve_ex(f, psi, steps, **kw)
    else:
        hs.hs_evolve(f, psi, steps)
    out = psi.cpu().numpy()
    f.close()
    return out


def oracle_evolve(labels, coeffs, t, steps, psi0):
    x, z, _ = O.parse_terms(labels)
    return O.evolve_direct(x, z, coeffs, t, steps, psi0)


def random_terms(rng, n, m, p_id=0.5):
    p = [p_id] + [(1 - p_id) / 3] * 3
    return ["".join(rng.choice(list("IXYZ"), p=p, size=n)) for _ in range(m)], rng.uniform(-1.2, 1.2, size=m)


# ----------------------------------------------------------------------------
# Factor build
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_factor_build_matches_oracle(dt):
    rng = np.random.default_rng(101)
    cases = [(W.tfim10().ham, 10, 4), (W.heisenberg_chain(8, rng.uniform(0.5, 1.5, 8)), 7, 8),
             (W.maxcut_3regular(10, 5), 3, 4), (W.tsp_onehot(3, 9), 2, 1)]
    for n in (1, 2, 5, 9):
        labels, coeffs = random_terms(rng, n, 9)
        cases.append((W.Hamiltonian("random", n, labels, coeffs), 3, int(rng.integers(1, 12))))
    for ham, steps, budget in cases:
        x, z, n = O.parse_terms(ham.labels)
        want = O.build_factors(x, z, ham.coeffs, n, 0.9, steps, budget)
        f = hs.hs_build_factors(ham.labels, ham.coeffs, 0.9, steps, budget, dt)
        assert f.n_factors == len(want)
        tol = 1e-13 if dt == "c128" else 1e-7
        for g, w in enumerate(want):
            first, last, offs, vals = f.factor(g)
            assert (first, last) == (w.first, w.last)
            assert list(offs) == w.offsets
            assert np.max(np.abs(vals - w.values)) <= tol
        f.close()


def test_build_rejects_bad_input():
    with pytest.raises(hs.HSError) as e:
        hs.hs_build_factors(["XQ"], [1.0], 1.0, 1, 4)
    assert e.value.code == hs.HS_EINVAL
    with pytest.raises(hs.HSError):
        hs.hs_build_factors(["XX", "X"], [1.0, 1.0], 1.0, 1, 4)
    with pytest.raises(hs.HSError):
        hs.hs_build_factors(["XX"], [float("nan")], 1.0, 1, 4)
    with pytest.raises(hs.HSError):
        hs.hs_build_factors(["XX"], [1.0], -1.0, 1, 4)
    with pytest.raises(hs.HSError):
        hs.hs_build_factors(["XX"], [1.0], 1.0, 0, 4)
    with pytest.raises(hs.HSError):
        hs.hs_build_factors(["XX"], [1.0], 1.0, 1, 0)


# ----------------------------------------------------------------------------
# Single factor application (plain kernel)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("n_rhs", [1, 3, 6, 9, 20])
def test_apply_factor_matches_oracle(dt, n_rhs):
    rng = np.random.default_rng(200 + n_rhs)
    ham = W.heisenberg_chain(12, rng.uniform(0.5, 1.5, 12))
    x, z, n = O.parse_terms(ham.labels)
    facs = O.build_factors(x, z, ham.coeffs, n, 1.0, 4, 8)
    f = hs.hs_build_factors(ham.labels, ham.coeffs, 1.0, 4, 8, dt)
    psi = np.stack([W.gaussian_state(n, rng) for _ in range(n_rhs)])
    xin = to_dev(psi, dt)
    y = torch.empty_like(xin)
    for g in (0, 5, len(facs) - 1):
        hs.hs_apply_factor(f, g, xin, y)
        # the oracle applies its own factor values to the same (possibly rounded) input
        xin_np = xin.cpu().numpy().astype(np.complex128)
        want = np.stack([O.dia_apply(facs[g].offsets, facs[g].starts, facs[g].values, r) for r in xin_np])
        check_state(y.cpu().numpy(), want, dt)
    f.close()


# ----------------------------------------------------------------------------
# Evolution
# ----------------------------------------------------------------------------

METHODS = [dict(), dict(method=hs.HS_METHOD_PLAIN), dict(method=hs.HS_METHOD_FUSED),
           dict(method=hs.HS_METHOD_FUSED, use_graph=True)]


@pytest.mark.parametrize("kw", METHODS, ids=["auto", "plain", "fused", "graph"])
def test_tfim10_complex128(kw):
    """TFIM n=10 open chain, |0..0>, t=1, 10 steps, budget 4, complex128."""
    job = W.tfim10()
    got = gpu_evolve(job.ham.labels, job.ham.coeffs, job.t, job.n_steps, job.budget, "c128", job.psi0, **kw)
    check_state(got, oracle_evolve(job.ham.labels, job.ham.coeffs, job.t, job.n_steps, job.psi0), "c128")


@pytest.fixture(scope="module")
def heis16_ref():
    job = W.heis16()
    return job, oracle_evolve(job.ham.labels, job.ham.coeffs, job.t, job.n_steps, job.psi0)


@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("kw", METHODS, ids=["auto", "plain", "fused", "graph"])
def test_heis16_full_config(heis16_ref, dt, kw):
    """Periodic Heisenberg n=16, 100 steps, budget 8: complex128 and complex64."""
    job, want = heis16_ref
    got = gpu_evolve(job.ham.labels, job.ham.coeffs, job.t, job.n_steps, job.budget, dt, job.psi0, **kw)
    check_state(got, want, dt)


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_random_hamiltonians_all_paths(dt):
    rng = np.random.default_rng(300)
    for n in (1, 2, 3, 5, 8, 11, 13):
        labels, coeffs = random_terms(rng, n, int(rng.integers(1, 10)), p_id=0.6)
        budget = int(rng.integers(1, 17))
        n_rhs = int(rng.integers(1, 6))
        psi0 = np.stack([W.gaussian_state(n, rng) for _ in range(n_rhs)])
        want = oracle_evolve(labels, coeffs, 0.7, 3, psi0)
        for kw in (dict(method=hs.HS_METHOD_PLAIN), dict(method=hs.HS_METHOD_FUSED), dict()):
            got = gpu_evolve(labels, coeffs, 0.7, 3, budget, dt, psi0, **kw)
            check_state(got, want, dt)


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_small_tiles_and_plain_fallback(dt):
    """Tiles narrower than a factor's flip span force plain launches between sweeps."""
    rng = np.random.default_rng(301)
    n = 12
    labels = [W.label_of(n, {0: "X", 11: "X"}), W.label_of(n, {3: "Y", 4: "Z"}), W.label_of(n, {5: "X", 9: "Y"}),
              W.label_of(n, {2: "Z"}), W.label_of(n, {1: "X", 2: "X", 3: "X", 10: "Z"})]
    coeffs = rng.uniform(-1, 1, len(labels))
    psi0 = np.stack([W.gaussian_state(n, rng) for _ in range(3)])
    want = oracle_evolve(labels, coeffs, 1.1, 4, psi0)
    for tb, rb in ((5, 1), (6, 2), (7, 1), (8, 4)):
        got = gpu_evolve(labels, coeffs, 1.1, 4, 4, dt, psi0, method=hs.HS_METHOD_FUSED, tile_bits=tb, rhs_block=rb)
        check_state(got, want, dt)


def test_maxcut16_multi_rhs_complex64():
    """MaxCut + mixer on 16 qubits with 16 states (|+> and Gaussians), complex64."""
    job = W.maxcut24(n=16, n_rhs=16, n_steps=6)
    want = oracle_evolve(job.ham.labels, job.ham.coeffs, job.t, job.n_steps, job.psi0)
    for kw in (dict(), dict(method=hs.HS_METHOD_PLAIN), dict(method=hs.HS_METHOD_FUSED, rhs_block=4)):
        got = gpu_evolve(job.ham.labels, job.ham.coeffs, job.t, job.n_steps, job.budget, "c64", job.psi0, **kw)
        check_state(got, want, "c64")


def _cut_values(ham, n, idx):
    E = np.zeros(idx.size)
    for (i, j), w in zip(ham.meta["edges"], ham.meta["weights"]):
        E += w * (((idx >> i) & 1) != ((idx >> j) & 1))
    return E


def test_maxcut24_full_size():
    """The full MaxCut configuration (n=24, 16 states, complex64) in the default
    launch configuration: one step against the oracle on every amplitude of
    state 0; 50 steps checked for norm preservation on all 16 states; and the
    exact phase exp(-i t E(b)) of the mixer-free Hamiltonian on sampled b."""
    job = W.maxcut24()
    n = job.ham.n_qubits
    f1 = hs.hs_build_factors(job.ham.labels, job.ham.coeffs, job.t / job.n_steps, 1, job.budget, "c64")
    psi = to_dev(job.psi0, "c64")
    hs.hs_evolve(f1, psi, 1)
    one = psi[0].cpu().numpy()
    f1.close()
    want = oracle_evolve(job.ham.labels, job.ham.coeffs, job.t / job.n_steps, 1, job.psi0[0])
    check_state(one, want, "c64")
    # 50 steps: norms
    f = hs.hs_build_factors(job.ham.labels, job.ham.coeffs, job.t, job.n_steps, job.budget, "c64")
    psi = to_dev(job.psi0, "c64")
    hs.hs_evolve(f, psi, job.n_steps)
    norms = (psi.abs().double() ** 2).sum(dim=1).cpu().numpy()
    assert np.max(np.abs(norms - 1.0)) < 1e-4
    f.close()
    # mixer-free: exact phase on sampled amplitudes
    ham0 = W.maxcut(n, job.ham.meta["edges"], job.ham.meta["weights"], mixer=0.0)
    f = hs.hs_build_factors(ham0.labels, ham0.coeffs, job.t, job.n_steps, 4, "c64")
    psi = to_dev(job.psi0, "c64")
    hs.hs_evolve(f, psi, job.n_steps)
    rng = np.random.default_rng(5)
    idx = rng.integers(0, 1 << n, size=4096)
    got = psi[:, idx].cpu().numpy()
    want = np.exp(-1j * job.t * _cut_values(ham0, n, idx))[None, :] * job.psi0[:, idx]
    assert np.max(np.abs(got - want)) < 1e-5
    f.close()


def test_steps_compose_and_determinism():
    """k steps then k' steps equals k + k' steps; repeated runs are bitwise equal."""
    rng = np.random.default_rng(400)
    ham = W.heisenberg_chain(14, rng.uniform(0.5, 1.5, 14))
    f = hs.hs_build_factors(ham.labels, ham.coeffs, 1.0, 40, 8, "c64")
    psi0 = W.gaussian_state(14, rng)
    a = to_dev(psi0, "c64")
    hs.hs_evolve(f, a, 40)
    b = to_dev(psi0, "c64")
    hs.hs_evolve(f, b, 15)
    hs.hs_evolve(f, b, 25)
    c = to_dev(psi0, "c64")
    hs.hs_evolve(f, c, 40)
    assert torch.equal(a, c)
    assert torch.max(torch.abs(a - b)).item() < 1e-6
    d = to_dev(psi0, "c64")
    hs.hs_evolve_ex(f, d, 40, method=hs.HS_METHOD_FUSED, use_graph=True)
    assert torch.equal(a, d)
    f.close()


def test_identity_and_zero_steps():
    f = hs.hs_build_factors(["III"], [0.8], 2.0, 5, 1, "c128")
    psi0 = W.gaussian_state(3, np.random.default_rng(1))
    psi = to_dev(psi0, "c128")
    hs.hs_evolve(f, psi, 0)
    assert np.array_equal(psi.cpu().numpy(), psi0)
    hs.hs_evolve(f, psi, 5)
    np.testing.assert_allclose(psi.cpu().numpy(), np.exp(-1.6j) * psi0, rtol=0, atol=1e-14)
    f.close()


def test_evolve_rejects_mismatches():
    f = hs.hs_build_factors(["XX", "ZZ"], [1.0, 0.5], 1.0, 2, 4, "c64")
    with pytest.raises(hs.HSError):
        hs.hs_evolve(f, torch.zeros(4, dtype=torch.complex128, device="cuda"), 2)
    with pytest.raises(ValueError):
        hs.hs_evolve(f, torch.zeros(8, dtype=torch.complex64, device="cuda"), 2)
    with pytest.raises(hs.HSError):
        hs.hs_evolve_ex(f, torch.zeros(4, dtype=torch.complex64, device="cuda"), 2, rhs_block=3)
    f.close()


# ----------------------------------------------------------------------------
# Reductions
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("n", [1, 7, 16, 21])
def test_fidelity_and_norms(dt, n):
    rng = np.random.default_rng(500 + n)
    a = W.gaussian_state(n, rng) * 1.3
    b = a + 0.05 * W.gaussian_state(n, rng)
    da, db = to_dev(a, dt), to_dev(b, dt)
    fid, na, nb = hs.hs_fidelity(da, db)
    ah, bh = da.cpu().numpy(), db.cpu().numpy()
    assert fid == pytest.approx(O.fidelity(ah, bh), rel=1e-12, abs=1e-15)
    assert na == pytest.approx(O.norm2(ah), rel=1e-12)
    assert nb == pytest.approx(O.norm2(bh), rel=1e-12)
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    hs.hs_inner_device(da, db, out)
    ip = O.inner(ah, bh)
    o = out.cpu().numpy()
    assert o[0] == pytest.approx(ip.real, rel=1e-12, abs=1e-14)
    assert o[1] == pytest.approx(ip.imag, rel=1e-10, abs=1e-12)


def test_kernel_launch_counter_counts_each_launch():
    """hs_kernel_launches advances by exactly the kernels an entry point launches:
    3 for a factor build with value tables (angles, factor values, tables), the
    planned sweeps for an evolution, 2 for a reduction, and a graph's kernels on
    every replay."""
    ham = W.heisenberg_chain(12, np.linspace(0.5, 1.5, 12), periodic=True)
    l0 = hs.hs_kernel_launches()
    f = hs.hs_build_factors(ham.labels, ham.coeffs, 1.0, 4, 8, "c64")
    assert hs.hs_kernel_launches() - l0 == 3
    psi = torch.from_numpy(W.gaussian_state(12, np.random.default_rng(3))).to("cuda", torch.complex64)
    opts = dict(method=hs.HS_METHOD_FUSED, tile_bits=8, rhs_block=1, low_bits=1)
    n_sweeps, n_plain, _, _ = hs.hs_evolve_plan(f, 1, 4, **opts)
    l1 = hs.hs_kernel_launches()
    hs.hs_evolve_ex(f, psi, 4, **opts)
    assert hs.hs_kernel_launches() - l1 == n_sweeps + n_plain > 0
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    l2 = hs.hs_kernel_launches()
    hs.hs_inner_device(psi, psi, out)
    assert hs.hs_kernel_launches() - l2 == 2
    l3 = hs.hs_kernel_launches()
    hs.hs_evolve_ex(f, psi, 4, use_graph=True, **opts)   # capture + first replay
    hs.hs_evolve_ex(f, psi, 4, use_graph=True, **opts)   # replay
    torch.cuda.synchronize()
    assert hs.hs_kernel_launches() - l3 == 2 * (n_sweeps + n_plain)


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_value_tables_bitwise_equal_to_staged_diagonals(dt):
    """Factors whose terms touch few qubits are read from value tables (one entry
    per pattern of the row's bits on those qubits) instead of their stored
    diagonals; the values are the same numbers, so the evolution is bitwise equal."""
    rng = np.random.default_rng(77)
    tdt = torch.complex64 if dt == "c64" else torch.complex128
    lb = 2 if dt == "c64" else 1
    labels = ["".join(rng.choice(list("IXYZ"), p=[0.7, 0.1, 0.1, 0.1], size=12)) for _ in range(10)]
    hams = [W.heisenberg_chain(14, rng.uniform(0.5, 1.5, 14), periodic=True),
            W.tfim_chain(13, 1.0, 0.6, periodic=False),
            W.Hamiltonian("random", 12, labels, rng.uniform(-1, 1, 10))]
    for ham, budget in zip(hams, (8, 4, 16)):
        f = hs.hs_build_factors(ham.labels, ham.coeffs, 0.7, 6, budget, dt)
        psi = torch.from_numpy(np.stack([W.gaussian_state(ham.n_qubits, rng) for _ in range(2)])).to("cuda", tdt)
        a, b = psi.clone(), psi.clone()
        opts = dict(method=hs.HS_METHOD_FUSED, tile_bits=9, rhs_block=1, low_bits=lb)
        hs.hs_evolve_ex(f, a, 6, **opts)
        hs.hs_evolve_ex(f, b, 6, no_tables=True, **opts)
        torch.cuda.synchronize()
        assert torch.equal(a, b), ham.family
        x, z, _ = O.parse_terms(ham.labels)
        want = O.evolve_direct(x, z, ham.coeffs, 0.7, 6, psi.cpu().numpy())
        tol = 1e-12 if dt == "c128" else 1e-5
        assert np.max(np.abs(a.cpu().numpy() - want)) <= tol
        f.close()
