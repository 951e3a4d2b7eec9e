"""GPU parity of the register-blocked sweeps (HS_METHOD_REG) against the FP64 oracle.

The register sweep applies a factor with a small value table from the table,
and any other factor term by term: exact rotations for the non-diagonal terms
and, for runs of diagonal terms, phases generated for every row from
(z_j, theta_j) instead of read from stored diagonals.  The tests cover both
kinds of factor (TFIM and MaxCut groups with wide ZZ runs, Heisenberg bond
tables including the non-window wrap-around bond, one-hot TSP as a pure phase,
random Pauli sums with Y and Z on register, thread and tile bits, terms that
flip three qubits and fall back to plain launches), both register widths,
several tile and low-bit choices, 16-state MaxCut, the higher-order formulas,
time-dependent H(t), graph replay, and the launch plan.
Tolerances: complex128 max-abs 1e-12; complex64 max-abs 1e-5, infidelity 1e-6.
"""
import numpy as np
import pytest

import oracle as O
from paper_2606_16959_gb300 import hs, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REG = hs.HS_METHOD_REG


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_16959_gb300 import _build
    _build.build()
    O.build()
    hs.lib()


def _tdt(dt):
    return torch.complex64 if dt == "c64" else torch.complex128


def _check(got, want, dt, what=""):
    got = np.asarray(got, np.complex128).reshape(np.shape(want))
    err = float(np.max(np.abs(got - want)))
    if dt == "c128":
        assert err <= 1e-12, f"{what}: max-abs {err:.3e}"
        return
    assert err <= 1e-5, f"{what}: max-abs {err:.3e}"
    g2, w2 = got.reshape(-1, got.shape[-1]), np.asarray(want).reshape(-1, got.shape[-1])
    for a, b in zip(g2, w2):
        assert 1 - O.fidelity(a, b) <= 1e-6, what


def _evolve(ham, t, steps, budget, dt, psi0, order=1, **kw):
    f = hs.hs_build_factors(ham.labels, ham.coeffs, t, steps, budget, dt, order=order)
    psi = torch.from_numpy(np.ascontiguousarray(psi0)).to("cuda", _tdt(dt))
    hs.hs_evolve_ex(f, psi, steps, **kw)
    out = psi.cpu().numpy()
    f.close()
    return out


def _oracle(ham, t, steps, psi0, order=1):
    x, z, _ = O.parse_terms(ham.labels)
    if order == 1:
        return O.evolve_direct(x, z, ham.coeffs, t, steps, psi0)
    return O.evolve_direct_order(x, z, ham.coeffs, t, steps, psi0, order)


def _random_ham(rng, n, m):
    """Pauli sums whose terms flip at most two qubits (register ops) plus a few
    diagonal terms with wide z support (phase runs)."""
    labels = []
    for _ in range(m):
        k = int(rng.integers(1, 4))
        qs = rng.choice(n, size=k, replace=False)
        ops = {int(q): str(rng.choice(list("XYZ"))) for q in qs}
        if sum(1 for p in ops.values() if p in "XY") > 2:
            ops[int(qs[0])] = "Z"
        labels.append(W.label_of(n, ops))
    for _ in range(3):
        qs = rng.choice(n, size=int(rng.integers(2, n)), replace=False)
        labels.append(W.label_of(n, {int(q): "Z" for q in qs}))
    return W.Hamiltonian("random", n, labels, rng.uniform(-1.2, 1.2, len(labels)))


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_reg_random_pauli_sums(dt):
    rng = np.random.default_rng(4100)
    for n in (10, 11, 13, 15):
        ham = _random_ham(rng, n, 14)
        psi0 = np.stack([W.gaussian_state(n, rng) for _ in range(2)])
        want = _oracle(ham, 0.8, 3, psi0)
        for budget in (4, 8, 16):
            for B in ((4, 5) if dt == "c64" else (4,)):
                got = _evolve(ham, 0.8, 3, budget, dt, psi0, method=REG, reg_bits=B)
                _check(got, want, dt, f"n={n} budget={budget} B={B}")


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_reg_chains_tiles_and_low_bits(dt):
    rng = np.random.default_rng(4101)
    n = 14
    hams = [(W.tfim_chain(n, 1.0, 0.7), 4), (W.tfim_chain(n, 0.8, 1.3), 8), (W.tfim_chain(n, 1.1, 0.4), 16),
            (W.heisenberg_chain(n, rng.uniform(0.5, 1.5, n), periodic=True), 8),
            (W.heisenberg_chain(n, rng.uniform(0.5, 1.5, n), periodic=True), 4)]
    psi0 = np.stack([W.gaussian_state(n, rng) for _ in range(3)])
    for ham, budget in hams:
        want = _oracle(ham, 1.0, 5, psi0)
        for tb, lb in ((0, 0), (10, 1), (11, 3), (12, 2), (13, 4)):
            if dt == "c128" and tb and tb < 9:
                continue
            got = _evolve(ham, 1.0, 5, budget, dt, psi0, method=REG, tile_bits=tb, low_bits=lb, reg_bits=4)
            _check(got, want, dt, f"{ham.family} budget={budget} tb={tb} lb={lb}")


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_reg_large_angles_every_quarter_turn(dt):
    """X-type rotations with angles over [-pi, pi] (every k = rint(2 theta / pi)
    mod 4 of the tan-form split, including the swapped-partner cases), single
    and two-qubit flips, between diagonal terms, against the oracle."""
    rng = np.random.default_rng(4103)
    n = 14
    labels, coeffs = [], []
    for q in range(n):
        labels.append(W.label_of(n, {q: "X"}))
        labels.append(W.label_of(n, {q: "Z", (q + 3) % n: "Z"}))
    for q in (0, 2, 5, 9, 12):
        labels.append(W.label_of(n, {q: "X", (q + 1) % n: "X"}))
    labels.append(W.label_of(n, {1: "X", 11: "X"}))
    coeffs = rng.uniform(-6.0, 6.0, len(labels))
    ham = W.Hamiltonian("random", n, labels, coeffs)
    t, steps = 1.0, 2  # theta = c * 0.5 spans about [-3, 3]
    thetas = np.asarray(coeffs) * t / steps
    ks = {int(np.rint(2 * th / np.pi)) % 4 for th in thetas}
    assert ks == {0, 1, 2, 3}
    psi0 = np.stack([W.gaussian_state(n, rng) for _ in range(2)])
    want = _oracle(ham, t, steps, psi0)
    for budget in (1, 4):
        for B in ((4, 5) if dt == "c64" else (4,)):
            got = _evolve(ham, t, steps, budget, dt, psi0, method=REG, reg_bits=B)
            _check(got, want, dt, f"budget={budget} B={B}")


def test_reg_maxcut_sixteen_states_and_tsp():
    job = W.maxcut24(n=16, n_rhs=16, n_steps=6)
    want = _oracle(job.ham, job.t, job.n_steps, job.psi0)
    for B in (5, 4):
        got = _evolve(job.ham, job.t, job.n_steps, job.budget, "c64", job.psi0, method=REG, reg_bits=B)
        _check(got, want, "c64", f"maxcut16 B={B}")
    # 2^14-row tiles (512 threads per CTA)
    for lb in (2, 3, 4):
        got = _evolve(job.ham, job.t, job.n_steps, job.budget, "c64", job.psi0, method=REG, reg_bits=5, tile_bits=14,
                      low_bits=lb)
        _check(got, want, "c64", f"maxcut16 T=14 lb={lb}")
    # one-hot TSP (16 qubits, every term diagonal): one phase run per step
    rng = np.random.default_rng(4102)
    tsp = W.tsp_onehot(4, 1234)
    psi0 = np.stack([W.gaussian_state(16, rng) for _ in range(2)])
    want = _oracle(tsp, 0.7, 4, psi0)
    for dt in ("c64", "c128"):
        got = _evolve(tsp, 0.7, 4, 1, dt, psi0, method=REG)
        _check(got, want, dt, f"tsp {dt}")


@pytest.mark.parametrize("order", [2, 4])
def test_reg_higher_order(order):
    rng = np.random.default_rng(4103 + order)
    n = 12
    for ham, budget in ((W.tfim_chain(n, 1.0, 0.9), 8), (W.heisenberg_chain(n, rng.uniform(0.5, 1.5, n)), 8),
                        (W.maxcut_3regular(n, 55), 4)):
        psi0 = W.gaussian_state(n, rng)
        want = _oracle(ham, 0.9, 3, psi0, order)
        for dt in ("c64", "c128"):
            got = _evolve(ham, 0.9, 3, budget, dt, psi0, order=order, method=REG)
            _check(got, want, dt, f"{ham.family} order {order} {dt}")


def test_reg_three_qubit_flips_fall_back_to_plain():
    rng = np.random.default_rng(4104)
    n = 12
    labels = [W.label_of(n, {0: "X", 5: "X", 9: "Y"}), W.label_of(n, {2: "Z", 3: "Z", 11: "Z"}),
              W.label_of(n, {4: "X"}), W.label_of(n, {1: "Y", 7: "Z"})]
    ham = W.Hamiltonian("random", n, labels, rng.uniform(-1, 1, len(labels)))
    f = hs.hs_build_factors(ham.labels, ham.coeffs, 0.6, 3, 8, "c64")
    n_sw, n_plain, _, _ = hs.hs_evolve_plan(f, 1, 3, method=REG)
    assert n_plain >= 3  # the factor holding the three-qubit flip, once per step
    f.close()
    psi0 = W.gaussian_state(n, rng)
    _check(_evolve(ham, 0.6, 3, 8, "c64", psi0, method=REG), _oracle(ham, 0.6, 3, psi0), "c64", "fallback")


def test_reg_time_dependent_and_graph():
    rng = np.random.default_rng(4105)
    t, steps = 0.9, 6
    fv = W.midpoint_samples(lambda s: np.cos(2.3 * s) + 0.4 * s, t, steps)
    for ham, budget in ((W.anneal_maxcut(14, seed=77), 4), (W.driven_tfim(13, 1.0, 0.9), 8)):
        x, z, n = O.parse_terms(ham.labels)
        psi0 = np.stack([W.gaussian_state(n, rng) for _ in range(2)])
        for dt in ("c64", "c128"):
            want = O.evolve_direct_td(x, z, ham.a, ham.b, fv, t, psi0, 1)
            for graph in (False, True):
                f = hs.hs_build_factors_td(x, z, ham.a, ham.b, n, t, steps, budget, dt)
                psi = torch.from_numpy(psi0).to("cuda", _tdt(dt))
                hs.hs_evolve_td(f, psi, fv, method=REG, use_graph=graph)
                _check(psi.cpu().numpy(), want, dt, f"{ham.family} td {dt} graph={graph}")
                # the stored values are left at the last drive sample
                _, _, _, vals = f.factor(0)
                g = hs.hs_build_factors_masks(x, z, ham.a + fv[-1] * ham.b, n, t, steps, budget, dt)
                _, _, _, ref = g.factor(0)
                assert np.max(np.abs(vals - ref)) <= (1e-13 if dt == "c128" else 1e-7)
                g.close()
                f.close()


def test_reg_time_dependent_sweeps_span_steps():
    """Register sweeps of a time-dependent set read per-step term records, so
    a sweep spans steps as in the time-independent schedule: the launches are
    that schedule's sweeps plus the record and end-of-run rebuild kernels, and
    the result matches the oracle at every step count (a sweep that starts
    mid-run included)."""
    rng = np.random.default_rng(4107)
    ham = W.anneal_maxcut(16, seed=78)
    x, z, n = O.parse_terms(ham.labels)
    t = 1.1
    for steps in (2, 7, 12):
        fv = W.midpoint_samples(lambda s: 0.3 + np.sin(1.7 * s), t, steps)
        psi0 = W.gaussian_state(n, rng)
        want = O.evolve_direct_td(x, z, ham.a, ham.b, fv, t, psi0[None], 1)
        f = hs.hs_build_factors_td(x, z, ham.a, ham.b, n, t, steps, 4, "c64")
        n_sw, n_plain, _, _ = hs.hs_evolve_td_plan(f, 1, steps, method=REG)
        assert n_plain == 0
        if steps >= 7:  # fewer launches than one step's schedule repeated
            assert n_sw < steps * hs.hs_evolve_td_plan(f, 1, 1, method=REG)[0]
        psi = torch.from_numpy(psi0[None]).to("cuda", torch.complex64)
        torch.cuda.synchronize()
        before = hs.hs_kernel_launches()
        hs.hs_evolve_td(f, psi, fv, method=REG)
        torch.cuda.synchronize()
        used = hs.hs_kernel_launches() - before
        assert used <= n_sw + 5, (steps, used, n_sw)
        _check(psi.cpu().numpy(), want, "c64", f"anneal16 td steps={steps}")
        f.close()
    g = hs.hs_build_factors(ham.labels, ham.a, t, 4, 4, "c64")
    with pytest.raises(hs.HSError):
        hs.hs_evolve_td_plan(g, 1, 4, method=REG)  # a static set
    g.close()


def test_reg_graph_replay_and_steps_compose():
    rng = np.random.default_rng(4106)
    ham = W.tfim_chain(15, 1.0, 0.8)
    f = hs.hs_build_factors(ham.labels, ham.coeffs, 1.0, 20, 8, "c64")
    psi0 = W.gaussian_state(15, rng)
    a = torch.from_numpy(psi0).to("cuda", torch.complex64)
    hs.hs_evolve_ex(f, a, 20, method=REG)
    b = torch.from_numpy(psi0).to("cuda", torch.complex64)
    hs.hs_evolve_ex(f, b, 20, method=REG, use_graph=True)
    c = torch.from_numpy(psi0).to("cuda", torch.complex64)
    hs.hs_evolve_ex(f, c, 20, method=REG, use_graph=True)  # replay
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(a, c)
    d = torch.from_numpy(psi0).to("cuda", torch.complex64)
    hs.hs_evolve_ex(f, d, 7, method=REG)
    hs.hs_evolve_ex(f, d, 13, method=REG)
    assert torch.max(torch.abs(a - d)).item() < 1e-6
    _check(a.cpu().numpy(), _oracle(ham, 1.0, 20, psi0), "c64", "tfim15")
    f.close()


def test_reg_maxcut24_against_fused_path():
    """The full 24-qubit, 16-state MaxCut instance for two steps: the register
    sweeps against the staged sweeps (both complex64) and state 0 against the
    oracle on every amplitude."""
    job = W.maxcut24(n_steps=50)
    f = hs.hs_build_factors(job.ham.labels, job.ham.coeffs, job.t / 25, 2, job.budget, "c64")
    a = torch.from_numpy(job.psi0).to("cuda", torch.complex64)
    b = a.clone()
    hs.hs_evolve_ex(f, a, 2, method=REG)
    hs.hs_evolve_ex(f, b, 2, method=hs.HS_METHOD_FUSED)
    torch.cuda.synchronize()
    assert torch.max(torch.abs(a - b)).item() < 1e-6
    n_sw, n_plain, tb, rb = hs.hs_evolve_plan(f, 16, 2, method=REG)
    assert n_plain == 0 and tb == 13 and rb == 1 and n_sw <= 5
    got0 = a[0].cpu().numpy()
    f.close()
    x, z, _ = O.parse_terms(job.ham.labels)
    want0 = O.evolve_direct(x, z, job.ham.coeffs, job.t / 25, 2, job.psi0[0])
    _check(got0, want0, "c64", "maxcut24 state 0")


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_reg_batch_equals_jobs_alone_bitwise_and_oracle(dt):
    """A register-sweep batch (one level launch per sweep index and tile size)
    reproduces every job evolved alone with the same options bit for bit: jobs
    above and below the batch's tile size, one too small for a register tile
    (its own launches), several states per job; small jobs against the oracle."""
    rng = np.random.default_rng(4200)
    tdt = _tdt(dt)
    B = 5 if dt == "c64" else 4
    hams = [(W.tfim_chain(14, 1.0, 0.7), 8), (W.heisenberg_chain(13, rng.uniform(0.5, 1.5, 13)), 8),
            (W.maxcut_3regular(12, 3), 4), (W.tfim_chain(11, 0.9, 1.2), 4), (W.heisenberg_chain(12, rng.uniform(0.5, 1.5, 12)), 4),
            (W.tfim_chain(8, 1.0, 0.5), 4), (_random_ham(rng, 12, 10), 8)]
    jobs = []
    for k, (ham, budget) in enumerate(hams):
        steps = int(rng.integers(2, 7))
        R = 1 + (k % 3 == 0)
        psi0 = np.stack([W.gaussian_state(ham.n_qubits, rng) for _ in range(R)])
        f = hs.hs_build_factors(ham.labels, ham.coeffs, 0.8, steps, budget, dt)
        jobs.append((ham, f, psi0, steps))
    states = [torch.from_numpy(p).to("cuda", tdt) for _, _, p, _ in jobs]
    b = hs.hs_batch_create([(f, s, st) for (_, f, _, st), s in zip(jobs, states)], method=REG, tile_bits=13 if dt == "c64" else 12,
                           low_bits=3 if dt == "c64" else 1)
    assert b.n_separate >= 1  # the 8-qubit job
    hs.hs_batch_launch(b)
    torch.cuda.synchronize()
    for (ham, f, p0, steps), got in zip(jobs, states):
        ref = torch.from_numpy(p0).to("cuda", tdt)
        if ham.n_qubits >= B + 5:
            hs.hs_evolve_ex(f, ref, steps, method=REG, tile_bits=13 if dt == "c64" else 12, low_bits=3 if dt == "c64" else 1,
                            reg_bits=B)
        else:
            hs.hs_evolve(f, ref, steps)
        assert torch.equal(got, ref), (ham.family, ham.n_qubits)
        _check(got.cpu().numpy(), _oracle(ham, 0.8, steps, p0), dt, f"{ham.family} n={ham.n_qubits}")
    # a second launch (graph replay) evolves by the same steps again
    hs.hs_batch_launch(b)
    torch.cuda.synchronize()
    ham, f, p0, steps = jobs[0]
    _check(states[0].cpu().numpy(), _oracle(ham, 1.6, 2 * steps, p0), dt, "relaunch")  # two launches: 2 steps of 0.8 / steps each
    b.close()
    for _, f, _, _ in jobs:
        f.close()


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_evolve_batch_one_call(dt):
    """hs_evolve_batch (one call over job arrays) is bitwise the register-sweep
    batch with default options, and each job agrees with the oracle."""
    rng = np.random.default_rng(4300)
    tdt = _tdt(dt)
    hams = [(W.tfim_chain(13, 1.0, 0.6), 4), (W.heisenberg_chain(12, rng.uniform(0.5, 1.5, 12)), 8),
            (W.maxcut_3regular(14, 7), 4), (W.tfim_chain(9, 0.8, 1.1), 4)]
    jobs = []
    for ham, budget in hams:
        steps = int(rng.integers(2, 6))
        psi0 = np.stack([W.gaussian_state(ham.n_qubits, rng) for _ in range(2)])
        jobs.append((ham, hs.hs_build_factors(ham.labels, ham.coeffs, 0.7, steps, budget, dt), psi0, steps))
    one = [torch.from_numpy(p).to("cuda", tdt) for _, _, p, _ in jobs]
    two = [s.clone() for s in one]
    hs.hs_evolve_batch([(f, s, st) for (_, f, _, st), s in zip(jobs, one)])
    b = hs.hs_batch_create([(f, s, st) for (_, f, _, st), s in zip(jobs, two)], method=REG, use_graph=False)
    hs.hs_batch_launch(b)
    torch.cuda.synchronize()
    b.close()
    for (ham, f, p0, steps), a, c in zip(jobs, one, two):
        assert torch.equal(a, c), (ham.family, ham.n_qubits)
        _check(a.cpu().numpy(), _oracle(ham, 0.7, steps, p0), dt, f"{ham.family} n={ham.n_qubits}")
        f.close()


def test_reg_state_aligned_to_16_bytes_only():
    """A state that is 16-byte but not 32-byte aligned (allowed by the C ABI)
    takes the 16-byte store path and gives the same bits as an aligned one."""
    rng = np.random.default_rng(4400)
    ham = W.maxcut_3regular(14, 11)
    psi0 = np.stack([W.gaussian_state(14, rng) for _ in range(2)])
    f = hs.hs_build_factors(ham.labels, ham.coeffs, 0.9, 4, 4, "c64")
    a = torch.from_numpy(psi0).to("cuda", torch.complex64)
    buf = torch.zeros(2 * (1 << 14) + 2, dtype=torch.complex64, device="cuda")
    b = buf[2:].view(2, 1 << 14)  # 16 bytes past a 256-byte boundary
    assert b.data_ptr() % 32 == 16
    b.copy_(a)
    for psi in (a, b):
        hs.hs_evolve_ex(f, psi, 4, method=REG, tile_bits=13, low_bits=3, reg_bits=5)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    _check(a.cpu().numpy(), _oracle(ham, 0.9, 4, psi0), "c64", "maxcut14")
    f.close()


def test_deferred_diagonals_every_consumer():
    """HS_BUILD_DEFER_DIAGONALS: register sweeps never build the stored
    diagonals; the first call that reads them (staged or plain evolution, a
    graph capture, hs_apply_factor, hs_factor_get, a staged batch) builds them,
    and every result is bitwise that of the eagerly built set."""
    rng = np.random.default_rng(4500)
    ham = W.tfim_chain(13, 1.0, 0.8)
    psi0 = np.stack([W.gaussian_state(13, rng) for _ in range(2)])
    t, steps, budget = 0.9, 4, 8

    def run(defer, **kw):
        f = hs.hs_build_factors(ham.labels, ham.coeffs, t, steps, budget, "c64", defer_diagonals=defer)
        psi = torch.from_numpy(psi0).to("cuda", torch.complex64)
        hs.hs_evolve_ex(f, psi, steps, **kw)
        torch.cuda.synchronize()
        return f, psi

    for kw in (dict(method=REG), dict(method=hs.HS_METHOD_FUSED), dict(method=hs.HS_METHOD_PLAIN),
               dict(method=hs.HS_METHOD_FUSED, use_graph=True)):
        fe, a = run(False, **kw)
        fd, b = run(True, **kw)
        assert torch.equal(a, b), kw
        if kw["method"] == REG:  # the deferred set still builds its diagonals when asked
            for g in range(fe.n_factors):
                assert np.array_equal(fe.factor(g)[3], fd.factor(g)[3])
        fe.close()
        fd.close()
    _check(a.cpu().numpy(), _oracle(ham, t, steps, psi0), "c64", "deferred")
    # hs_apply_factor and a staged batch on fresh deferred sets
    fe = hs.hs_build_factors(ham.labels, ham.coeffs, t, steps, budget, "c64")
    fd = hs.hs_build_factors(ham.labels, ham.coeffs, t, steps, budget, "c64", defer_diagonals=True)
    x = torch.from_numpy(psi0).to("cuda", torch.complex64)
    ye, yd = torch.empty_like(x), torch.empty_like(x)
    hs.hs_apply_factor(fe, 0, x, ye)
    hs.hs_apply_factor(fd, 0, x, yd)
    torch.cuda.synchronize()
    assert torch.equal(ye, yd)
    fd.close()
    fd = hs.hs_build_factors(ham.labels, ham.coeffs, t, steps, budget, "c64", defer_diagonals=True)
    a, b = x.clone(), x.clone()
    be = hs.hs_batch_create([(fe, a, steps)], use_graph=False)
    bd = hs.hs_batch_create([(fd, b, steps)], use_graph=False)
    hs.hs_batch_launch(be)
    hs.hs_batch_launch(bd)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    be.close()
    bd.close()
    fe.close()
    fd.close()
