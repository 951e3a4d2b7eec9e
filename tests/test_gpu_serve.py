"""Serving: continuous batching with HBM admission.

Each request's result must be the same when it is served alone and when it is
served in a mix with others (the same per-job schedule and arithmetic, so the
same bits), requests are admitted only while the HBM budget allows, and a small
real-time Poisson stream completes with latency statistics.
"""
import numpy as np
import pytest

import oracle as O
from paper_2606_16959_gb300 import hs, serve, workloads as W

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


def _requests(seed, count, n_lo, n_hi, rate=None):
    rng = np.random.default_rng(seed)
    out, t = [], 0.0
    for k in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        fam = k % 4
        if fam == 0:
            ham = W.tfim_chain(n, 1.0, float(rng.uniform(0, 2)))
        elif fam == 1:
            ham = W.heisenberg_chain(n, rng.uniform(0.5, 1.5, n))
        elif fam == 2:
            n += n % 2
            ham = W.maxcut_3regular(n, int(rng.integers(1 << 30)))
        else:
            ham = W.tsp_onehot(3, int(rng.integers(1 << 30)))  # 9 qubits
        if rate:
            t += float(rng.exponential(1.0 / rate))
        psi0 = W.gaussian_state(ham.n_qubits, rng)
        out.append(serve.Request(list(ham.labels), ham.coeffs, ham.n_qubits, float(rng.uniform(0.5, 2.0)),
                                 int(rng.integers(2, 12)), W.FAMILY_BUDGET[ham.family], arrival=t, psi0=psi0, rid=k))
    return out


def test_results_same_alone_and_in_mix():
    mix = _requests(5, 12, 9, 13)
    srv = serve.Server(keep_results=True, max_group=3, n_streams=3)
    stats = srv.run(mix, realtime=False)
    assert stats["n"] == 12
    for r in mix:
        alone = serve.Request(r.labels, r.coeffs, r.n_qubits, r.t, r.n_steps, r.budget, psi0=r.psi0, rid=r.rid)
        serve.Server(keep_results=True).run([alone], realtime=False)
        assert np.array_equal(alone.result, r.result), r.rid
    # every served result against the FP64 oracle: max-abs and infidelity
    for r in mix:
        x, z, _ = O.parse_terms(r.labels)
        want = O.evolve_direct(x, z, r.coeffs, r.t, r.n_steps, r.psi0)
        got = np.asarray(r.result, np.complex128).ravel()
        assert np.max(np.abs(got - want)) <= 1e-5, r.rid
        fid = abs(np.vdot(got, want)) ** 2 / (np.vdot(got, got).real * np.vdot(want, want).real)
        assert 1.0 - fid <= 1e-6, r.rid


def test_admission_respects_hbm_budget():
    reqs = _requests(6, 10, 14, 16)
    srv = serve.Server(keep_results=False)
    per = max(srv._bytes(r) for r in reqs)
    srv.budget = int(2.5 * per)  # room for two requests at a time
    stats = srv.run(reqs, realtime=False)
    assert stats["n"] == 10
    assert srv.peak_used <= srv.budget
    assert all(r.done is not None and abs(r.norm2 - 1.0) < 1e-4 for r in reqs)
    small = serve.Server()
    small.budget = per // 4
    with pytest.raises(RuntimeError):
        small.run(reqs[:1], realtime=False)


def test_poisson_stream_latency():
    reqs = _requests(7, 40, 10, 14, rate=400.0)
    stats = serve.Server().run(reqs, realtime=True)
    assert stats["n"] == 40 and 0 < stats["p50_ms"] <= stats["p99_ms"]
    assert stats["throughput"] > 0
    assert all(abs(r.norm2 - 1.0) < 1e-4 for r in reqs)


def _alone(r):
    a = serve.Request(r.labels, r.coeffs, r.n_qubits, r.t, r.n_steps, r.budget, psi0=r.psi0, rid=r.rid)
    serve.Server(keep_results=True).run([a], realtime=False)
    return a.result


def test_allocation_failure_is_retried_and_the_rest_unchanged():
    """A build that runs out of device memory (injected on the host as HS_ENOMEM
    on request 3's first attempt) puts its group back in the queue; every
    request completes with the bits it has when served alone."""
    mix = _requests(11, 9, 9, 12)
    srv = serve.Server(keep_results=True, max_group=2, n_streams=2)

    def fault(stage, r):
        if stage == "build" and r.rid == 3 and r.attempts == 1:
            raise hs.HSError(hs.HS_ENOMEM, "injected allocation failure")
    srv.fault = fault
    stats = srv.run(mix, realtime=False)
    assert stats["n"] == 9 and stats["alloc_failures"] == 1 and stats["n_failed"] == 0
    assert mix[3].attempts == 2
    for r in mix:
        assert np.array_equal(r.result, _alone(r)), r.rid


def test_persistent_allocation_failure_fails_one_request_only():
    mix = _requests(12, 6, 9, 11)
    srv = serve.Server(keep_results=True, max_group=1)
    srv.fault = lambda stage, r: (_ for _ in ()).throw(hs.HSError(hs.HS_ENOMEM, "injected")) if r.rid == 2 else None
    stats = srv.run(mix, realtime=False)
    assert stats["n"] == 5 and stats["n_failed"] == 1 and mix[2].error and mix[2].result is None
    for r in mix:
        if r.rid != 2:
            assert np.array_equal(r.result, _alone(r)), r.rid


def test_cancelled_request_never_runs_and_the_rest_unchanged():
    mix = _requests(13, 8, 9, 12)
    srv = serve.Server(keep_results=True, max_group=2)
    srv.cancel(5)
    stats = srv.run(mix, realtime=False)
    assert stats["n"] == 7 and stats["n_cancelled"] == 1
    assert mix[5].cancelled and mix[5].result is None and mix[5].updates == 0
    for r in mix:
        if r.rid != 5:
            assert np.array_equal(r.result, _alone(r)), r.rid


def test_slow_job_does_not_hold_back_the_others():
    """A 22-qubit, 100-step request admitted first runs on its own stream; the
    small requests admitted after it finish before it and keep their bits."""
    rng = np.random.default_rng(14)
    big_h = W.heisenberg_chain(22, rng.uniform(0.5, 1.5, 22))
    big = serve.Request(list(big_h.labels), big_h.coeffs, 22, 1.0, 100, 8, psi0=W.gaussian_state(22, rng), rid=100)
    small = _requests(15, 6, 9, 11)
    srv = serve.Server(keep_results=True, max_group=1, n_streams=8)  # the big request's stream takes no other
    stats = srv.run([big] + small, realtime=False)
    assert stats["n"] == 7
    assert max(r.done for r in small) < big.done
    for r in small:
        assert np.array_equal(r.result, _alone(r)), r.rid
    assert abs(big.norm2 - 1.0) < 1e-4
