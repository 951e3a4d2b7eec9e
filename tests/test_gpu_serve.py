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
