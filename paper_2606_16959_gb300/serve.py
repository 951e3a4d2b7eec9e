"""Continuous-batching request loop for evolution jobs on one GPU.

Requests (a Hamiltonian, a time, a step count, an initial state) arrive over
time.  The loop admits waiting requests while in-flight slots and an HBM budget
allow (each request is charged its factor bytes from the structural dry run,
hs_plan_factors, plus its state bytes), builds their factors and launches them
as one batch (hs_batch_*) on the next of several CUDA streams, so that groups
admitted while earlier groups still run overlap on the device.  Factors and
states stay on the device; memory is returned in stream order when a group
finishes.  Completion times come from CUDA events measured against a start
event, so latency = GPU completion time - arrival time.

Factor sets are built with their stored diagonals deferred
(HS_BUILD_DEFER_DIAGONALS): the register-sweep batches generate every factor
from its terms, so the diagonals are only built if a batch's own options need
them.  A request's device bytes come from the structural dry run of its terms,
cached per Hamiltonian structure (labels and budget), so admission does no
planning work for a structure it has seen.  A build that fails for lack of
device memory (HS_ENOMEM) puts its group back at the head of the queue and
admission pauses until an in-flight group retires; a request that fails three
times is reported failed and the stream goes on.  cancel() withdraws a request:
a waiting one never runs, an in-flight one finishes on the device and its
result is dropped.  The `fault` hook (called as fault(stage, request) before
each request's build) lets tests inject such failures on the host.

All computation runs in libhs; this module only schedules.  shard_jobs splits
a request stream across ranks (independent jobs, no data exchange).
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

from . import hs


@dataclass
class Request:
    labels: List[str]
    coeffs: np.ndarray
    n_qubits: int
    t: float
    n_steps: int
    budget: int
    arrival: float = 0.0                 # seconds after the start of the run
    psi0: Optional[np.ndarray] = None    # initial state (host); None: seeded Gaussian made on the device
    seed: int = 0
    rid: int = -1
    # filled by the server
    admitted: Optional[float] = None
    done: Optional[float] = None
    updates: int = 0
    norm2: Optional[float] = None
    result: Optional[np.ndarray] = None
    attempts: int = 0
    cancelled: bool = False
    error: Optional[str] = None


def requests_from_jobs(jobs) -> List[Request]:
    """Requests from workloads.Job objects (arrival times included)."""
    out = []
    for k, j in enumerate(jobs):
        out.append(Request(list(j.ham.labels), np.asarray(j.ham.coeffs), j.ham.n_qubits, j.t, j.n_steps, j.budget,
                           arrival=j.arrival, psi0=j.psi0, seed=j.seed if j.psi0 is None else k, rid=k))
    return out


def shard_jobs(items: Sequence, rank: int, world: int) -> list:
    """Round-robin share of independent jobs for one rank (no collective needed)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    return [x for k, x in enumerate(items) if k % world == rank]


@dataclass
class _Group:
    reqs: list
    factors: list
    states: list
    batch: object
    stream: object
    event: object
    bytes: int
    out: object = None
    host: list = field(default_factory=list)


class Server:
    def __init__(self, dtype: str = "c64", hbm_bytes: Optional[int] = None, max_inflight: int = 64,
                 max_group: int = 32, n_streams: int = 4, tile_bits: int = 0, keep_results: bool = False,
                 batch_opts: Optional[dict] = None):
        import torch
        self.torch = torch
        self.dtype = dtype
        self.tdt = torch.complex64 if dtype == "c64" else torch.complex128
        self.esize = 8 if dtype == "c64" else 16
        free, _ = torch.cuda.mem_get_info()
        self.budget = int(hbm_bytes) if hbm_bytes else int(free * 0.8)
        self.max_inflight = max_inflight
        self.max_group = max_group
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        # options of every batch (hs_batch_create keywords, e.g. from
        # hs.hs_batch_autotune on a representative group)
        self.batch_opts = dict(batch_opts or {})
        if tile_bits:
            self.batch_opts["tile_bits"] = tile_bits
        self.keep_results = keep_results
        self.used = 0
        self.peak_used = 0
        self._next_stream = 0
        self._plan_bytes = collections.OrderedDict()  # (labels, budget) -> factor bytes
        self._cancel = set()
        self._paused = False  # admission paused after an allocation failure
        self.fault = None     # fault(stage, request): host-side fault injection (tests)
        self.n_alloc_failures = 0

    def cancel(self, rid: int) -> None:
        """Withdraw request rid: if it is still waiting it never runs; if it is in
        flight its result is dropped when its group finishes."""
        self._cancel.add(rid)

    def _bytes(self, r: Request) -> int:
        """Device bytes a request holds while in flight: its factor values (structural
        dry run, cached per structure), its state, and a margin for tables."""
        key = (tuple(r.labels), r.budget)
        vbytes = self._plan_bytes.get(key)
        if vbytes is None:
            x, z, n = hs.hs_parse_terms(r.labels)
            _, vbytes = hs.hs_plan_factors(x, z, n, r.budget, self.dtype)
            self._plan_bytes[key] = vbytes
            if len(self._plan_bytes) > 4096:
                self._plan_bytes.popitem(last=False)
        else:
            self._plan_bytes.move_to_end(key)
        return int(vbytes) + (1 << r.n_qubits) * self.esize + (1 << 20)

    def _launch(self, group: List[Request], t0_event):
        """Build and launch one group; None if a build ran out of device memory
        (everything built so far is released in stream order)."""
        torch = self.torch
        s = self.streams[self._next_stream % len(self.streams)]
        self._next_stream += 1
        states, facs = [], []
        try:
            return self._launch_on(group, s, states, facs)
        except hs.HSError as e:
            if e.code != hs.HS_ENOMEM:
                raise
            for f in facs:
                f.close(stream=s)
            self.n_alloc_failures += 1
            return None

    def _launch_on(self, group, s, states, facs):
        torch = self.torch
        with torch.cuda.stream(s):
            for r in group:
                r.attempts += 1
                if self.fault is not None:
                    self.fault("build", r)
                if r.psi0 is not None:
                    st = torch.from_numpy(np.ascontiguousarray(r.psi0)).to("cuda", self.tdt, non_blocking=True)
                else:
                    g = torch.Generator(device="cuda")
                    g.manual_seed(int(r.seed))
                    re = torch.randn(1 << r.n_qubits, generator=g, device="cuda", dtype=torch.float32)
                    im = torch.randn(1 << r.n_qubits, generator=g, device="cuda", dtype=torch.float32)
                    st = torch.complex(re, im).to(self.tdt)
                    st /= torch.linalg.vector_norm(st)
                states.append(st)
                # stored diagonals deferred: the register-sweep batches generate the
                # factors from their terms (a staged batch would build them first)
                facs.append(hs.hs_build_factors(r.labels, r.coeffs, r.t, r.n_steps, r.budget, self.dtype, stream=s,
                                                defer_diagonals=True))
                r.updates = r.n_steps * facs[-1].n_factors * (1 << r.n_qubits)
            b = hs.hs_batch_create([(f, st, r.n_steps) for f, st, r in zip(facs, states, group)], use_graph=False,
                                   **self.batch_opts)
            hs.hs_batch_launch(b, stream=s)
            out = torch.zeros(len(group), 4, dtype=torch.float64, device="cuda")
            for k, st in enumerate(states):
                hs.hs_inner_device(st, st, out[k], stream=s)
            host = []
            if self.keep_results:
                host = [st.to("cpu", non_blocking=True) for st in states]
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(s)
        return _Group(group, facs, states, b, s, ev, 0, out, host)

    def _runnable(self, r: Request) -> bool:
        if r.rid in self._cancel:
            r.cancelled = True
            return False
        return True

    def run(self, requests: Sequence[Request], realtime: bool = True, poll_s: float = 5e-5):
        """Serve the requests (sorted by arrival).  realtime: wait for arrival times;
        otherwise every request is available at once.  Returns a stats dict."""
        torch = self.torch
        l0 = hs.hs_kernel_launches()
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting: collections.deque = collections.deque()
        inflight: List[_Group] = []
        n_inflight = 0
        t0_event = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0_event.record()
        t0 = time.perf_counter()
        while pending or waiting or inflight:
            now = time.perf_counter() - t0
            while pending and (not realtime or pending[0].arrival <= now):
                r = pending.popleft()
                if self._runnable(r):
                    waiting.append(r)
            # retire finished groups
            keep = []
            for g in inflight:
                if g.event.query():
                    t_done = t0_event.elapsed_time(g.event) / 1000.0
                    norms = g.out[:, 2].cpu().numpy()
                    for k, r in enumerate(g.reqs):
                        if r.rid in self._cancel:
                            r.cancelled = True
                            continue
                        r.done = t_done
                        r.norm2 = float(norms[k])
                        if self.keep_results:
                            r.result = g.host[k].numpy()
                    g.batch.close(stream=g.stream)
                    for f in g.factors:
                        f.close(stream=g.stream)
                    self.used -= g.bytes
                    n_inflight -= len(g.reqs)
                    self._paused = False
                else:
                    keep.append(g)
            inflight = keep
            # admit
            group, gbytes = [], 0
            while (waiting and not self._paused and n_inflight + len(group) < self.max_inflight
                   and len(group) < self.max_group):
                r = waiting[0]
                if not self._runnable(r):
                    waiting.popleft()
                    continue
                need = self._bytes(r)
                if self.used + gbytes + need > self.budget:
                    if not inflight and not group and self.used == 0:
                        raise RuntimeError(f"request {r.rid} needs {need} bytes, above the HBM budget")
                    break
                waiting.popleft()
                r.admitted = time.perf_counter() - t0
                group.append(r)
                gbytes += need
            if group:
                g = self._launch(group, t0_event)
                if g is None:
                    # out of device memory: requests that failed three times are
                    # reported failed, the rest wait (at the head of the queue)
                    # until an in-flight group returns its memory
                    for r in reversed(group):
                        if r.attempts >= 3:
                            r.error = "device memory exhausted"
                            r.done = time.perf_counter() - t0
                        else:
                            waiting.appendleft(r)
                    self._paused = bool(inflight)
                    continue
                g.bytes = gbytes
                self.used += gbytes
                self.peak_used = max(self.peak_used, self.used)
                n_inflight += len(group)
                inflight.append(g)
                continue
            # nothing to admit: wait a little (for an arrival or a completion)
            wait = poll_s
            if pending and not waiting and not inflight:
                wait = min(1e-3, max(0.0, pending[0].arrival - (time.perf_counter() - t0)))
            time.sleep(wait)
        torch.cuda.synchronize()
        served = [r for r in requests if not r.cancelled and r.error is None]
        lat = np.array([r.done - r.arrival for r in served]) if served else np.zeros(1)
        t_first = min(r.arrival for r in requests)
        t_last = max((r.done for r in served), default=t_first)
        updates = sum(r.updates for r in served)
        # Queue growth: requests still in the system when the last one arrived,
        # the drain after it, and the median latency of the second and the last
        # quarter of the requests by arrival (equal when the queue is bounded).
        t_arr = max(r.arrival for r in requests)
        by_arr = sorted(served, key=lambda r: r.arrival)
        q = max(1, len(by_arr) // 4)

        def _p50(rs):
            return float(np.median([r.done - r.arrival for r in rs]) * 1e3) if rs else 0.0
        growth = dict(backlog_at_last_arrival=sum(r.done > t_arr for r in served), drain_s=max(0.0, t_last - t_arr),
                      p50_q2_ms=_p50(by_arr[q:2 * q]), p50_q4_ms=_p50(by_arr[-q:]))
        return dict(n=len(served), n_cancelled=sum(r.cancelled for r in requests),
                    n_failed=sum(r.error is not None for r in requests),
                    p50_ms=float(np.percentile(lat, 50) * 1e3), p99_ms=float(np.percentile(lat, 99) * 1e3),
                    mean_ms=float(lat.mean() * 1e3), makespan_s=t_last - t_first, updates=updates,
                    throughput=updates / max(t_last - t_first, 1e-9), peak_bytes=self.peak_used,
                    alloc_failures=self.n_alloc_failures, launches=hs.hs_kernel_launches() - l0, **growth)
