"""Process fan-out of the oracle over independent inputs -- TEST INFRASTRUCTURE ONLY.

Runs the unchanged single-threaded oracle (``oracle.evolve_direct`` and the
other evolution functions) on several independent inputs at once -- states of
a multi-state job, or whole jobs of a batch -- one input per worker process.
Nothing of the method's arithmetic lives here: each worker calls the oracle as
it stands, so a result equals the one a single call would give.

Workers are started with the ``spawn`` method: a process forked after the
parent has initialised CUDA can hang, and spawn never copies that state.  Only
``tests/`` and ``bench.py``'s CPU-baseline leg use this module.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import time
from concurrent.futures import ProcessPoolExecutor
from typing import List, Optional, Sequence, Tuple


def _run(task: Tuple[str, tuple]):
    """Worker: one oracle evolution.  task = (kind, args); returns (result, seconds)."""
    import oracle
    kind, args = task
    t0 = time.perf_counter()
    if kind == "direct":          # (x, z, coeffs, t, n_steps, psi)
        out = oracle.evolve_direct(*args)
    elif kind == "order":         # (x, z, coeffs, t, n_steps, psi, order)
        out = oracle.evolve_direct_order(*args)
    elif kind == "td":            # (x, z, a, b, drive, t, psi, order)
        out = oracle.evolve_direct_td(*args)
    else:
        raise ValueError(f"unknown task kind {kind!r}")
    return out, time.perf_counter() - t0


def host_cores() -> int:
    """Cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def run_many(tasks: Sequence[Tuple[str, tuple]], workers: Optional[int] = None) -> List[tuple]:
    """Run the tasks on up to `workers` spawned processes (default: one per
    task, at most the host's cores); returns [(result, seconds)] in task order."""
    if not tasks:
        return []
    n = min(len(tasks), workers or host_cores())
    if n <= 1:
        return [_run(t) for t in tasks]
    with ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_run, tasks))
