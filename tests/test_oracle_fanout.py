"""The oracle's process fan-out returns exactly what the oracle returns when called directly."""
import numpy as np

import oracle as O
from oracle import fanout
from paper_2606_16959_gb300 import workloads as W


def test_fanout_equals_direct_calls():
    O.build()
    rng = np.random.default_rng(11)
    ham = W.tfim_chain(8, 1.0, 0.7, periodic=False)
    x, z, _ = O.parse_terms(ham.labels)
    states = [W.gaussian_state(8, rng) for _ in range(3)]
    tasks = [("direct", (x, z, ham.coeffs, 0.9, 5, s)) for s in states]
    tasks.append(("order", (x, z, ham.coeffs, 0.9, 3, states[0], 2)))
    got = fanout.run_many(tasks, workers=2)
    for (res, secs), s in zip(got[:3], states):
        assert np.array_equal(res, O.evolve_direct(x, z, ham.coeffs, 0.9, 5, s)) and secs >= 0
    assert np.array_equal(got[3][0], O.evolve_direct_order(x, z, ham.coeffs, 0.9, 3, states[0], 2))
    assert fanout.host_cores() >= 1
