"""GPU parity of the second- and fourth-order product formulas (Strang,
Suzuki) against the oracle's term-by-term evolution; the step sequence of the
stored factors; value tables and batches on higher-order factor sets."""
import numpy as np
import pytest

import oracle as O
from paper_2606_16959_gb300 import hs, workloads as W

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


def _hams(rng):
    labels = ["".join(rng.choice(list("IXYZ"), p=[0.6, 0.14, 0.13, 0.13], size=10)) for _ in range(8)]
    return [("heis12", W.heisenberg_chain(12, rng.uniform(0.5, 1.5, 12), periodic=True), 8),
            ("tfim11", W.tfim_chain(11, 1.0, 0.7, periodic=False), 4),
            ("rand10", W.Hamiltonian("random", 10, labels, rng.uniform(-1, 1, 8)), 16)]


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_order_matches_oracle(order, dt):
    rng = np.random.default_rng(500 + order)
    tdt = torch.complex128 if dt == "c128" else torch.complex64
    for name, ham, budget in _hams(rng):
        x, z, n = O.parse_terms(ham.labels)
        psi = np.stack([W.gaussian_state(n, rng) for _ in range(2)])
        want = O.evolve_direct_order(x, z, ham.coeffs, 0.8, 5, psi, order)
        f = hs.hs_build_factors(ham.labels, ham.coeffs, 0.8, 5, budget, dt, order=order)
        assert f.order == order
        for kw in (dict(), dict(method=hs.HS_METHOD_PLAIN),
                   dict(method=hs.HS_METHOD_FUSED, tile_bits=8, rhs_block=1, low_bits=1)):
            pd = torch.from_numpy(psi).to("cuda", tdt)
            hs.hs_evolve_ex(f, pd, 5, **kw)
            got = pd.cpu().numpy().astype(np.complex128)
            if dt == "c128":
                assert np.max(np.abs(got - want)) <= 1e-12, (name, kw)
            else:
                assert np.max(np.abs(got - want)) <= 1e-5, (name, kw)
                assert max(1 - O.fidelity(got[k], want[k]) for k in range(2)) <= 1e-6
        f.close()


def test_step_sequence_layout():
    ham = W.heisenberg_chain(10, np.linspace(0.5, 1.5, 10), periodic=True)
    f1 = hs.hs_build_factors(ham.labels, ham.coeffs, 1.0, 3, 8, "c128", order=1)
    G = f1.n_factors
    assert f1.sequence == list(range(G))
    f2 = hs.hs_build_factors(ham.labels, ham.coeffs, 1.0, 3, 8, "c128", order=2)
    assert f2.n_factors == 2 * G
    assert f2.sequence == list(range(G)) + list(range(2 * G - 1, G - 1, -1))
    f4 = hs.hs_build_factors(ham.labels, ham.coeffs, 1.0, 3, 8, "c128", order=4)
    assert f4.n_factors == 4 * G and len(f4.sequence) == 10 * G
    # the reversed copies share the forward factors' structure (same offsets, same terms)
    for g in range(G):
        a, b = f2.factor(g, values=False), f2.factor(G + g, values=False)
        assert a[0] == b[0] and a[1] == b[1] and np.array_equal(a[2], b[2])
    for f in (f1, f2, f4):
        f.close()


def test_order2_value_tables_and_batch_bitwise():
    rng = np.random.default_rng(61)
    jobs, facs, s1, s2, s3 = [], [], [], [], []
    for k in range(5):
        n = int(rng.integers(11, 14))
        ham = W.heisenberg_chain(n, rng.uniform(0.5, 1.5, n), periodic=True) if k % 2 else \
            W.tfim_chain(n, 1.0, float(rng.uniform(0.2, 1.5)))
        f = hs.hs_build_factors(ham.labels, ham.coeffs, 1.0, 7, 8, "c64", order=2)
        psi = torch.from_numpy(W.gaussian_state(n, rng)).to("cuda", torch.complex64)
        facs.append(f)
        s1.append(psi.clone())
        s2.append(psi.clone())
        s3.append(psi.clone())
        jobs.append(ham)
    for f, a, b in zip(facs, s1, s2):
        opts = dict(method=hs.HS_METHOD_FUSED, tile_bits=9, rhs_block=1, low_bits=2)
        hs.hs_evolve_ex(f, a, 7, **opts)
        hs.hs_evolve_ex(f, b, 7, no_tables=True, **opts)
    b = hs.hs_batch_create([(f, s, 7) for f, s in zip(facs, s3)], tile_bits=9, low_bits=2)
    assert b.n_updates == sum(7 * len(f.sequence) * (1 << f.n_qubits) for f in facs)
    hs.hs_batch_launch(b)
    torch.cuda.synchronize()
    for a, bb, c in zip(s1, s2, s3):
        assert torch.equal(a, bb)
        assert torch.equal(a, c)
    b.close()
