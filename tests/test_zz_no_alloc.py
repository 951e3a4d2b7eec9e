"""The allocation-free inner-product entry point against the allocating one.

hs_inner_batch_noalloc is for callers that cannot allocate device memory (a
serving loop that keeps all of it reserved for resident states and factors, or
an application whose device memory belongs to its own allocator).  It keeps its
scratch in a static device array instead.  This file is collected last so that
a run stopping at the first failure has already run every other test; it also
passes alone in a fresh process (its first call performs the per-device set-up).
"""
import numpy as np
import pytest

from paper_2606_16959_gb300 import hs, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_16959_gb300 import _build
    _build.build()
    hs.lib()


def _states(rng, n, R, tdt):
    return torch.from_numpy(np.stack([W.gaussian_state(n, rng) * rng.uniform(0.5, 2.0) for _ in range(R)])).to(
        device="cuda", dtype=tdt)


@pytest.mark.parametrize("tdt", [torch.complex64, torch.complex128])
def test_noalloc_matches_allocating_entry_point(tdt):
    rng = np.random.default_rng(4242)
    for call, (n, R) in enumerate([(17, 5), (9, 8)]):  # two calls in a row, different sizes and data
        a = _states(rng, n, R, tdt)
        b = a + 0.1 * _states(rng, n, R, tdt)
        out = torch.full((R, 4), float("nan"), dtype=torch.float64, device="cuda")
        hs.hs_inner_batch_noalloc(a, b, out)
        got = out.cpu().numpy()
        for i in range(R):
            ref = torch.zeros(4, dtype=torch.float64, device="cuda")
            hs.hs_inner_device(a[i], b[i], ref)
            np.testing.assert_allclose(got[i], ref.cpu().numpy(), rtol=1e-12, atol=1e-14)


def test_noalloc_rejects_oversize():
    a = torch.zeros((9, 1 << 18), dtype=torch.complex64, device="cuda")
    out = torch.zeros((9, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(hs.HSError) as e:
        hs.hs_inner_batch_noalloc(a, a, out)
    assert e.value.code == hs.HS_EINVAL and "static scratch" in str(e.value)
