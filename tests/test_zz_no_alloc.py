"""The allocation-free inner-product entry point against the allocating one and the oracle.

hs_inner_batch_noalloc is for callers that cannot allocate device memory (a
serving loop that keeps all of it reserved for resident states and factors, or
an application whose device memory belongs to its own allocator).  It keeps its
scratch in a static device array instead.  This file is collected last so that
a run stopping at the first failure has already run every other test; it also
passes alone in a fresh process (its first call performs the per-device set-up).
"""
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
        l0 = hs.hs_kernel_launches()
        hs.hs_inner_batch_noalloc(a, b, out)
        assert hs.hs_kernel_launches() - l0 == 2  # both of its kernels are counted
        got = out.cpu().numpy()
        ah, bh = a.cpu().numpy(), b.cpu().numpy()
        for i in range(R):
            ref = torch.zeros(4, dtype=torch.float64, device="cuda")
            hs.hs_inner_device(a[i], b[i], ref)
            np.testing.assert_allclose(got[i], ref.cpu().numpy(), rtol=1e-12, atol=1e-14)
            # and against the FP64 oracle's pairwise sums of the same (stored) amplitudes
            ip = O.inner(ah[i], bh[i])
            np.testing.assert_allclose(got[i], [ip.real, ip.imag, O.norm2(ah[i]), O.norm2(bh[i])],
                                       rtol=1e-12, atol=1e-13)


def test_noalloc_rejects_oversize():
    a = torch.zeros((9, 1 << 18), dtype=torch.complex64, device="cuda")
    out = torch.zeros((9, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(hs.HSError) as e:
        hs.hs_inner_batch_noalloc(a, a, out)
    assert e.value.code == hs.HS_EINVAL and "static scratch" in str(e.value)


def test_noalloc_rejects_wrong_output_dtype():
    """A float32 or complex64 output of 4R elements is too small for 4R doubles."""
    a = torch.zeros((3, 1 << 10), dtype=torch.complex64, device="cuda")
    for bad in (torch.zeros((3, 4), dtype=torch.float32, device="cuda"),
                torch.zeros((3, 4), dtype=torch.complex64, device="cuda"),
                torch.zeros((3, 4), dtype=torch.float64)):
        with pytest.raises(ValueError):
            hs.hs_inner_batch_noalloc(a, a, bad)
        with pytest.raises(ValueError):
            hs.hs_inner_device(a[0], a[0], bad)
