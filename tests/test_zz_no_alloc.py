"""The allocation-free SHT analysis (clc_sht_analysis_noalloc) against the
allocating entry point clc_sht_analysis.

Callers that cannot allocate device memory - work recorded into a CUDA
graph, code under a framework's caching allocator, fixed-footprint services -
use the noalloc variant; it must give the same coefficients.  Kept in its own
file, collected last, so that a run stopping at the first failure has run
every other test already."""
import ctypes

import pytest
import torch

from tests.gpu_util import ctx, rel_l2

pytestmark = pytest.mark.gpu


def _noalloc():
    import paper_1210_3069_gb300 as clc
    f = clc.lib().clc_sht_analysis_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    return f


def test_noalloc_analysis_matches_allocating_entry_point():
    c = ctx()
    f = _noalloc()
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row, the second smaller than the first, so leftovers of
    # the first call in the shared scratch array would show
    for nside, lmax, seed in [(128, 256, 1), (16, 40, 2)]:
        g = torch.Generator().manual_seed(seed)
        m = torch.randn(12 * nside * nside, dtype=torch.float64, generator=g).cuda()
        ref = c.sht_analysis(m, nside, lmax)
        out = torch.full_like(ref, float("nan"))
        assert f(ctypes.c_void_p(m.data_ptr()), nside, lmax, ctypes.c_void_p(out.data_ptr()),
                 ctypes.c_void_p(stream)) == 0
        torch.cuda.synchronize()
        assert rel_l2(out, ref) < 1e-10, (nside, lmax)


def test_noalloc_rejects_sizes_beyond_its_maximum():
    ctx()
    f = _noalloc()
    m = torch.zeros(12 * 256 * 256, dtype=torch.float64, device="cuda")
    out = torch.zeros(300 * 300, dtype=torch.complex128, device="cuda")
    p, q = ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(out.data_ptr())
    assert f(p, 256, 100, q, None) == 1        # nside above 128
    assert f(p, 64, 257, q, None) == 1         # lmax above 256
    assert f(p, 8, 33, q, None) == 1           # lmax above 4 nside
    assert f(p, 48, 10, q, None) == 1          # nside not a power of two
    assert f(None, 8, 10, q, None) == 1


@pytest.mark.parametrize("nside,lmax", [(1, 2), (1, 4), (2, 5), (2, 8), (4, 11), (4, 16), (8, 23), (8, 32)])
def test_noalloc_analysis_at_the_smallest_nsides(nside, lmax):
    """A single ring-group of pixels per face (nside 1) up to nside 8, at
    lmax 3 nside - 1 and at the entry point's limit 4 nside: the few-ring
    grids where the polar and equatorial ring lengths differ most."""
    c = ctx()
    f = _noalloc()
    g = torch.Generator().manual_seed(100 + nside)
    m = torch.randn(12 * nside * nside, dtype=torch.float64, generator=g).cuda()
    ref = c.sht_analysis(m, nside, lmax)
    out = torch.full_like(ref, float("nan"))
    stream = torch.cuda.current_stream().cuda_stream
    assert f(ctypes.c_void_p(m.data_ptr()), nside, lmax, ctypes.c_void_p(out.data_ptr()),
             ctypes.c_void_p(stream)) == 0
    torch.cuda.synchronize()
    assert rel_l2(out, ref) < 1e-10, (nside, lmax)
