"""The split-precision tcgen05 contraction against an FP64 CPU product of
the same FP16 operands."""
import pytest
import torch

from tests.gpu_util import ctx

pytestmark = pytest.mark.gpu


def split(x):
    hi = x.half()
    lo = (x - hi.float()).half()
    return hi, lo


@pytest.mark.parametrize("batch,M,N,K", [(1, 128, 16, 64), (3, 300, 48, 256), (2, 256, 256, 1024), (1, 77, 112, 128)])
def test_gemm_f16x3_matches_fp64_product(batch, M, N, K):
    c = ctx()
    g = torch.Generator().manual_seed(M + N + K)
    a = torch.randn(batch, M, K, generator=g)
    b = torch.randn(batch, N, K, generator=g)
    ah, al = split(a)
    bh, bl = split(b)
    d = c.gemm_f16x3(ah.cuda(), al.cuda(), bh.cuda(), bl.cuda())
    c.sync()
    A = [t.double() for t in (ah, al)]
    B = [t.double() for t in (bh, bl)]
    ref = A[0] @ B[0].transpose(1, 2) + A[0] @ B[1].transpose(1, 2) + A[1] @ B[0].transpose(1, 2)
    err = (d.cpu().double() - ref).abs().max() / ref.abs().max()
    assert err < 1e-5, float(err)
    # and the split recovers the FP32 product of the unsplit operands closely
    full = a.double() @ b.double().transpose(1, 2)
    assert float((d.cpu().double() - full).abs().max() / full.abs().max()) < 1e-5
