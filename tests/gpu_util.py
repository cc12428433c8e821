"""Helpers of the GPU parity tests: one library context per session."""
import pytest
import torch

_CTX = None


def ctx():
    global _CTX
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    if _CTX is None:
        import paper_1210_3069_gb300 as clc
        clc.build()
        _CTX = clc.Context(0)
    return _CTX


def rel_l2(a, b):
    a = a.detach().cpu()
    b = b.detach().cpu()
    if a.is_complex() or b.is_complex():
        a = torch.view_as_real(a.to(torch.complex128))
        b = torch.view_as_real(b.to(torch.complex128))
    a = a.double()
    b = b.double()
    den = float(torch.linalg.vector_norm(b))
    return float(torch.linalg.vector_norm(a - b)) / (den if den > 0 else 1.0)
