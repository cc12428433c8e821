"""The bounded-wait error path: a device wait that never completes gives up
after its poll limit, the next sync reports CLC_ETIMEOUT, and the context
keeps working (no fault, no hang)."""
import pytest
import torch

from tests.gpu_util import ctx

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives():
    import paper_1210_3069_gb300 as clc
    c = ctx()
    c.sync()
    c.diag_bounded_wait(1000)
    with pytest.raises(clc.CalclensError) as e:
        c.sync()
    assert e.value.code == clc.ETIMEOUT
    # the error word was cleared and the context still computes
    c.sync()
    m = torch.ones(12 * 16 * 16, dtype=torch.float64, device="cuda")
    alm = c.sht_analysis(m, 16, 32)
    c.sync()
    assert abs(float(alm[0].real) - (4 * 3.141592653589793) ** 0.5) < 1e-12
    with pytest.raises(clc.CalclensError):
        c.diag_bounded_wait(0)
