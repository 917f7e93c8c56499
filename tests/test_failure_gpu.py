"""Failure detection on the GPU without a fault: a bounded wait runs out and reports a status."""
import pytest
import torch

from _gpu import hsmm, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


def test_wait_timeout_reports_status():
    h = hsmm()
    st = h.selftest_timeout(2_000_000)          # 2 ms limit on an mbarrier nothing arrives on
    assert st == h.hsmm.TIMEOUT
    # the context stays usable and the status word was cleared
    assert h.sync_status() == h.hsmm.SUCCESS
    x = torch.ones(4, device="cuda")
    assert float((x * 2).sum()) == 8.0
