"""Failure paths exercised without faulting the GPU.

- A device-memory cap that create cannot meet returns SYNIM_ERR_OOM, leaves
  nothing allocated that a later context could trip over, and a context with
  a sufficient cap computes the same IMs as one without.
- The bounded device wait (the mbarrier wait helper of the tensor-core
  kernels) gives up on a barrier that nothing arrives at: the call returns
  SYNIM_ERR_TIMEOUT after a short limit and the context keeps working.
"""
import pytest
import torch

from paper_2606_07759_b300 import abi
from paper_2606_07759_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _ctx(**kw):
    from paper_2606_07759_b300.synim import SynIM
    wl = W.scao_small()
    return wl, SynIM(wl.dms, wl.wfss, **kw)


def test_create_beyond_the_memory_cap_returns_oom():
    with pytest.raises(abi.SynimError) as ex:
        _ctx(device_mem_cap=4096)
    assert ex.value.status == 3   # SYNIM_ERR_OOM
    # a capped create that failed left the device usable for the next one
    wl, s = _ctx()
    out = s.compute(wl.misregs)
    s.check()
    assert torch.isfinite(out[0]).all()
    s.close()


def test_a_sufficient_cap_changes_nothing():
    wl, a = _ctx()
    _, b = _ctx(device_mem_cap=1 << 31)
    ia, ib = a.compute(wl.misregs), b.compute(wl.misregs)
    a.check()
    b.check()
    assert torch.equal(ia[0], ib[0])
    a.close()
    b.close()


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    wl, s = _ctx()
    ref = s.compute(wl.misregs)[0].clone()
    s.check()
    # about half a millisecond at 2 GHz: nothing arrives, the wait returns
    assert s.wait_selftest(1 << 20) == 5          # SYNIM_ERR_TIMEOUT
    assert "timed out" in abi.last_error(s._ctx)
    # the flag was consumed; compute and check succeed afterwards
    out = s.compute(wl.misregs)[0]
    s.check()
    assert torch.equal(out, ref)
    assert s.wait_selftest(1 << 16) == 5
    s.check()
    s.close()
