"""Failure paths that must not hang or fault the GPU: bounded device waits and allocation failures.

* Bounded waits.  The plan option ``test_fail_waits`` makes every bounded device wait give
  up at its first poll (the M2L kernel's operator-slice copy, the tensor-core MMA
  completion).  The kernel then waits for its own copies with the normal limit, raises the
  plan's error flag and returns.  The next synchronising call reports MLFMA_ERR_TIMEOUT
  once; the context stays usable (a normal plan still gives the right potentials).
* Allocation failures.  An allocator callback that returns NULL on its k-th call makes plan
  creation fail with MLFMA_ERR_OUT_OF_MEMORY, and every block the callback handed out before
  is given back (nothing leaks), for every k up to the plan's own number of allocations.
"""
import math

import numpy as np
import pytest

import synth
from oracle import direct

from gpu_common import apply_plan, make_plan, rel

pytestmark = pytest.mark.gpu
K = 2.0 * math.pi
TIMEOUT, OOM = 4, 2


def _timeout_then_recover(prec, pts, q):
    import torch

    import paper_2006_15367_gb300 as mf
    dev = torch.device("cuda", 0)
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    plan = make_plan(pts, K, 3, prec, test_fail_waits=True)
    qt = torch.as_tensor(q, device=dev).to(cdt)
    plan.apply(qt)                                   # asynchronous: the flag is raised on the device
    with pytest.raises(mf.MLFMAError) as e:
        plan.info()
    assert e.value.status == TIMEOUT
    assert "bounded device wait" in str(e.value)
    plan.info()                                      # reported once, then cleared
    # host pointers: the call synchronises and reports the timeout itself
    qh = q.astype(np.complex128 if prec == "fp64" else np.complex64)
    out = np.zeros_like(qh)
    with pytest.raises(mf.MLFMAError) as e:
        mf.mlfma_apply(plan.handle, qh, out, 1)
    assert e.value.status == TIMEOUT
    plan.close()
    # the context is still usable: a normal plan gives the 3-digit potentials
    good = make_plan(pts, K, 3, prec)
    phi = apply_plan(good, q, prec)
    tg = np.arange(0, pts.shape[0], 5)
    assert rel(phi[tg], direct.direct(pts, q, K, targets=tg)) < 1e-3
    good.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_m2l_wait_timeout_is_reported(sphere4k, prec):
    pts, q, _ = sphere4k
    _timeout_then_recover(prec, pts, q[0])


def test_tensor_core_wait_timeout_is_reported():
    """16,377 points on a radius-4 sphere: the tf32x3 plan runs k_theta_map_tc on the 3 -> 4 pair."""
    pts = synth.sphere(16384 - 7, 4.0, seed=81)
    q = synth.complex_normal(82, pts.shape[0])[0]
    _timeout_then_recover("tf32x3", pts, q)


class _FailingAllocator:
    """Device memory from PyTorch's caching allocator; the fail_at-th call returns NULL."""

    def __init__(self, fail_at):
        import torch

        import paper_2006_15367_gb300 as mf
        self.fail_at = fail_at
        self.calls = 0
        self.live = {}

        def _alloc(size, stream, ctx):
            self.calls += 1
            if self.calls == self.fail_at:
                return None
            p = int(torch.cuda.caching_allocator_alloc(int(size), device=0, stream=int(stream or 0)))
            self.live[p] = int(size)
            return p

        def _free(ptr, stream, ctx):
            self.live.pop(int(ptr))
            torch.cuda.caching_allocator_delete(int(ptr))
        self.fns = (mf.ALLOC_FN(_alloc), mf.FREE_FN(_free))


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
def test_allocation_failure_leaks_nothing(prec):
    import torch

    import paper_2006_15367_gb300 as mf
    pts = synth.sphere(3000, 1.5, seed=4711)
    q = synth.complex_normal(4712, pts.shape[0])[0]
    ptd = torch.as_tensor(pts, device="cuda:0")
    # count the allocations of a successful plan creation and first apply
    counter = _FailingAllocator(fail_at=-1)
    plan = mf.Plan(ptd, K, 3, precision=prec, allocator=counter.fns)
    n_create = counter.calls
    ref = plan.apply(torch.as_tensor(q.astype(np.complex64), device="cuda:0")).cpu().numpy()
    n_total = counter.calls
    plan.close()
    assert not counter.live
    assert n_create >= 10
    for k in sorted(set(list(range(1, n_create + 1, 3)) + [n_create])):
        fa = _FailingAllocator(fail_at=k)
        with pytest.raises(mf.MLFMAError) as e:
            mf.Plan(ptd, K, 3, precision=prec, allocator=fa.fns)
        assert e.value.status == OOM, k
        assert "returned NULL" in str(e.value)
        assert not fa.live, (k, len(fa.live))
    # a failure inside the first apply (its buffers are allocated then) leaves the plan usable
    if n_total > n_create:
        fa = _FailingAllocator(fail_at=n_create + 1)
        plan = mf.Plan(ptd, K, 3, precision=prec, allocator=fa.fns)
        qt = torch.as_tensor(q.astype(np.complex64), device="cuda:0")
        with pytest.raises(mf.MLFMAError) as e:
            plan.apply(qt)
        assert e.value.status == OOM
        torch.cuda.synchronize()
        got = plan.apply(qt).cpu().numpy()
        assert rel(got, ref) < 1e-6
        plan.close()
        assert not fa.live
