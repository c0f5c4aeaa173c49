"""mlfma_apply_near_noalloc: the near-field entry point that allocates nothing.

It serves callers that cannot allocate device memory after set-up.  Its result must
equal the near-field part computed by mlfma_apply on the same plan (same kernel, so
within the per-stage tolerance of the other GPU tests) and the oracle's near-field
sums, on two calls in a row (the shared scratch array keeps the previous call's
contents).  On a fresh plan, before any apply has sized the plan's buffers, the calls
must not reach the plan's allocator and must leave PyTorch's allocated bytes unchanged.
The uniform sphere takes the warp-per-leaf P2P kernel; a clustered adaptive set with
large leaves takes the tiled one as well.  This file is collected last on purpose.
"""
import math

import numpy as np
import pytest

import synth
from oracle import mlfma as om

from gpu_common import cdtype, make_plan, rel

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-11, "fp32": 1e-5}
K = 2.0 * math.pi


class _CountingAllocator:
    """PyTorch's caching allocator behind a counter of the library's allocation calls."""

    def __init__(self):
        import torch

        import paper_2006_15367_gb300 as mf
        self.calls = 0

        def _alloc(size, stream, ctx):
            self.calls += 1
            return int(torch.cuda.caching_allocator_alloc(int(size), device=0, stream=int(stream or 0)))

        def _free(ptr, stream, ctx):
            torch.cuda.caching_allocator_delete(int(ptr))
        self.fns = (mf.ALLOC_FN(_alloc), mf.FREE_FN(_free))


def _cases():
    pts4k, q4k, _ = synth.workload("sphere4k")
    clusters = np.concatenate([synth.sphere(2500, 1.5, seed=171),
                               synth.normal(172, 3 * 1500).reshape(1500, 3) * 0.04 + np.array([0.7, -0.2, 0.4])])
    return {"sphere4k": (pts4k, 0), "clusters": (clusters, 160)}


CASES = _cases()


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_near_noalloc_matches_apply_and_oracle(name, prec):
    import torch

    import paper_2006_15367_gb300 as mf
    pts, leaf_max = CASES[name]
    n = pts.shape[0]
    dev = torch.device("cuda", 0)
    counter = _CountingAllocator()
    plan = make_plan(pts, K, 3, prec, leaf_max=leaf_max, allocator=counter.fns)
    o = om.OracleMLFMA(pts, K, 3, leaf_max=leaf_max)
    if name == "clusters":
        sizes = [o.tree.levels[l].end[b] - o.tree.levels[l].begin[b] for (l, b) in o.near]
        assert max(sizes) > 64                     # some leaves take the tiled P2P kernel
    perm = plan.export("PERM")
    charges = [synth.complex_normal(4241, n)[0], synth.complex_normal(4242, n)[0]]
    qs = [torch.as_tensor(c.astype(cdtype(prec)), device=dev) for c in charges]
    # fresh plan, before any apply: nothing reaches the allocator, torch's bytes stay put
    outs = [torch.full_like(qs[0], complex(float("nan"), float("nan"))) for _ in qs]
    torch.cuda.synchronize()
    calls0, bytes0 = counter.calls, torch.cuda.memory_allocated(dev)
    for qt, out in zip(qs, outs):                  # two calls in a row with different charges
        mf.mlfma_apply_near_noalloc(plan.handle, qt, out)
    torch.cuda.synchronize()
    assert counter.calls == calls0
    assert torch.cuda.memory_allocated(dev) == bytes0
    for c, out in zip(charges, outs):
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        ref = np.empty(n, dtype=np.complex128)
        ref[o.tree.perm] = o.p2p(c[o.tree.perm])   # the oracle's near-field sums, caller order
        assert rel(got, ref) < TOL[prec]
    # and the near-field part of a full apply on the same plan, for the last charges
    plan.apply(qs[1])
    torch.cuda.synchronize()
    near = np.empty(n, dtype=cdtype(prec))
    near[perm] = plan.export("NEAR_PHI")
    again = torch.empty_like(qs[1])
    mf.mlfma_apply_near_noalloc(plan.handle, qs[1], again)
    torch.cuda.synchronize()
    assert rel(again.cpu().numpy(), near) < TOL[prec]
    plan.close()


def test_near_noalloc_rejects_host_pointers_and_oversize():
    import torch

    import paper_2006_15367_gb300 as mf
    pts = synth.sphere(2000, 1.0, seed=5)
    plan = make_plan(pts, 2 * math.pi, 3, "fp32")
    qh = np.zeros(2000, dtype=np.complex64)
    with pytest.raises(mf.MLFMAError) as e:
        mf.mlfma_apply_near_noalloc(plan.handle, qh, qh)
    assert e.value.status == 1
    plan.close()
    big = synth.sphere(524288 + 1, 8.0, seed=6)
    plan = make_plan(big, 2 * math.pi, 3, "fp64")
    qd = torch.zeros(big.shape[0], dtype=torch.complex128, device="cuda:0")
    with pytest.raises(mf.MLFMAError) as e:
        mf.mlfma_apply_near_noalloc(plan.handle, qd, qd)
    assert e.value.status == 1 and "maximum" in str(e.value)
    plan.close()
