"""mlfma_apply_near_noalloc: the near-field entry point that allocates nothing.

It serves callers that cannot allocate device memory after set-up.  Its result
must equal the near-field part computed by mlfma_apply on the same plan (same
kernel, so within the per-stage tolerance of the other GPU tests), on two calls
in a row (the shared scratch array keeps the previous call's contents).  This
file is collected last on purpose.
"""
import math

import numpy as np
import pytest

import synth

from gpu_common import cdtype, make_plan, rel

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-11, "fp32": 1e-5}


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_near_noalloc_matches_apply(prec):
    import torch

    import paper_2006_15367_gb300 as mf
    pts, q, prm = synth.workload("sphere4k")
    plan = make_plan(pts, prm["k"], 3, prec)
    dev = torch.device("cuda", 0)
    qs = [torch.as_tensor(q[0].astype(cdtype(prec)), device=dev),
          torch.as_tensor(synth.complex_normal(4242, pts.shape[0])[0].astype(cdtype(prec)), device=dev)]
    perm = plan.export("PERM")
    for qt in qs:                      # two calls in a row with different charges
        plan.apply(qt)
        torch.cuda.synchronize()
        ref = np.empty(pts.shape[0], dtype=cdtype(prec))
        ref[perm] = plan.export("NEAR_PHI")
        out = torch.full_like(qt, complex(float("nan"), float("nan")))
        mf.mlfma_apply_near_noalloc(plan.handle, qt, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel(got, ref) < TOL[prec]
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
