"""Reverse mode in the library: mlfma_apply_vjp against the oracle's FP64 direct sums.

For an upstream gradient g (PyTorch's convention g = dL/dRe phi + i dL/dIm phi) of a real
loss L(phi), the exact gradients are (psi = A conj(g), A the exact matrix of Eq. (1))
    grad_q = conj(psi)
    grad_r_m = Re[conj(g_m) grad phi_m + q_m grad psi_m]
with grad the target-position gradient (oracle direct_grad).  The seeded g stands in for the
upstream gradient, so every expected value comes from the oracle alone.  Central differences
of L(r) = Re sum_i conj(g_i) phi_i(r) check the formula itself: moving point m changes phi_m
(target) and every phi_i through q_m (source), which is q_m times the change of psi_m.
"""
import math

import numpy as np
import pytest

import synth
from oracle import direct

from gpu_common import cdtype, make_plan, rel

pytestmark = pytest.mark.gpu
K = 2.0 * math.pi


@pytest.fixture(scope="module")
def case():
    pts = synth.ellipsoid(8192, 2.0, 1.0, 0.5, seed=6101)
    q = synth.complex_normal(6102, pts.shape[0])[0]
    g = synth.complex_normal(6103, pts.shape[0])[0]
    tg = np.sort(np.random.default_rng(6104).choice(pts.shape[0], 512, replace=False))
    gphi = direct.direct_grad(pts, q, K, targets=tg)
    gpsi = direct.direct_grad(pts, np.conj(g), K, targets=tg)
    ref_q = np.conj(direct.direct(pts, np.conj(g), K, targets=tg))
    ref_r = np.real(np.conj(g[tg])[:, None] * gphi + q[tg][:, None] * gpsi)
    return pts, q, g, tg, ref_q, ref_r


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("recompute", [False, True])
def test_vjp_matches_oracle(case, prec, recompute):
    import torch
    pts, q, g, tg, ref_q, ref_r = case
    dev = torch.device("cuda", 0)
    plan = make_plan(pts, K, 3, prec, recompute_signatures=recompute)
    assert plan.info()["recompute_signatures"] == recompute
    qt = torch.as_tensor(q.astype(cdtype(prec)), device=dev)
    gt = torch.as_tensor(g.astype(cdtype(prec)), device=dev)
    gphi = None if recompute else plan.apply_grad(qt)[1]
    gq, gr = plan.vjp(qt, gt, gphi)
    gq, gr = gq.cpu().numpy(), gr.cpu().numpy()
    assert gr.dtype == np.float64 and gr.shape == (pts.shape[0], 3)
    assert rel(gq[tg], ref_q) < 3e-3
    assert rel(gr[tg], ref_r) < 3e-3
    # grad_q alone is the adjoint apply, bit for bit
    gq2, none = plan.vjp(qt, gt, gphi, want_r=False)
    assert none is None
    assert np.array_equal(gq2.cpu().numpy(), plan.adjoint(gt).cpu().numpy())
    plan.close()


def test_stored_and_recomputed_gradients_agree(case):
    import torch
    pts, q, g, *_ = case
    dev = torch.device("cuda", 0)
    a = make_plan(pts, K, 3, "fp32")
    b = make_plan(pts, K, 3, "fp32", recompute_signatures=True)
    qt = torch.as_tensor(q.astype(np.complex64), device=dev)
    gt = torch.as_tensor(g.astype(np.complex64), device=dev)
    ra = a.vjp(qt, gt, a.apply_grad(qt)[1])
    rb = b.vjp(qt, gt, None)
    # same kernels on the same data: the recomputed grad phi is the stored one
    assert np.array_equal(ra[0].cpu().numpy(), rb[0].cpu().numpy())
    assert np.array_equal(ra[1].cpu().numpy(), rb[1].cpu().numpy())
    a.close()
    b.close()


def test_vjp_several_rhs_sums_position_gradients(case):
    import torch
    pts, q, g, tg, *_ = case
    dev = torch.device("cuda", 0)
    Q = synth.complex_normal(6111, pts.shape[0], nrhs=2)
    Gu = synth.complex_normal(6112, pts.shape[0], nrhs=2)
    plan = make_plan(pts, K, 3, "fp64")
    qt = torch.as_tensor(Q, device=dev)
    gt = torch.as_tensor(Gu, device=dev)
    gq, gr = plan.vjp(qt, gt, None)
    ref = 0.0
    for r in range(2):
        gphi = direct.direct_grad(pts, Q[r], K, targets=tg)
        gpsi = direct.direct_grad(pts, np.conj(Gu[r]), K, targets=tg)
        ref = ref + np.real(np.conj(Gu[r][tg])[:, None] * gphi + Q[r][tg][:, None] * gpsi)
        assert rel(gq[r].cpu().numpy()[tg], np.conj(direct.direct(pts, np.conj(Gu[r]), K, targets=tg))) < 1e-3
    assert rel(gr.cpu().numpy()[tg], ref) < 1e-3
    plan.close()


def test_position_gradient_formula_by_central_differences(case):
    """L(r) = Re sum_i conj(g_i) phi_i(r): its change under moving point m, from exact FP64 sums
    at target m (phi_m and psi_m with the moved point), against the library's grad_r."""
    import torch
    pts, q, g, tg, _, ref_r = case
    plan = make_plan(pts, K, 3, "fp64")
    dev = torch.device("cuda", 0)
    _, gr = plan.vjp(torch.as_tensor(q, device=dev), torch.as_tensor(g, device=dev), None)
    gr = gr.cpu().numpy()
    h = 1e-5
    scale = np.sqrt(np.mean(ref_r ** 2))
    for m, a in [(int(tg[3]), 0), (int(tg[200]), 1), (int(tg[400]), 2)]:
        vals = []
        for s in (+1, -1):
            p = pts.copy()
            p[m, a] += s * h
            phi_m = direct.direct(p, q, K, targets=[m])[0]
            psi_m = direct.direct(p, np.conj(g), K, targets=[m])[0]
            vals.append(np.real(np.conj(g[m]) * phi_m + q[m] * psi_m))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - gr[m, a]) < 2e-3 * scale, (m, a, fd, gr[m, a])
    plan.close()


def test_vjp_rejects_bad_arguments(case):
    import torch

    import paper_2006_15367_gb300 as mf
    pts, q, g, *_ = case
    plan = make_plan(pts, K, 3, "fp32")
    qt = torch.as_tensor(q.astype(np.complex64), device="cuda:0")
    with pytest.raises(mf.MLFMAError) as e:
        mf.mlfma_apply_vjp(plan.handle, qt, qt, None, None, None, 1)     # no output wanted
    assert e.value.status == 1
    qh = q.astype(np.complex64)
    out = np.zeros_like(qh)
    with pytest.raises(mf.MLFMAError) as e:
        mf.mlfma_apply_vjp(plan.handle, qh, qh, None, out, None, 1)      # host pointers
    assert e.value.status == 1
    with pytest.raises(mf.MLFMAError) as e:
        mf.mlfma_apply_vjp(plan.handle, qt, qt, None, qt.clone(), None, 0)
    assert e.value.status == 1
    plan.close()
