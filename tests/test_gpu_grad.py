"""Gradients: mlfma_apply_grad and the autograd Function vs the oracle (FP64 direct sums).

Loss L = sum_i |phi_i - t_i|^2 on points of an ellipsoid surface.  Exact gradients
from the oracle: g = 2 (phi - t); q.grad = conj(direct(conj g)); r.grad =
Re[conj(g) grad phi + q grad psi] with psi = direct(conj g) (direct_grad for the
target gradients).  The MLFMA gradients must match them to the 3-digit accuracy of
the matvec; a few position components are also checked by central differences of
the exact loss (h = 1e-4).
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
def ellipsoid_case():
    pts = synth.ellipsoid(8192, 2.0, 1.0, 0.5, seed=5101)
    q = synth.complex_normal(5102, pts.shape[0])[0]
    t = synth.complex_normal(5103, pts.shape[0])[0]
    return pts, q, t


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_apply_grad_vs_direct_grad(ellipsoid_case, prec):
    import torch
    pts, q, _ = ellipsoid_case
    plan = make_plan(pts, K, 3, prec)
    phi, grad = plan.apply_grad(torch.as_tensor(q.astype(cdtype(prec)), device="cuda:0"))
    phi, grad = phi.cpu().numpy(), grad.cpu().numpy()
    tg = np.sort(np.random.default_rng(7).choice(pts.shape[0], 512, replace=False))
    ref = direct.direct_grad(pts, q, K, targets=tg)
    assert rel(grad[tg], ref) < 3e-3
    assert rel(phi[tg], direct.direct(pts, q, K, targets=tg)) < 1e-3
    # phi from apply_grad equals apply's up to the rounding of the fused gradient kernels
    phi2 = plan.apply(torch.as_tensor(q.astype(cdtype(prec)), device="cuda:0")).cpu().numpy()
    assert rel(phi, phi2) < (1e-12 if prec == "fp64" else 2e-4)
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_apply_grad_clustered_leaves(prec):
    """Adaptive tree with leaf_max 64 over a sphere and a dense cluster: near-field gradients of
    leaves with 33-64 points (two targets per lane) and of the tiled large leaves, against the
    direct-sum gradient at sampled targets, most of them in the cluster."""
    import torch
    pts = np.concatenate([synth.sphere(3000, 1.5, seed=5111),
                          synth.normal(5112, 3 * 2000).reshape(2000, 3) * 0.04 + np.array([0.2, -0.8, 0.4])])
    q = synth.complex_normal(5113, pts.shape[0])[0]
    plan = make_plan(pts, K, 3, prec, leaf_max=64)
    phi, grad = plan.apply_grad(torch.as_tensor(q.astype(cdtype(prec)), device="cuda:0"))
    phi, grad = phi.cpu().numpy(), grad.cpu().numpy()
    rng = np.random.default_rng(8)
    tg = np.sort(np.concatenate([rng.choice(3000, 100, replace=False), 3000 + rng.choice(2000, 412, replace=False)]))
    assert rel(grad[tg], direct.direct_grad(pts, q, K, targets=tg)) < 3e-3
    assert rel(phi[tg], direct.direct(pts, q, K, targets=tg)) < 1e-3
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_autograd_loss_gradients(ellipsoid_case, prec):
    import torch

    import paper_2006_15367_gb300 as mf
    pts, q, t = ellipsoid_case
    dev = torch.device("cuda", 0)
    plan = make_plan(pts, K, 3, prec)
    qt = torch.as_tensor(q.astype(cdtype(prec)), device=dev).requires_grad_(True)
    rt = torch.as_tensor(pts, device=dev).requires_grad_(True)
    tt = torch.as_tensor(t.astype(cdtype(prec)), device=dev)
    phi = mf.mlfma(qt, rt, plan)
    loss = torch.sum(torch.abs(phi - tt) ** 2)
    loss.backward()
    gq, gr = qt.grad.cpu().numpy(), rt.grad.cpu().numpy()
    # exact gradients from the oracle (FP64 direct sums)
    n = pts.shape[0]
    phi_ex = direct.direct(pts, q, K)
    g = 2.0 * (phi_ex - t)
    tg = np.sort(np.random.default_rng(11).choice(n, 512, replace=False))
    psi_t = direct.direct(pts, np.conj(g), K, targets=tg)
    gq_ref = np.conj(psi_t)
    gphi = direct.direct_grad(pts, q, K, targets=tg)
    gpsi = direct.direct_grad(pts, np.conj(g), K, targets=tg)
    gr_ref = np.real(np.conj(g[tg])[:, None] * gphi + q[tg][:, None] * gpsi)
    assert rel(gq[tg], gq_ref) < 3e-3
    assert rel(gr[tg], gr_ref) < 3e-3
    # central differences of the exact loss for a few position components
    def exact_loss(p):
        return float(np.sum(np.abs(direct.direct(p, q, K) - t) ** 2))
    h = 1e-4
    errs = []
    for m, a in [(tg[0], 0), (tg[100], 1), (tg[300], 2)]:
        pp, pm = pts.copy(), pts.copy()
        pp[m, a] += h
        pm[m, a] -= h
        fd = (exact_loss(pp) - exact_loss(pm)) / (2 * h)
        errs.append(abs(fd - gr[m, a]))
    scale = np.sqrt(np.mean(gr_ref ** 2))
    assert max(errs) < 1e-2 * scale
    plan.close()
