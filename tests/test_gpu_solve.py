"""GPU restarted GMRES around the matvec vs the oracle's dense solve.

The system is (sigma I + A) x = b with A the potential matrix.  GMRES converges
to the solution of the MLFMA operator, which differs from the exact one by the
MLFMA's own error.  So each test takes the true residual r = b - sigma x - A x of
the GPU iterate through the oracle's FP64 direct sum and bounds the distance to
the dense solution x* by the perturbation bound ||x - x*|| / ||x*|| <= kappa ||r|| /
||b||.  For sigma = 100i on the 4,096-point sphere (radius 2, k = 2 pi) kappa(sigma I
+ A) = 8.6 (SVD); the tests use kappa = 10.  The true residual itself is bounded by
the GMRES tolerance plus the MLFMA error times ||A x|| / ||b|| (below 10 here).
"""
import math

import numpy as np
import pytest

import synth
from oracle import direct, solve

from gpu_common import cdtype, make_plan, rel

pytestmark = pytest.mark.gpu
K = 2.0 * math.pi
SIGMA = 100j
KAPPA = 10.0


@pytest.fixture(scope="module")
def system4k(sphere4k):
    pts, _, prm = sphere4k
    b = synth.complex_normal(1005, pts.shape[0])[0]
    return pts, b, solve.solve_dense(pts, b, K, SIGMA)


def _run(plan, b, prec, **kw):
    import torch
    bt = torch.as_tensor(b.astype(cdtype(prec)), device="cuda")
    x, info = plan.solve(bt, **kw)
    torch.cuda.synchronize()
    return x.cpu().numpy().astype(np.complex128), info


def _true_residual(pts, b, x):
    return np.linalg.norm(b - SIGMA * x - direct.direct(pts, x, K)) / np.linalg.norm(b)


@pytest.mark.parametrize("prec,digits,tol", [("fp64", 6, 1e-8), ("fp32", 3, 1e-4)])
def test_gmres_matches_dense_solve(system4k, prec, digits, tol):
    pts, b, xs = system4k
    plan = make_plan(pts, K, digits, prec)
    x, info = _run(plan, b, prec, sigma=SIGMA, tol=tol, restart=30, max_iter=400)
    assert info["converged"] and info["rel_residual"] <= tol
    assert info["matvecs"] == info["iterations"] + info["restarts"] + 2
    r = _true_residual(pts, b, x)
    assert r <= tol + 10 * 10.0 ** -digits
    assert rel(x, xs) <= KAPPA * r


def test_gmres_restarts_and_initial_guess(system4k):
    import torch
    pts, b, xs = system4k
    plan = make_plan(pts, K, 6, "fp64")
    x, info = _run(plan, b, "fp64", sigma=SIGMA, tol=1e-8, restart=8, max_iter=800)
    assert info["converged"] and info["restarts"] > 0
    assert rel(x, xs) <= KAPPA * _true_residual(pts, b, x)
    # a converged iterate as the initial guess: the first true residual already meets tol
    bt = torch.as_tensor(b, device="cuda")
    x2, info2 = plan.solve(bt, sigma=SIGMA, tol=1e-8, restart=8, max_iter=800,
                           x0=torch.as_tensor(x, device="cuda"))
    assert info2["iterations"] == 0 and info2["matvecs"] == 1 and info2["converged"]
    assert np.array_equal(x2.cpu().numpy(), x)


def test_gmres_zero_rhs_and_iteration_cap(system4k):
    import torch
    pts, b, _ = system4k
    plan = make_plan(pts, K, 3, "fp32")
    x, info = _run(plan, np.zeros_like(b), "fp32", sigma=SIGMA, tol=1e-3)
    assert info["converged"] and info["iterations"] == 0 and not np.any(x)
    x, info = _run(plan, b, "fp32", sigma=SIGMA, tol=1e-6, restart=30, max_iter=3)
    assert not info["converged"] and info["iterations"] == 3 and info["matvecs"] == 5
    assert 1e-6 < info["rel_residual"] < 1.0
    assert abs(info["rel_residual"] - _true_residual(pts, b, x)) < 1e-2 * info["rel_residual"]


def test_gmres_rejects_bad_arguments(system4k):
    import torch

    import paper_2006_15367_gb300 as mf
    pts, b, _ = system4k
    plan = make_plan(pts, K, 3, "fp32")
    bt = torch.as_tensor(b.astype(np.complex64), device="cuda")
    x = torch.zeros_like(bt)
    for kw in (dict(restart=0), dict(restart=257), dict(tol=0.0), dict(tol=1.0), dict(max_iter=0),
               dict(sigma=complex(float("nan"), 0.0))):
        args = dict(sigma=SIGMA, tol=1e-3, restart=30, max_iter=10)
        args.update(kw)
        with pytest.raises(mf.MLFMAError) as e:
            mf.mlfma_solve_gmres(plan.handle, bt, x, args["sigma"], args["tol"], args["restart"], args["max_iter"])
        assert e.value.status == 1
    with pytest.raises(mf.MLFMAError) as e:
        mf.mlfma_solve_gmres(plan.handle, bt.cpu(), x, SIGMA, 1e-3, 30, 10)
    assert e.value.status == 1


def test_gmres_batched_plan_is_block_diagonal():
    """Three ellipsoids in one forest plan: A is block diagonal, one dense solve per block.
    kappa(sigma I + A_g) = 4.4, 19.3 and 3.4 for the three blocks (SVD), so the bound
    uses kappa = 25."""
    geoms, sizes, _ = synth.ellipsoid_batch(3, seed=4101, nmin=800, nmax=2500, amin=0.8, amax=2.0)
    pts = np.concatenate(geoms)
    off = np.concatenate([[0], np.cumsum(sizes)])
    b = synth.complex_normal(4102, pts.shape[0])[0]
    plan = make_plan(pts, K, 6, "fp64", offsets=off)
    x, info = _run(plan, b, "fp64", sigma=SIGMA, tol=1e-8, restart=30, max_iter=400)
    assert info["converged"]
    blocks = [slice(off[g], off[g + 1]) for g in range(len(sizes))]
    xs = np.concatenate([solve.solve_dense(pts[s], b[s], K, SIGMA) for s in blocks])
    ax = np.concatenate([direct.direct(pts[s], x[s], K) for s in blocks])
    r = np.linalg.norm(b - SIGMA * x - ax) / np.linalg.norm(b)
    assert r <= 1e-8 + 10 * 1e-6
    assert rel(x, xs) <= 25.0 * r
