"""Parity at the workloads' full sizes, through the paths that only large plans take.

Each test compares the CUDA path with the oracle at the size the benchmark and the paper's
workloads use:

* 2^20-point sphere (radius 32, 9 levels), FP32: the two top levels' M2L (level 3 has
  K = 78,800 samples per box and runs the list-split M2L kernel, four warps per parent),
  the M2M pair 4 -> 3 and the L2L pair 3 -> 4, each against the oracle's own stage
  function applied to the signatures the GPU exported (Sec. 3.2.2-3.2.4, Alg. 1-2), 1e-5
  norm-relative per level.
* the same sphere with the FP64 path at 6 digits (half-wavelength leaves): 1e-6 against the
  oracle's FP64 direct sum (Eq. (1)) on 2,000 sampled targets.
* the same sphere with sampled translation operators at the levels of wavelength-sized boxes
  and above (Sec. 3.2.3): the top level's M2L against the oracle's, 1e-4 (FP32); the
  potentials against the direct sum, 1e-3 (FP32) and 1e-6 (FP64, 6 digits, oversampling 16).
* the same sphere with split-TF32 tensor-core theta maps: 1e-3 against the direct sum and
  1e-5 per level (F and G) against the FP32 plan.
* 4,194,304 points on a cube surface with 64 dense clusters (adaptive tree, leaf_max 64,
  4 digits), FP32 and split-BF16 tensor-core theta maps: 1e-4 against the direct sum on
  2,000 sampled targets.
* 256 ellipsoids in one batched plan: 1e-3 against the direct sum of each of 8 sampled
  geometries (250 targets each).
* the (8, 4, 2) ellipsoid with 262,144 points: reverse mode (charges and positions) through
  the autograd Function, 512 sampled entries against the oracle's direct sums and their
  gradients, 1e-3, and the position gradient by central differences of exact sums.
"""
import math

import numpy as np
import pytest

import synth
from oracle import direct
from oracle import mlfma as om

from gpu_common import apply_plan, make_plan, rel

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
K = 2.0 * math.pi


def _targets(n, m, seed):
    return np.sort(np.random.default_rng(seed).choice(n, m, replace=False))


@pytest.fixture(scope="module")
def sphere1m():
    return synth.workload("sphere1m")


def test_sphere1m_top_levels_against_oracle_stages(sphere1m):
    pts, q, prm = sphere1m
    plan = make_plan(pts, prm["k"], 3, "fp32")
    apply_plan(plan, q[0], "fp32")
    o = om.OracleMLFMA(pts, prm["k"], 3, margin=0)
    info = plan.info()
    assert info["top"] == o.top == 3
    assert [info["L"][l] for l in range(3, 10)] == [o.L[l] for l in range(3, 10)]
    assert info["K"][3] >= 49152                    # the list-split M2L path
    F = {l: plan.export("F", l).reshape(o.tree.levels[l].nbox, -1).astype(np.complex128) for l in (3, 4)}
    G = {l: plan.export("G", l).reshape(o.tree.levels[l].nbox, -1).astype(np.complex128) for l in (3, 4)}
    # M2M 4 -> 3 (no leaves at level 3: F_3 is the sum over the children)
    F3 = np.zeros_like(F[3])
    o.m2m(3, F[4], F3)
    assert rel(F[3], F3) < 1e-5
    # M2L at level 3 (the top: G_3 is its M2L alone)
    assert rel(G[3], o.m2l(3, F[3])) < 1e-5
    # level 4: its own M2L plus the L2L from level 3
    G4 = o.m2l(4, F[4])
    o.l2l(3, G[3], G4)
    assert rel(G[4], G4) < 1e-5
    # the leaf level (K = 162: five full 32-sample slices and a ragged slice of two samples,
    # taken by the tail kernel) on 400 sampled target boxes: their M2L sums from the exported
    # F_9 plus the L2L of the exported G_8 to them
    lev9, lev8 = o.tree.levels[9], o.tree.levels[8]
    F9 = plan.export("F", 9).reshape(lev9.nbox, -1).astype(np.complex128)
    G8 = plan.export("G", 8).reshape(lev8.nbox, -1).astype(np.complex128)
    G9 = plan.export("G", 9).reshape(lev9.nbox, -1).astype(np.complex128)
    tb = np.sort(np.random.default_rng(2003).choice(lev9.nbox, 400, replace=False))
    offs, cols = o.V[9]
    ref = np.zeros((tb.shape[0], F9.shape[1]), dtype=np.complex128)
    for i, t in enumerate(tb):
        for src in cols[offs[t]:offs[t + 1]]:
            ref[i] += o.T(9, lev9.ijk[t] - lev9.ijk[src]) * F9[src]
    par = lev9.parent[tb]
    sh = np.conj(o.shift_m2m(8, lev9.center[tb] - lev8.center[par])) * G8[par]
    ref += om.anterpolate(sh, o.grid[9], o.grid[8], o.A[8])
    assert rel(G9[tb], ref) < 1e-5
    assert rel(G9[tb][:, 160:], ref[:, 160:]) < 1e-5
    plan.close()


def test_sphere1m_fp64_six_digits(sphere1m):
    pts, q, prm = sphere1m
    plan = make_plan(pts, prm["k"], 6, "fp64")
    assert abs(plan.info()["leaf_edge"] - 0.5) < 1e-15
    phi = apply_plan(plan, q[0], "fp64")
    plan.close()
    tg = _targets(pts.shape[0], 2000, 2001)
    assert rel(phi[tg], direct.direct(pts, q[0], prm["k"], targets=tg)) < 1e-6


def test_sphere1m_sampled_operators(sphere1m):
    """Sampled translation operators (Sec. 3.2.3) on the 2^20 sphere: the levels with boxes of
    16 down to 1 wavelength keep angle tables instead of T[316][K].  FP32 (oversampling 6): the
    top level's M2L (list-split kernel) against the oracle's m2l with sampled operators on the
    exported F_3, 1e-4 (FP32 angles good to ~2e-7 and dT/dpsi up to L |T|, L ~ 200 there); the
    potentials within 1e-3 of the direct sum.  FP64 at 6 digits (oversampling 16): 1e-6 against
    the direct sum.  At 6 digits the one-wavelength level has L = 26 and max |T| some 10^4 times
    the sums it produces, so the interpolation error relative to max |T| must stay near 1e-11:
    with oversampling 8 (1e-8) the potentials are off by 1.5e-4 (the oracle with the same
    sampled operators gives 1.7e-4 on the 4,096-point sphere; 6.6e-8 at oversampling 16)."""
    pts, q, prm = sphere1m
    plan = make_plan(pts, prm["k"], 3, "fp32", sampled_operators=6)
    phi = apply_plan(plan, q[0], "fp32")
    o = om.OracleMLFMA(pts, prm["k"], 3, margin=0, sampled_operators=6)
    info = plan.info()
    assert [l for l, v in enumerate(info["sampled"]) if v] == \
        [l for l in sorted(o.L) if om.level_is_sampled(o.k, o.tree.levels[l].edge, 6)] == [3, 4, 5, 6, 7]
    F3 = plan.export("F", 3).reshape(o.tree.levels[3].nbox, -1).astype(np.complex128)
    G3 = plan.export("G", 3).reshape(o.tree.levels[3].nbox, -1).astype(np.complex128)
    assert rel(G3, o.m2l(3, F3)) < 1e-4
    plan.close()
    tg = _targets(pts.shape[0], 2000, 2004)
    assert rel(phi[tg], direct.direct(pts, q[0], prm["k"], targets=tg)) < 1e-3
    p64 = make_plan(pts, prm["k"], 6, "fp64", sampled_operators=16)
    assert sum(p64.info()["sampled"]) >= 3
    phi64 = apply_plan(p64, q[0], "fp64")
    p64.close()
    assert rel(phi64[tg], direct.direct(pts, q[0], prm["k"], targets=tg)) < 1e-6


def test_sphere1m_tf32x3(sphere1m):
    pts, q, prm = sphere1m
    p32 = make_plan(pts, prm["k"], 3, "fp32")
    ptc = make_plan(pts, prm["k"], 3, "tf32x3")
    phi32 = apply_plan(p32, q[0], "fp32")
    phitc = apply_plan(ptc, q[0], "tf32x3")
    info = ptc.info()
    for l in range(info["top"], info["nlev"] + 1):
        assert rel(ptc.export("F", l), p32.export("F", l)) < 1e-5, ("F", l)
        assert rel(ptc.export("G", l), p32.export("G", l)) < 1e-5, ("G", l)
    assert rel(phitc, phi32) < 1e-5
    ptc.close()
    p32.close()
    tg = _targets(pts.shape[0], 2000, 2002)
    assert rel(phitc[tg], direct.direct(pts, q[0], prm["k"], targets=tg)) < 1e-3


@pytest.fixture(scope="module")
def cube4m():
    pts, q, prm = synth.workload("cubeclusters4m")
    tg = _targets(pts.shape[0], 2000, 3003)
    return pts, q, prm, tg, direct.direct(pts, q[0], prm["k"], targets=tg)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_cubeclusters4m_four_digits(cube4m, prec):
    pts, q, prm, tg, ref = cube4m
    plan = make_plan(pts, prm["k"], prm["digits"], prec, leaf_max=prm["leaf_max"])
    phi = apply_plan(plan, q[0], prec)
    info = plan.info()
    plan.close()
    assert info["top"] > 0
    assert rel(phi[tg], ref) < 1e-4


def test_batch256_sampled_geometries():
    import torch

    import paper_2006_15367_gb300 as mf
    geoms, sizes, _ = synth.ellipsoid_batch(256, seed=4001)
    pts = np.concatenate(geoms)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    q = synth.complex_normal(4002, pts.shape[0])[0]
    dev = torch.device("cuda", 0)
    plan = mf.Plan(torch.as_tensor(pts, device=dev), K, 3, offsets=off)
    assert plan.info()["n_geom"] == 256
    phi = plan.apply(torch.as_tensor(q.astype(np.complex64), device=dev)).cpu().numpy()
    plan.close()
    rng = np.random.default_rng(4005)
    for g in np.sort(rng.choice(256, 8, replace=False)):
        a, b = int(off[g]), int(off[g + 1])
        tg = np.sort(rng.choice(b - a, min(250, b - a), replace=False))
        ref = direct.direct(pts[a:b], q[a:b], K, targets=tg)
        assert rel(phi[a:b][tg], ref) < 1e-3, g


def test_ellipsoid256k_reverse_mode():
    """Config of the adjoint form: the autograd Function on 262,144 points of the (8, 4, 2)
    ellipsoid, upstream gradient g seeded (phi.backward(g): the loss Re sum conj(g) phi)."""
    import torch

    import paper_2006_15367_gb300 as mf
    pts, q, prm = synth.workload("ellipsoid256k")
    q = q[0]
    g = synth.complex_normal(5003, pts.shape[0])[0]
    dev = torch.device("cuda", 0)
    plan = make_plan(pts, prm["k"], 3, "fp32")
    qt = torch.as_tensor(q.astype(np.complex64), device=dev).requires_grad_(True)
    rt = torch.as_tensor(pts, device=dev).requires_grad_(True)
    phi = mf.mlfma(qt, rt, plan)
    phi.backward(torch.as_tensor(g.astype(np.complex64), device=dev))
    gq, gr = qt.grad.cpu().numpy(), rt.grad.cpu().numpy()
    plan.close()
    tg = _targets(pts.shape[0], 512, 5004)
    psi_conj = np.conj(direct.direct(pts, np.conj(g), prm["k"], targets=tg))
    gphi = direct.direct_grad(pts, q, prm["k"], targets=tg)
    gpsi = direct.direct_grad(pts, np.conj(g), prm["k"], targets=tg)
    ref_r = np.real(np.conj(g[tg])[:, None] * gphi + q[tg][:, None] * gpsi)
    assert rel(gq[tg], psi_conj) < 1e-3
    assert rel(gr[tg], ref_r) < 1e-3
    # central differences (h = 1e-4) of L(r) = Re sum conj(g_i) phi_i(r) by exact sums at the moved point
    h = 1e-4
    scale = np.sqrt(np.mean(ref_r ** 2))
    for m, a in [(int(tg[5]), 0), (int(tg[250]), 1), (int(tg[500]), 2)]:
        vals = []
        for s in (+1, -1):
            p = pts.copy()
            p[m, a] += s * h
            phi_m = direct.direct(p, q, prm["k"], targets=[m])[0]
            psi_m = direct.direct(p, np.conj(g), prm["k"], targets=[m])[0]
            vals.append(np.real(np.conj(g[m]) * phi_m + q[m] * psi_m))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - gr[m, a]) < 1e-2 * scale, (m, a, fd, gr[m, a])
