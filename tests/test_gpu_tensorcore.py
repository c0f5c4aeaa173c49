"""Tensor-core theta maps (precisions "tf32x3" and "bf16x3") against the oracle and the FP32 path.

The tf32x3 plans run the theta maps of the level pairs that are too large for the fused
FFT + theta-map kernels as tcgen05 GEMMs with operands split into two TF32 parts and
three products accumulated in FP32, so every stage keeps the FP32 tolerances (1e-5 per
stage against the FP64 oracle, 1e-3 end to end).  The bf16x3 plans split into BF16 parts
(16 significant bits in hi + lo): 1e-4 per stage.
"""
import math

import numpy as np
import pytest

import synth
from oracle import direct
from oracle import mlfma as om

from gpu_common import apply_plan, make_plan, rel

pytestmark = pytest.mark.gpu
K = 2.0 * math.pi


def test_tf32x3_stages_match_oracle_mid_sphere():
    """16,377 points on a radius-4 sphere: the L2L pair of levels 3 -> 4 runs on the tensor cores."""
    pts = synth.sphere(16384 - 7, 4.0, seed=81)
    q = synth.complex_normal(82, pts.shape[0])[0]
    o = om.OracleMLFMA(pts, K, 3, margin=0)
    phio, dump = o.apply(q, dump=True)
    plan = make_plan(pts, K, 3, "tf32x3")
    phi = apply_plan(plan, q, "tf32x3")
    for l in range(o.top, o.tree.nlev + 1):
        nb = o.tree.levels[l].nbox
        assert rel(plan.export("F", l).reshape(nb, -1), dump["F"][l]) < 1e-5, ("F", l)
        assert rel(plan.export("G", l).reshape(nb, -1), dump["G"][l]) < 1e-5, ("G", l)
    assert rel(phi, phio) < 1e-3
    tg = np.arange(0, pts.shape[0], 7)
    assert rel(phi[tg], direct.direct(pts, q, K, targets=tg)) < 1e-3
    assert plan.info()["precision"] == 3          # no device error flag raised
    plan.close()


def test_tf32x3_matches_fp32_large_sphere():
    """65,536 points on a radius-8 sphere: M2M and L2L theta maps of the upper levels on the
    tensor cores (several K chunks); every level's F and G against the FP32 plan."""
    pts = synth.sphere(65536, 8.0, seed=91)
    q = synth.complex_normal(92, pts.shape[0])[0]
    p32 = make_plan(pts, K, 3, "fp32")
    ptc = make_plan(pts, K, 3, "tf32x3")
    phi32 = apply_plan(p32, q, "fp32")
    phitc = apply_plan(ptc, q, "tf32x3")
    info = ptc.info()
    assert info["L"] == p32.info()["L"]
    for l in range(info["top"], info["nlev"] + 1):
        assert rel(ptc.export("F", l), p32.export("F", l)) < 1e-5, ("F", l)
        assert rel(ptc.export("G", l), p32.export("G", l)) < 1e-5, ("G", l)
    assert rel(phitc, phi32) < 1e-5
    tg = np.sort(np.random.default_rng(5).choice(pts.shape[0], 500, replace=False))
    assert rel(phitc[tg], direct.direct(pts, q, K, targets=tg)) < 1e-3
    # graph replay gives the same bits
    assert np.array_equal(apply_plan(ptc, q, "tf32x3"), phitc)
    ptc.close()
    p32.close()


def test_bf16x3_stages_match_oracle_mid_sphere():
    """Split-BF16 theta maps (hi + lo BF16 parts, three products, FP32 accumulation): every
    stage against the FP64 oracle at 1e-4 (the products carry about 16 significant bits), the
    potentials at the 3-digit target."""
    pts = synth.sphere(16384 - 7, 4.0, seed=81)
    q = synth.complex_normal(82, pts.shape[0])[0]
    o = om.OracleMLFMA(pts, K, 3, margin=0)
    phio, dump = o.apply(q, dump=True)
    plan = make_plan(pts, K, 3, "bf16x3")
    phi = apply_plan(plan, q, "bf16x3")
    for l in range(o.top, o.tree.nlev + 1):
        nb = o.tree.levels[l].nbox
        assert rel(plan.export("F", l).reshape(nb, -1), dump["F"][l]) < 1e-4, ("F", l)
        assert rel(plan.export("G", l).reshape(nb, -1), dump["G"][l]) < 1e-4, ("G", l)
    assert rel(phi, phio) < 1e-3
    tg = np.arange(0, pts.shape[0], 7)
    assert rel(phi[tg], direct.direct(pts, q, K, targets=tg)) < 1e-3
    assert plan.info()["precision"] == 2
    plan.close()


def test_bf16x3_matches_fp32_large_sphere():
    """65,536 points on a radius-8 sphere: the upper levels' theta maps in split BF16, every
    level's F and G within 1e-4 of the FP32 plan, graph replay bit-identical."""
    pts = synth.sphere(65536, 8.0, seed=91)
    q = synth.complex_normal(92, pts.shape[0])[0]
    p32 = make_plan(pts, K, 3, "fp32")
    pbf = make_plan(pts, K, 3, "bf16x3")
    phi32 = apply_plan(p32, q, "fp32")
    phibf = apply_plan(pbf, q, "bf16x3")
    info = pbf.info()
    for l in range(info["top"], info["nlev"] + 1):
        assert rel(pbf.export("F", l), p32.export("F", l)) < 1e-4, ("F", l)
        assert rel(pbf.export("G", l), p32.export("G", l)) < 1e-4, ("G", l)
    assert rel(phibf, phi32) < 1e-4
    assert np.array_equal(apply_plan(pbf, q, "bf16x3"), phibf)
    tg = np.sort(np.random.default_rng(5).choice(pts.shape[0], 500, replace=False))
    assert rel(phibf[tg], direct.direct(pts, q, K, targets=tg)) < 1e-3
    pbf.close()
    p32.close()


@pytest.mark.parametrize("prec,tol", [("tf32x3", 1e-5), ("bf16x3", 1e-4)])
@pytest.mark.parametrize("geom", ["sphere", "clusters"])
def test_dense_pairs_match_fft_path(prec, tol, geom):
    """The fine level pairs as dense tensor-core maps (opt-in: phi transforms, theta maps and shifts
    folded into one real matrix per pair and direction) against the same precision on the FFT
    path, level by level, on a level-uniform sphere and on an adaptive clustered set
    (parent-level leaves, ragged child counts); and against the direct sum."""
    if geom == "sphere":
        pts, leaf_max = synth.sphere(65536, 8.0, seed=91), 0
    else:
        pts, leaf_max = synth.cube_surface_clusters(60000, half=3.0, seed=97), 24
    q = synth.complex_normal(92, pts.shape[0])[0]
    pd = make_plan(pts, K, 3, prec, leaf_max=leaf_max, dense_samples=400)
    pf = make_plan(pts, K, 3, prec, leaf_max=leaf_max)
    info = pd.info()
    assert any(info["dense"]) and not any(pf.info()["dense"])
    for l in range(info["top"], info["nlev"]):
        if info["L"][l + 1] > 0:                                   # (l, l + 1) is a far-field pair
            assert info["dense"][l] == int(info["K"][l + 1] <= 400), l
    phid = apply_plan(pd, q, prec)
    phif = apply_plan(pf, q, prec)
    for l in range(info["top"], info["nlev"] + 1):
        if info["nbox"][l] == 0:
            continue
        assert rel(pd.export("F", l), pf.export("F", l)) < tol, ("F", l)
        assert rel(pd.export("G", l), pf.export("G", l)) < tol, ("G", l)
    assert rel(phid, phif) < tol
    assert np.array_equal(apply_plan(pd, q, prec), phid)          # graph replay: same bits
    tg = np.sort(np.random.default_rng(6).choice(pts.shape[0], 500, replace=False))
    assert rel(phid[tg], direct.direct(pts, q, K, targets=tg)) < 1e-3
    assert pd.info()["precision"] == {"tf32x3": 3, "bf16x3": 2}[prec]   # no device error flag raised
    pd.close()
    pf.close()


def test_dense_pairs_in_forest_match_single_plans():
    """A batched forest plan (tf32x3, dense fine pairs) over ellipsoids and geometries without a
    far field or without a parent level: every geometry matches its own plan and the direct
    sum (the dense kernels find parents and children through the forest's merged levels)."""
    import torch
    geoms, sizes, axes = synth.ellipsoid_batch(4, seed=4101, nmin=2000, nmax=20000, amin=1.0, amax=3.0)
    geoms = list(geoms) + [np.array([[0.0, 0.0, 0.0], [0.3, 0.1, -0.2]]), synth.sphere(900, 0.8, seed=4102)]
    pts = np.concatenate(geoms)
    off = np.concatenate([[0], np.cumsum([g.shape[0] for g in geoms])])
    Q = synth.complex_normal(4103, pts.shape[0], nrhs=1)
    dev = torch.device("cuda", 0)
    plan = make_plan(pts, K, 3, "tf32x3", offsets=off, dense_samples=400)
    assert any(plan.info()["dense"])
    out = plan.apply(torch.as_tensor(Q[0].astype(np.complex64), device=dev)).cpu().numpy()
    for gi, g in enumerate(geoms):
        sl = slice(off[gi], off[gi + 1])
        single = make_plan(g, K, 3, "tf32x3", graphs=False, dense_samples=400)
        ref = single.apply(torch.as_tensor(Q[0, sl].astype(np.complex64), device=dev)).cpu().numpy()
        assert rel(out[sl], ref) < 1e-6, gi
        assert rel(out[sl], direct.direct(g, Q[0, sl], K)) < 1e-3, gi
        single.close()
    assert plan.info()["precision"] == 3
    plan.close()
