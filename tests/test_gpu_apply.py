"""GPU MLFMA apply vs the oracle: every stage, the final potentials, and the API contract.

Tolerances:
* FP64 path vs the FP64 oracle MLFMA (same grids, lists and operators): only
  summation order differs -> 1e-11 per stage and end to end.
* FP32 path vs the oracle: rounding of complex64 data and operators, ~1e-7 per
  stage (tolerance 1e-5); the far field at quarter-wavelength leaves multiplies it
  by |T| ~ 1e3 (low-frequency growth of h_n) -> 1e-3 end to end, which is also
  the 3-digit target against the exact sum.
* Against the FP64 direct sum: 10^-digits (the requested accuracy).
"""
import math

import numpy as np
import pytest

import synth
from oracle import direct
from oracle import mlfma as om

from gpu_common import apply_plan, cdtype, make_plan, rel

pytestmark = pytest.mark.gpu
K = 2.0 * math.pi
STAGE_TOL = {"fp64": 1e-11, "fp32": 1e-5}
END_TOL = {"fp64": 1e-11, "fp32": 1e-3}


# the library's default truncation margin: d0 = digits + 1 (FP64), digits + 0 (FP32)
MARGIN = {"fp64": 1, "fp32": 0}


@pytest.fixture(scope="module")
def oracle4k(sphere4k):
    pts, q, prm = sphere4k
    out = {}
    for prec in ("fp64", "fp32"):
        o = om.OracleMLFMA(pts, prm["k"], 3, margin=MARGIN[prec])
        phi, dump = o.apply(q[0], dump=True)
        out[prec] = (o, phi, dump)
    ref = direct.direct(pts, q[0], prm["k"])
    return out, ref


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_stages_match_oracle_sphere4k(sphere4k, oracle4k, prec):
    pts, q, prm = sphere4k
    (o, phio, dump), ref = oracle4k[0][prec], oracle4k[1]
    plan = make_plan(pts, prm["k"], 3, prec)
    phi = apply_plan(plan, q[0], prec)
    assert rel(plan.export("NEAR_PHI"), dump["near"]) < STAGE_TOL[prec]
    for l in range(o.top, o.tree.nlev + 1):
        nb = o.tree.levels[l].nbox
        assert rel(plan.export("F", l).reshape(nb, -1), dump["F"][l]) < STAGE_TOL[prec], ("F", l)
        assert rel(plan.export("G", l).reshape(nb, -1), dump["G"][l]) < STAGE_TOL[prec], ("G", l)
        T = plan.export("TRANSLATION", l).reshape(316, -1)
        ci = 0
        for dz in range(-3, 4):
            for dy in range(-3, 4):
                for dx in range(-3, 4):
                    if max(abs(dx), abs(dy), abs(dz)) <= 1:
                        continue
                    if ci % 11 == 0:
                        assert rel(T[ci], o.T(l, (dx, dy, dz))) < (1e-12 if prec == "fp64" else 1e-6), (l, ci)
                    ci += 1
    assert rel(phi, phio) < END_TOL[prec]
    assert rel(phi, ref) < 1e-3
    plan.close()


def test_six_digits_fp64_half_wavelength_leaves(sphere4k):
    pts, q, prm = sphere4k
    plan = make_plan(pts, prm["k"], 6, "fp64")
    assert abs(plan.info()["leaf_edge"] - 0.5) < 1e-15         # default leaf for digits >= 5
    phi = apply_plan(plan, q[0], "fp64")
    o = om.OracleMLFMA(pts, prm["k"], 6, leaf_edge=0.5)
    # roundoff amplified by max |T| ~ 1e6 at the leaf level (L = 18, k|X| = 2 pi)
    assert rel(phi, o.apply(q[0])) < 1e-9
    assert rel(phi, direct.direct(pts, q[0], prm["k"])) < 1e-6
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("leaf_max", [24, 64, 200])
def test_adaptive_tree_matches_oracle(prec, leaf_max):
    """A sphere with a dense cluster, adaptive tree: every stage against the oracle.  With
    leaf_max 64 the cluster's leaves hold 33-64 points (the near-field warp takes two targets
    per lane); with 200 they hold up to 200 (tiles of 128 targets, and the pairs of mutually near
    large leaves evaluated once by the symmetric pass)."""
    pts = np.concatenate([synth.sphere(3000, 1.5, seed=71),
                          synth.normal(72, 3 * 1200).reshape(1200, 3) * 0.05 + np.array([0.9, 0.2, -0.3])])
    q = synth.complex_normal(73, pts.shape[0])[0]
    o = om.OracleMLFMA(pts, K, 3, leaf_max=leaf_max, margin=MARGIN[prec])
    phio, dump = o.apply(q, dump=True)
    plan = make_plan(pts, K, 3, prec, leaf_max=leaf_max)
    phi = apply_plan(plan, q, prec)
    for l in range(o.top, o.tree.nlev + 1):
        nb = o.tree.levels[l].nbox
        assert rel(plan.export("F", l).reshape(nb, -1), dump["F"][l]) < STAGE_TOL[prec], ("F", l)
        assert rel(plan.export("G", l).reshape(nb, -1), dump["G"][l]) < STAGE_TOL[prec], ("G", l)
    assert rel(plan.export("NEAR_PHI"), dump["near"]) < STAGE_TOL[prec]
    assert rel(phi, phio) < END_TOL[prec]
    assert rel(phi, direct.direct(pts, q, K)) < 1e-3
    plan.close()


def test_mid_size_sphere_stages_fp64():
    """16,384 points on a radius-4 sphere (6 levels, several tiles per kernel, ragged counts)."""
    pts = synth.sphere(16384 - 7, 4.0, seed=81)
    q = synth.complex_normal(82, pts.shape[0])[0]
    o = om.OracleMLFMA(pts, K, 3)
    phio, dump = o.apply(q, dump=True)
    plan = make_plan(pts, K, 3, "fp64")
    phi = apply_plan(plan, q, "fp64")
    for l in range(o.top, o.tree.nlev + 1):
        nb = o.tree.levels[l].nbox
        assert rel(plan.export("F", l).reshape(nb, -1), dump["F"][l]) < 1e-11, ("F", l)
        assert rel(plan.export("G", l).reshape(nb, -1), dump["G"][l]) < 1e-11, ("G", l)
    assert rel(phi, phio) < 1e-11
    tg = np.arange(0, pts.shape[0], 7)
    assert rel(phi[tg], direct.direct(pts, q, K, targets=tg)) < 1e-3
    plan.close()


def test_adjoint_identity_and_conjugation(sphere4k):
    import torch
    pts, q, prm = sphere4k
    r = synth.complex_normal(91, pts.shape[0])[0]
    for prec, tol in (("fp64", 1e-12), ("fp32", 1e-5)):
        plan = make_plan(pts, prm["k"], 3, prec)
        dev = torch.device("cuda", 0)
        qt = torch.as_tensor(q[0].astype(cdtype(prec)), device=dev)
        rt = torch.as_tensor(r.astype(cdtype(prec)), device=dev)
        Aq = plan.apply(qt).cpu().numpy().astype(np.complex128)
        AHr = plan.adjoint(rt).cpu().numpy().astype(np.complex128)
        lhs = np.vdot(r, Aq)                    # <r, A q>
        rhs = np.vdot(AHr, q[0])                # <A^H r, q>
        assert abs(lhs - rhs) <= tol * np.linalg.norm(r) * np.linalg.norm(Aq)
        Acr = plan.apply(torch.as_tensor(np.conj(r).astype(cdtype(prec)), device=dev)).cpu().numpy()
        assert np.array_equal(np.conj(Acr), AHr.astype(cdtype(prec)))
        plan.close()


def test_reciprocity_fp64(sphere4k):
    pts, q, prm = sphere4k
    p = synth.complex_normal(93, pts.shape[0])[0]
    plan = make_plan(pts, prm["k"], 3, "fp64")
    Aq, Ap = apply_plan(plan, q[0], "fp64"), apply_plan(plan, p, "fp64")
    assert abs(p @ Aq - q[0] @ Ap) <= 1e-3 * np.linalg.norm(p) * np.linalg.norm(Aq)
    plan.close()


def test_multiple_rhs_and_host_pointers(sphere4k):
    import torch
    pts, _, prm = sphere4k
    Q = synth.complex_normal(95, pts.shape[0], nrhs=3).astype(np.complex64)
    plan = make_plan(pts, prm["k"], 3, "fp32")
    dev = torch.device("cuda", 0)
    batch = plan.apply(torch.as_tensor(Q, device=dev)).cpu().numpy()
    for r in range(3):
        single = plan.apply(torch.as_tensor(Q[r], device=dev)).cpu().numpy()
        assert np.array_equal(batch[r], single)
    # host (numpy) buffers through the same C call give the same bits
    host_out = np.zeros_like(Q)
    import paper_2006_15367_gb300 as mf
    mf.mlfma_apply(plan.handle, Q, host_out, 3)
    assert np.array_equal(host_out, batch)
    plan.close()


def test_edge_cases_exact():
    """No far field (one leaf / tiny sets): the result is the exact direct sum."""
    cases = [np.zeros((1, 3)), np.array([[0.0, 0, 0], [0.1, 0.2, 0.05]]), np.zeros((4, 3)),
             synth.sphere(40, 0.05, seed=5)]
    for pts in cases:
        q = synth.complex_normal(97, pts.shape[0])[0]
        plan = make_plan(pts, K, 3, "fp64")
        assert plan.info()["top"] == 0
        phi = apply_plan(plan, q, "fp64")
        ref = direct.direct(pts, q, K)
        assert np.max(np.abs(phi - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
        plan.close()


def test_invalid_arguments_report_status():
    import torch

    import paper_2006_15367_gb300 as mf
    dev = torch.device("cuda", 0)
    bad = synth.sphere(100, 1.0, seed=1)
    bad[17, 1] = np.nan
    with pytest.raises(mf.MLFMAError) as e:
        make_plan(bad, K, 3)
    assert e.value.status == 1 and "non-finite" in str(e.value)
    pts = synth.sphere(100, 1.0, seed=1)
    plan = make_plan(pts, K, 3)
    q = torch.zeros(100, dtype=torch.complex64, device=dev)
    with pytest.raises(mf.MLFMAError) as e:
        mf.mlfma_apply(plan.handle, q, q, 0)
    assert e.value.status == 1
    with pytest.raises(mf.MLFMAError) as e:
        plan.export("F", 99)
    assert e.value.status == 1
    plan.close()


@pytest.mark.slow
def test_full_size_sphere_fp32_three_digits():
    """2^20 points, radius 32: 3 digits against the FP64 direct sum on 2,000 sampled targets."""
    pts, q, prm = synth.workload("sphere1m")
    plan = make_plan(pts, prm["k"], 3, "fp32")
    phi = apply_plan(plan, q[0], "fp32")
    tg = np.sort(np.random.default_rng(2001).choice(pts.shape[0], 2000, replace=False))
    ref = direct.direct(pts, q[0], prm["k"], targets=tg)
    assert rel(phi[tg], ref) < 1e-3
    plan.close()


@pytest.mark.slow
def test_full_size_sphere_fp64_three_digits():
    """The FP64 path at 2^20 points: the top level's transforms (length 400) take row tiles of
    more than 48 KB of shared memory."""
    pts, q, prm = synth.workload("sphere1m")
    plan = make_plan(pts, prm["k"], 3, "fp64")
    phi = apply_plan(plan, q[0], "fp64")
    tg = np.sort(np.random.default_rng(2001).choice(pts.shape[0], 2000, replace=False))
    ref = direct.direct(pts, q[0], prm["k"], targets=tg)
    assert rel(phi[tg], ref) < 1e-3
    plan.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_rhs_passes_match_single_applies(sphere4k, prec):
    """9 right-hand sides run as two passes of 4 (kernels sharing exponentials and operator
    loads) and one single pass; each matches its own single apply.  Graphs captured before and
    after the signature buffers grow give the same results."""
    import torch
    pts, _, prm = sphere4k
    Q = synth.complex_normal(98, pts.shape[0], nrhs=9).astype(cdtype(prec))
    plan = make_plan(pts, prm["k"], 3, prec)
    dev = torch.device("cuda", 0)
    before = [plan.apply(torch.as_tensor(Q[r], device=dev)).cpu().numpy() for r in range(2)]
    batch = plan.apply(torch.as_tensor(Q, device=dev)).cpu().numpy()
    tol = 1e-6 if prec == "fp32" else 1e-13
    for r in range(9):
        single = plan.apply(torch.as_tensor(Q[r], device=dev)).cpu().numpy()
        assert rel(batch[r], single) < tol, r
        if r < 2:
            assert np.array_equal(single, before[r])
    plan.close()


def test_rhs_passes_batched_geometries():
    """A plan over 3 geometries with 5 right-hand sides (one pass of 4, one single)."""
    import torch

    import paper_2006_15367_gb300 as mf
    geoms = [synth.sphere(1500, 1.2, seed=101), synth.sphere(900, 0.8, seed=102), synth.sphere(2100, 1.5, seed=103)]
    pts = np.concatenate(geoms)
    off = np.concatenate([[0], np.cumsum([g.shape[0] for g in geoms])]).astype(np.int64)
    dev = torch.device("cuda", 0)
    plan = mf.Plan(torch.as_tensor(pts, device=dev), K, 3, offsets=off)
    Q = synth.complex_normal(99, pts.shape[0], nrhs=5).astype(np.complex64)
    one = plan.apply(torch.as_tensor(Q[0], device=dev)).cpu().numpy()
    batch = plan.apply(torch.as_tensor(Q, device=dev)).cpu().numpy()
    again = plan.apply(torch.as_tensor(Q[0], device=dev)).cpu().numpy()
    assert np.array_equal(one, again)
    assert rel(batch[0], one) < 1e-6
    for g in range(3):
        a, b = int(off[g]), int(off[g + 1])
        ref = direct.direct(pts[a:b], Q[4][a:b].astype(np.complex128), K)
        assert rel(batch[4][a:b], ref) < 1e-3
    plan.close()


TILE_CANDIDATES = [[20480, 32768, 40960], [16384, 24576, 32768], [32768, 65536, 65536], [12288, 16384, 24576]]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_autotuned_tiles_keep_results(sphere4k, prec):
    """The plan-time autotuner picks one of its candidate tile budgets; the potentials match the
    default plan up to the summation order of the theta maps (a budget can move a level pair
    between the fused kernels and the GEMM path)."""
    pts, q, prm = sphere4k
    plan0 = make_plan(pts, K, 3, prec)
    plan1 = make_plan(pts, K, 3, prec, autotune=True)
    assert plan0.info()["tile_bytes"] == TILE_CANDIDATES[0]
    assert plan1.info()["tile_bytes"] in TILE_CANDIDATES
    a = apply_plan(plan0, q[0], prec)
    b = apply_plan(plan1, q[0], prec)
    assert rel(b, a) < (1e-12 if prec == "fp64" else 1e-5)
    assert rel(b, direct.direct(pts, q[0], K)) < 1e-3
