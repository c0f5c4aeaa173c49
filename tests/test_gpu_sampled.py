"""Sampled translation operators (Sec. 3.2.3, "Translation Operators"): the CUDA path against
the oracle's sampled operators.

Levels whose boxes are a wavelength or more keep T tabulated in the angle psi between khat and
the offset (s L intervals on [0, pi], padded by the reflections) and M2L interpolates each
(offset, sample) entry with 10-point Lagrange weights as it stages its operator slice.

Tolerances:
* tables: FP64 1e-12 (the same Legendre series in FP64 on both sides), FP32 1e-6 (one
  rounding to complex64).
* per stage, FP64 1e-10: the interpolation node u = psi S / pi (S = s L, up to ~10^3) carries
  the rounding of psi into the Lagrange weights, an order above plain summation-order noise.
* per stage, FP32 3e-5: psi from FP32 directions is good to ~1e-7 absolute, and T varies by up
  to L |T| per radian (Bernstein), so the operators differ from the FP64 oracle's by ~L 1e-7
  relative (L ~ 20-30 at the sampled levels of these spheres), against ~1e-7 for tabulated
  operators (tolerance 1e-5 there).
* end to end: 10^-digits against the FP64 direct sum.
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
S_OVER = 6
STAGE_TOL = {"fp64": 1e-10, "fp32": 3e-5}
MARGIN = {"fp64": 1, "fp32": 0}


def _sampled_levels(o, s):
    return [l for l in sorted(o.L) if om.level_is_sampled(o.k, o.tree.levels[l].edge, s)]


def _check_tables(plan, o, s, prec):
    tol = 1e-12 if prec == "fp64" else 1e-6
    info = plan.info()
    for l in _sampled_levels(o, s):
        L, edge = o.L[l], o.tree.levels[l].edge
        n = s * L + 2 * om.SAMPLED_ORDER + 1
        tab = plan.export("OPERATOR_SAMPLES", l).reshape(28, n)
        d2s = {dx * dx + dy * dy + dz * dz for dx in range(-3, 4) for dy in range(-3, 4) for dz in range(-3, 4)
               if max(abs(dx), abs(dy), abs(dz)) >= 2}
        for d2 in range(28):
            if d2 in d2s:
                ref = om.operator_samples(L, K, math.sqrt(d2) * edge, s)
                assert rel(tab[d2], ref) < tol, (l, d2)
            else:
                assert not np.any(tab[d2]), (l, d2)
        with pytest.raises(RuntimeError):
            plan.export("TRANSLATION", l)
    assert info["sampled_operators"] == s
    assert [l for l in range(len(info["sampled"])) if info["sampled"][l]] == _sampled_levels(o, s)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sampled_operators_stages_sphere4k(sphere4k, prec):
    """The 4,096-point sphere (level 3, edge one wavelength, sampled): tables, every stage and
    the potentials against the oracle with the same sampled operators."""
    pts, q, prm = sphere4k
    o = om.OracleMLFMA(pts, prm["k"], 3, margin=MARGIN[prec], sampled_operators=S_OVER)
    assert _sampled_levels(o, S_OVER) == [3]
    phio, dump = o.apply(q[0], dump=True)
    plan = make_plan(pts, prm["k"], 3, prec, sampled_operators=S_OVER)
    phi = apply_plan(plan, q[0], prec)
    _check_tables(plan, o, S_OVER, prec)
    for l in range(o.top, o.tree.nlev + 1):
        nb = o.tree.levels[l].nbox
        assert rel(plan.export("F", l).reshape(nb, -1), dump["F"][l]) < STAGE_TOL[prec], ("F", l)
        assert rel(plan.export("G", l).reshape(nb, -1), dump["G"][l]) < STAGE_TOL[prec], ("G", l)
    assert rel(phi, phio) < (1e-10 if prec == "fp64" else 1e-3)
    assert rel(phi, direct.direct(pts, q[0], K)) < 1e-3
    plan.close()


def test_sampled_operators_mid_size_sphere_fp64():
    """16,377 points on a radius-4 sphere: the levels with 4, 2 and 1 wavelength boxes are
    sampled (ragged last slices, several slices per level), every stage against the oracle."""
    pts = synth.sphere(16384 - 7, 4.0, seed=81)
    q = synth.complex_normal(82, pts.shape[0])[0]
    o = om.OracleMLFMA(pts, K, 3, sampled_operators=S_OVER)
    assert len(_sampled_levels(o, S_OVER)) >= 2
    phio, dump = o.apply(q, dump=True)
    plan = make_plan(pts, K, 3, "fp64", sampled_operators=S_OVER)
    phi = apply_plan(plan, q, "fp64")
    _check_tables(plan, o, S_OVER, "fp64")
    for l in range(o.top, o.tree.nlev + 1):
        nb = o.tree.levels[l].nbox
        assert rel(plan.export("F", l).reshape(nb, -1), dump["F"][l]) < 1e-10, ("F", l)
        assert rel(plan.export("G", l).reshape(nb, -1), dump["G"][l]) < 1e-10, ("G", l)
    assert rel(phi, phio) < 1e-10
    plan.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_sampled_operators_rhs_passes_and_memory(prec):
    """Radius-3 sphere: passes of 4 right-hand sides through the sampled M2L match single
    applies; the plan holds less device memory than the full-table plan, and the two agree to
    the interpolation error."""
    import torch
    pts = synth.sphere(12000, 3.0, seed=91)
    Q = synth.complex_normal(92, pts.shape[0], nrhs=5).astype(cdtype(prec))
    full = make_plan(pts, K, 3, prec)
    plan = make_plan(pts, K, 3, prec, sampled_operators=S_OVER)
    assert sum(plan.info()["sampled"]) >= 2
    assert plan.info()["device_bytes"] < full.info()["device_bytes"]
    dev = torch.device("cuda", 0)
    batch = plan.apply(torch.as_tensor(Q, device=dev)).cpu().numpy()
    tol = 1e-6 if prec == "fp32" else 1e-13
    for r in range(5):
        single = plan.apply(torch.as_tensor(Q[r], device=dev)).cpu().numpy()
        assert rel(batch[r], single) < tol, r
    ref = full.apply(torch.as_tensor(Q[0], device=dev)).cpu().numpy()
    assert rel(batch[0], ref) < 1e-4
    assert rel(batch[0], direct.direct(pts, Q[0].astype(np.complex128), K)) < 1e-3
    plan.close()
    full.close()


def test_sampled_operators_batched_geometries_match_separate_plans():
    """A batched plan over three spheres with sampled operators gives each geometry's separate
    plan bit for bit (the forest shares the sampled tables of a level)."""
    import torch

    import paper_2006_15367_gb300 as mf
    geoms = [synth.sphere(3000, 2.5, seed=111), synth.sphere(2500, 2.2, seed=112), synth.sphere(3500, 2.8, seed=113)]
    pts = np.concatenate(geoms)
    off = np.concatenate([[0], np.cumsum([g.shape[0] for g in geoms])]).astype(np.int64)
    dev = torch.device("cuda", 0)
    plan = mf.Plan(torch.as_tensor(pts, device=dev), K, 3, offsets=off, sampled_operators=S_OVER)
    q = synth.complex_normal(114, pts.shape[0])[0].astype(np.complex64)
    phi = plan.apply(torch.as_tensor(q, device=dev)).cpu().numpy()
    plan.close()
    for g in range(3):
        a, b = int(off[g]), int(off[g + 1])
        sp = make_plan(geoms[g], K, 3, "fp32", sampled_operators=S_OVER)
        assert sum(sp.info()["sampled"]) >= 1
        one = apply_plan(sp, q[a:b], "fp32")
        sp.close()
        assert np.array_equal(phi[a:b], one), g
        assert rel(one, direct.direct(geoms[g], q[a:b].astype(np.complex128), K)) < 1e-3


def test_sampled_operators_option_range(sphere4k):
    pts, _, prm = sphere4k
    for bad in (1, 2, 33, -1):
        with pytest.raises(RuntimeError):
            make_plan(pts, prm["k"], 3, "fp32", sampled_operators=bad)
