"""Octree, Morton keys and interaction lists built on the GPU are bit-exact to the oracle."""
import math

import numpy as np
import pytest

import synth
from oracle import mlfma as om
from oracle import tree as otr

from gpu_common import (assert_tree_matches, make_plan, near_lists_from_plan, oracle_near_lists,
                        uniform_tree_and_v)

pytestmark = pytest.mark.gpu
K = 2.0 * math.pi


def test_tree_and_lists_sphere4k(sphere4k):
    pts, q, prm = sphere4k
    o = om.OracleMLFMA(pts, prm["k"], 3, margin=0)        # FP32 plans: d0 = digits
    plan = make_plan(pts, prm["k"], 3)
    assert_tree_matches(plan, o.tree, o.V)
    assert near_lists_from_plan(plan, o.tree) == oracle_near_lists(o)
    info = plan.info()
    assert info["top"] == o.top
    assert [info["L"][l] for l in range(o.top, o.tree.nlev + 1)] == [o.L[l] for l in range(o.top, o.tree.nlev + 1)]
    plan.close()


@pytest.mark.parametrize("leaf_max", [8, 24])
def test_tree_and_lists_adaptive(leaf_max):
    pts = np.concatenate([synth.sphere(3000, 1.5, seed=61),
                          synth.normal(62, 3 * 1500).reshape(1500, 3) * 0.05 + np.array([0.9, 0.2, -0.3]),
                          synth.normal(63, 3 * 500).reshape(500, 3) * 0.02 - 0.8])
    o = om.OracleMLFMA(pts, K, 3, leaf_max=leaf_max)
    plan = make_plan(pts, K, 3, leaf_max=leaf_max)
    assert_tree_matches(plan, o.tree, o.V)
    assert near_lists_from_plan(plan, o.tree) == oracle_near_lists(o)
    plan.close()


def test_degenerate_point_sets():
    # single point, two points, coincident points, a line, everything in one leaf
    cases = [np.zeros((1, 3)), np.array([[0.0, 0, 0], [0.1, 0.2, 0.05]]), np.zeros((5, 3)),
             np.stack([np.linspace(0, 7, 300), np.zeros(300), np.zeros(300)], axis=1),
             synth.sphere(50, 0.05, seed=3)]
    for pts in cases:
        o = om.OracleMLFMA(pts, K, 3)
        plan = make_plan(pts, K, 3)
        assert_tree_matches(plan, o.tree, o.V)
        assert near_lists_from_plan(plan, o.tree) == oracle_near_lists(o)
        assert plan.info()["top"] == (o.top or 0)
        plan.close()


@pytest.mark.slow
def test_tree_and_vlists_full_size_sphere():
    """2^20 points on the 64-wavelength sphere (9 levels): every key, box and V list."""
    pts, q, prm = synth.workload("sphere1m")
    t, coll, V = uniform_tree_and_v(pts, 0.25)
    plan = make_plan(pts, prm["k"], 3)
    assert t.nlev == 9
    assert_tree_matches(plan, t, V)
    info = plan.info()
    # near pairs: sum over leaves of n_b * sum_{u in U(b)} n_u minus self pairs
    L = t.levels[t.nlev]
    offs, cols = otr.uniform_u_lists(t, coll)
    cnt = L.end - L.begin
    pairs = sum(int(cnt[b]) * int(cnt[cols[offs[b]:offs[b + 1]]].sum()) for b in range(L.nbox)) - t.n
    assert info["near_pairs"] == pairs
    plan.close()
