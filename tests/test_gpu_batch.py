"""Batching forms: CUDA-graph replay, several right-hand sides, many geometries in one plan."""
import math

import numpy as np
import pytest

import synth
from oracle import direct

from gpu_common import cdtype, make_plan, rel

pytestmark = pytest.mark.gpu
K = 2.0 * math.pi


def test_graph_replay_matches_direct_launches(sphere4k):
    import torch
    pts, q, prm = sphere4k
    dev = torch.device("cuda", 0)
    g = make_plan(pts, prm["k"], 3, "fp32")                 # graphs on (default)
    e = make_plan(pts, prm["k"], 3, "fp32", graphs=False)
    Q = torch.as_tensor(synth.complex_normal(31, pts.shape[0], nrhs=3).astype(np.complex64), device=dev)
    ref = e.apply(Q[0]).cpu().numpy()
    for _ in range(3):                                     # eager + capture, then two replays
        assert np.array_equal(g.apply(Q[0]).cpu().numpy(), ref)
    # growing nrhs drops and recaptures graphs; results stay identical
    both = g.apply(Q[:2]).cpu().numpy()
    assert np.array_equal(both[0], ref)
    assert np.array_equal(both[1], e.apply(Q[1]).cpu().numpy())
    assert np.array_equal(g.apply(Q[0]).cpu().numpy(), ref)
    three = g.apply(Q).cpu().numpy()
    assert np.array_equal(three[2], e.apply(Q[2]).cpu().numpy())
    # adjoint through a graph
    assert np.array_equal(g.adjoint(Q[1]).cpu().numpy(), e.adjoint(Q[1]).cpu().numpy())
    g.close()
    e.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batched_geometries(prec):
    import torch
    geoms, sizes, axes = synth.ellipsoid_batch(5, seed=4001, nmin=500, nmax=4000, amin=0.8, amax=2.5)
    pts = np.concatenate(geoms)
    off = np.concatenate([[0], np.cumsum(sizes)])
    Q = synth.complex_normal(4002, pts.shape[0], nrhs=2)
    dev = torch.device("cuda", 0)
    plan = make_plan(pts, K, 3, prec, offsets=off)
    info = plan.info()
    assert info["n_geom"] == 5 and info["n"] == pts.shape[0]
    out = plan.apply(torch.as_tensor(Q.astype(cdtype(prec)), device=dev)).cpu().numpy()
    out2 = plan.apply(torch.as_tensor(Q.astype(cdtype(prec)), device=dev)).cpu().numpy()   # graph replay
    assert np.array_equal(out, out2)
    for gi in range(5):
        sl = slice(off[gi], off[gi + 1])
        single = make_plan(geoms[gi], K, 3, prec, graphs=False)
        for r in range(2):
            ref = single.apply(torch.as_tensor(Q[r, sl].astype(cdtype(prec)), device=dev)).cpu().numpy()
            assert np.array_equal(out[r, sl], ref)
            assert rel(out[r, sl], direct.direct(geoms[gi], Q[r, sl], K)) < 1e-3
        single.close()
    plan.close()


def test_forest_mixes_tiny_and_large_geometries():
    """Geometries without a far field (a few points), small ones and a 20k-point sphere in one
    forest plan: every geometry matches its own plan bit for bit and the direct sum."""
    import torch
    geoms = [np.array([[0.0, 0.0, 0.0], [0.3, 0.1, -0.2], [0.05, 0.0, 0.1]]),
             synth.sphere(20000, 3.0, seed=111),
             synth.sphere(40, 0.1, seed=112),
             synth.sphere(1500, 1.0, seed=113),
             np.array([[1.0, 2.0, 3.0]])]
    pts = np.concatenate(geoms)
    off = np.concatenate([[0], np.cumsum([g.shape[0] for g in geoms])])
    Q = synth.complex_normal(4012, pts.shape[0], nrhs=1)
    dev = torch.device("cuda", 0)
    plan = make_plan(pts, K, 3, "fp32", offsets=off)
    out = plan.apply(torch.as_tensor(Q[0].astype(np.complex64), device=dev)).cpu().numpy()
    for gi, g in enumerate(geoms):
        sl = slice(off[gi], off[gi + 1])
        single = make_plan(g, K, 3, "fp32", graphs=False)
        ref = single.apply(torch.as_tensor(Q[0, sl].astype(np.complex64), device=dev)).cpu().numpy()
        assert np.array_equal(out[sl], ref), gi
        assert rel(out[sl], direct.direct(g, Q[0, sl], K)) < 1e-3, gi
        single.close()
    plan.close()


@pytest.mark.parametrize("case", ["sphere", "clusters"])
def test_near_field_stream_matches_sequential(case):
    """The near field runs on a second stream beside the far field (L2O waits for it); with stage
    timings on, the two run one after the other.  Both orders give the same bits: potentials
    (one and four right-hand sides), gradients, eager and graph-replayed applies, on a uniform
    tree (L2O at the leaf level) and an adaptive one (L2O at several levels)."""
    import torch
    if case == "sphere":
        pts, leaf_max = synth.sphere(20000, 3.0, seed=121), 0
    else:
        pts = np.concatenate([synth.sphere(6000, 2.0, seed=122),
                              synth.normal(123, 3 * 3000).reshape(3000, 3) * 0.05 + np.array([0.5, 1.2, -1.0])])
        leaf_max = 32
    dev = torch.device("cuda", 0)
    Q = torch.as_tensor(synth.complex_normal(124, pts.shape[0], nrhs=4).astype(np.complex64), device=dev)
    g = make_plan(pts, K, 3, "fp32", leaf_max=leaf_max)                  # graphs
    e = make_plan(pts, K, 3, "fp32", leaf_max=leaf_max, graphs=False)
    conc = [p.apply(Q).cpu().numpy() for p in (g, e)] + [g.apply(Q[0]).cpu().numpy()]
    gconc = [t.cpu().numpy() for t in e.apply_grad(Q[1])]
    for p in (g, e):
        p.profile(True)
    seq = [p.apply(Q).cpu().numpy() for p in (g, e)] + [g.apply(Q[0]).cpu().numpy()]
    gseq = [t.cpu().numpy() for t in e.apply_grad(Q[1])]
    for a, b in zip(conc, seq):
        assert np.array_equal(a, b)
    for a, b in zip(gconc, gseq):
        assert np.array_equal(a, b)
    assert np.array_equal(conc[0], conc[1])                           # graph replay = eager launches
    assert rel(conc[2], direct.direct(pts, synth.complex_normal(124, pts.shape[0], nrhs=4)[0], K)) < 1e-3
    g.close()
    e.close()
