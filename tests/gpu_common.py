"""Shared helpers of the GPU parity tests (comparison with the oracle)."""
import numpy as np

from oracle import tree as otr


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def cdtype(prec):
    return np.complex128 if prec == "fp64" else np.complex64


def make_plan(pts, k, digits, prec="fp32", leaf_max=0, **kw):
    import torch

    import paper_2006_15367_gb300 as mf
    dev = torch.device("cuda", 0)
    return mf.Plan(torch.as_tensor(np.ascontiguousarray(pts), device=dev), k, digits, leaf_max=leaf_max,
                   precision=prec, **kw)


def apply_plan(plan, q, prec):
    import torch
    dev = torch.device("cuda", 0)
    qt = torch.as_tensor(np.ascontiguousarray(q).astype(cdtype(prec)), device=dev)
    out = plan.apply(qt)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def assert_tree_matches(plan, t, V=None, levels=None):
    """Bit-exact comparison of keys, permutation, boxes (and V lists) with an oracle tree."""
    assert np.array_equal(plan.export("PERM"), t.perm.astype(np.int32))
    assert np.array_equal(plan.export("KEYS"), t.key)
    info = plan.info()
    assert info["nlev"] == t.nlev
    for l in (levels or range(1, t.nlev + 1)):
        L = t.levels[l]
        assert np.array_equal(plan.export("BOX_KEY", l), L.key), l
        assert np.array_equal(plan.export("BOX_BEGIN", l), L.begin.astype(np.int32)), l
        assert np.array_equal(plan.export("BOX_END", l), L.end.astype(np.int32)), l
        if l > 1:
            assert np.array_equal(plan.export("BOX_PARENT", l), L.parent.astype(np.int32)), l
        assert np.array_equal(plan.export("BOX_LEAF", l).astype(bool), L.leaf), l
        if V is not None and l >= 2 and l in V:
            offs, cols = V[l]
            assert np.array_equal(plan.export("V_OFFSETS", l), offs.astype(np.int32)), l
            assert np.array_equal(plan.export("V_SOURCES", l), cols.astype(np.int32)), l


def near_lists_from_plan(plan, t):
    """Near sources per leaf (level, box) as exported by the plan."""
    offs = plan.export("NEAR_OFFSETS")
    src = plan.export("NEAR_SOURCES")
    m = src.shape[0] // 2
    lev, box = src[:m], src[m:]
    leaves = [(l, int(b)) for l in range(1, t.nlev + 1) for b in np.nonzero(t.levels[l].leaf)[0]]
    assert offs.shape[0] == len(leaves) + 1
    return {leaf: [(int(lev[e]), int(box[e])) for e in range(offs[i], offs[i + 1])] for i, leaf in enumerate(leaves)}


def oracle_near_lists(o):
    t = o.tree
    if o.uniform:
        offs, cols = o.U
        return {(t.nlev, b): [(t.nlev, int(s)) for s in cols[offs[b]:offs[b + 1]]] for b in range(t.levels[t.nlev].nbox)}
    return o.near


def uniform_tree_and_v(pts, leaf_edge, leaf_max=0):
    t = otr.build_tree(pts, leaf_edge, leaf_max)
    coll = {l: otr.colleagues(t, l) for l in range(1, t.nlev + 1)}
    return t, coll, otr.v_lists(t, coll)
