"""Pins for the oracle's octree, Morton keys and interaction lists (CPU only).

Brute force on tiny trees, the paper's worked example (12-level tree for the
512-wavelength grid, Sec. 5.1), the paper's bound of 6^d - 3^d far-field boxes
(Sec. 4) and the pair-partition invariant.
"""
import os

import numpy as np
import pytest

import synth
from oracle import tree as tr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def test_morton_roundtrip_and_bit_order():
    rng = np.random.default_rng(0)
    u = rng.integers(0, 2 ** 21, size=(1000, 3))
    k = tr.morton_encode(u[:, 0], u[:, 1], u[:, 2])
    x, y, z = tr.morton_decode(k)
    assert np.array_equal(x, u[:, 0]) and np.array_equal(y, u[:, 1]) and np.array_equal(z, u[:, 2])
    # bit order by brute force on python integers
    for i in range(50):
        ref = 0
        for b in range(21):
            ref |= ((int(u[i, 0]) >> b) & 1) << (3 * b)
            ref |= ((int(u[i, 1]) >> b) & 1) << (3 * b + 1)
            ref |= ((int(u[i, 2]) >> b) & 1) << (3 * b + 2)
        assert int(k[i]) == ref


def test_level_count_rule():
    # smallest L with L >= log2(D0 / D(L)) + 1 (Sec. 3.1)
    for D0, e in [(4.0, 0.25), (3.999, 0.25), (4.0001, 0.25), (64.0, 0.25), (0.1, 0.25), (511.75, 0.25)]:
        L = tr.uniform_level_count(D0, e)
        assert e * 2 ** (L - 1) >= D0
        assert L == 1 or e * 2 ** (L - 2) < D0


def test_paper_grid_example():
    g = _golden("paper_grid512.txt")
    side = int(g["grid_side_points"])
    i = np.arange(side) * g["spacing"]
    X, Y = np.meshgrid(i, i, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)
    assert pts.shape[0] == int(g["n_points"])
    t = tr.build_tree(pts, g["leaf_edge"], 0, max_depth=14)
    assert t.nlev == int(g["levels"])
    leaves = t.levels[t.nlev]
    assert leaves.nbox == int(g["n_points"])
    assert np.all(leaves.end - leaves.begin == int(g["points_per_leaf"]))
    # levels of computation: levels with far-field (V) interactions; level 2 has none
    coll = {l: tr.colleagues(t, l) for l in (1, 2)}
    assert tr.v_list_level(t, coll, 2)[1].shape[0] == 0
    assert tr.v_list_level(t, coll, 3)[1].shape[0] > 0
    assert t.nlev - 3 + 1 == int(g["levels_of_computation"])


def _brute_keys(pts, x0, scale):
    keys = []
    for p in pts:
        u = [min(max(int(np.floor((p[a] - x0[a]) * scale)), 0), 2 ** 21 - 1) for a in range(3)]
        k = 0
        for b in range(21):
            for a in range(3):
                k |= ((u[a] >> b) & 1) << (3 * b + a)
        keys.append(k)
    return keys


@pytest.mark.parametrize("leaf_max", [0, 3])
def test_tree_brute_force(leaf_max):
    pts = synth.sphere(300, 1.3, seed=77)
    pts[5] = pts[6]                                   # a coincident pair
    t = tr.build_tree(pts, 0.25, leaf_max=leaf_max)
    bk = _brute_keys(pts, t.x0, t.scale)
    assert [int(v) for v in t.key_unsorted] == bk
    order = sorted(range(len(bk)), key=lambda i: (bk[i], i))
    assert list(t.perm) == order
    for l in range(1, t.nlev + 1):
        lev = t.levels[l]
        covered = np.zeros(t.n, dtype=int)
        for b in range(lev.nbox):
            seg = t.key[lev.begin[b]:lev.end[b]] >> np.uint64(3 * (22 - l))
            assert np.all(seg == lev.key[b])
            covered[lev.begin[b]:lev.end[b]] += 1
            if l > 1:
                p = lev.parent[b]
                par = t.levels[l - 1]
                assert par.begin[p] <= lev.begin[b] and lev.end[b] <= par.end[p]
                assert par.child_begin[p] <= b < par.child_end[p]
                assert not par.leaf[p]
            sp_ = pts[t.perm[lev.begin[b]:lev.end[b]]]
            assert np.all(np.abs(sp_ - lev.center[b]) <= 0.5 * lev.edge * (1 + 1e-9))
        if leaf_max == 0 or l == 1:
            assert np.all(covered == 1)
        # leaves at level l plus children of non-leaves partition the points
    # every point lies in exactly one leaf
    cnt = np.zeros(t.n, dtype=int)
    for l in range(1, t.nlev + 1):
        lev = t.levels[l]
        for b in np.nonzero(lev.leaf)[0]:
            cnt[lev.begin[b]:lev.end[b]] += 1
    assert np.all(cnt == 1)
    if leaf_max > 0:
        for l in range(1, t.nlev + 1):
            lev = t.levels[l]
            n = lev.end - lev.begin
            assert np.all(n[~lev.leaf] > leaf_max)
            assert np.all((n[lev.leaf] <= leaf_max) | (l == t.nlev))


def test_points_inside_their_leaf():
    pts = synth.sphere(2000, 2.0, seed=5)
    t = tr.build_tree(pts, 0.25)
    sp = pts[t.perm]
    lev = t.levels[t.nlev]
    for b in range(lev.nbox):
        d = np.abs(sp[lev.begin[b]:lev.end[b]] - lev.center[b])
        assert np.all(d <= 0.5 * lev.edge * (1 + 1e-9))


def _brute_colleagues_and_v(t, l):
    lev = t.levels[l]
    nb = lev.nbox
    coll = []
    V = []
    for b in range(nb):
        coll.append(sorted(c for c in range(nb) if np.max(np.abs(lev.ijk[c] - lev.ijk[b])) <= 1))
        if l >= 2:
            par = t.levels[l - 1]
            pb = lev.parent[b]
            vv = []
            for s in range(nb):
                near_par = np.max(np.abs(par.ijk[lev.parent[s]] - par.ijk[pb])) <= 1
                near = np.max(np.abs(lev.ijk[s] - lev.ijk[b])) <= 1
                if near_par and not near:
                    vv.append(s)
            V.append(vv)
    return coll, V


def test_lists_brute_force_uniform():
    pts = synth.sphere(1500, 1.0, seed=11)
    t = tr.build_tree(pts, 0.25)
    coll = {l: tr.colleagues(t, l) for l in range(1, t.nlev + 1)}
    V = tr.v_lists(t, coll)
    for l in range(1, t.nlev + 1):
        bc, bv = _brute_colleagues_and_v(t, l)
        for b in range(t.levels[l].nbox):
            assert sorted(int(c) for c in coll[l][b] if c >= 0) == bc[b]
            if l >= 2:
                offs, cols = V[l]
                assert list(cols[offs[b]:offs[b + 1]]) == bv[b]


def test_vlist_bound_from_paper():
    g = _golden("paper_vlist_bound.txt")
    # dense volume grid: interior boxes reach 6^3 - 3^3
    i = (np.arange(16) + 0.5) * 0.25
    X, Y, Z = np.meshgrid(i, i, i, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    t = tr.build_tree(pts, 0.25)
    coll = {l: tr.colleagues(t, l) for l in range(1, t.nlev + 1)}
    V = tr.v_lists(t, coll)
    sizes = np.diff(V[t.nlev][0])
    assert sizes.max() == int(g["volume_max"])
    # planar grid: 6^2 - 3^2
    X, Y = np.meshgrid(i, i, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)
    t = tr.build_tree(pts, 0.25)
    coll = {l: tr.colleagues(t, l) for l in range(1, t.nlev + 1)}
    V = tr.v_lists(t, coll)
    assert np.diff(V[t.nlev][0]).max() == int(g["planar_max"])


def _pair_cover(t, V, near):
    """Count, for every ordered pair (i, j), how many list entries cover it."""
    n = t.n
    C = np.zeros((n, n), dtype=np.int32)
    for l in range(2, t.nlev + 1):
        lev = t.levels[l]
        offs, cols = V[l]
        for b in range(lev.nbox):
            for s in cols[offs[b]:offs[b + 1]]:
                C[lev.begin[b]:lev.end[b], lev.begin[s]:lev.end[s]] += 1
    for (l, b), srcs in near.items():
        lev = t.levels[l]
        for (ls, s) in srcs:
            ss = t.levels[ls]
            C[lev.begin[b]:lev.end[b], ss.begin[s]:ss.end[s]] += 1
    return C


@pytest.mark.parametrize("leaf_max", [0, 4, 12])
def test_pair_partition_invariant(leaf_max):
    """Every ordered pair is covered exactly once: by a near list or one V pair."""
    if leaf_max == 0:
        pts = synth.sphere(900, 1.2, seed=21)
    else:
        pts = np.concatenate([synth.sphere(500, 1.5, seed=22),
                              synth.normal(23, 3 * 400).reshape(400, 3) * 0.05 + 0.7])
    t = tr.build_tree(pts, 0.25, leaf_max=leaf_max)
    coll = {l: tr.colleagues(t, l) for l in range(1, t.nlev + 1)}
    V = tr.v_lists(t, coll)
    if leaf_max == 0:
        offs, cols = tr.uniform_u_lists(t, coll)
        near = {(t.nlev, b): [(t.nlev, int(s)) for s in cols[offs[b]:offs[b + 1]]]
                for b in range(t.levels[t.nlev].nbox)}
    else:
        U, W, X = tr.near_lists_general(t, coll)
        near = tr.near_source_ranges(t, U, W, X)
        assert len({lv for (lv, _) in U}) > 1          # leaves on several levels
    C = _pair_cover(t, V, near)
    assert np.all(C == 1)


def test_adaptive_lists_definitions():
    pts = np.concatenate([synth.sphere(400, 1.5, seed=31),
                          synth.normal(32, 3 * 300).reshape(300, 3) * 0.05 - 0.6])
    t = tr.build_tree(pts, 0.25, leaf_max=5)
    coll = {l: tr.colleagues(t, l) for l in range(1, t.nlev + 1)}
    U, W, X = tr.near_lists_general(t, coll)
    allbox = [(l, b) for l in range(1, t.nlev + 1) for b in range(t.levels[l].nbox)]

    def adj(a, c):
        return tr._adjacent(a[0], t.levels[a[0]].ijk[a[1]], c[0], t.levels[c[0]].ijk[c[1]])

    def is_desc(d, a):
        while d[0] > a[0]:
            d = (d[0] - 1, int(t.levels[d[0]].parent[d[1]]))
        return d == a
    leaves = [x for x in allbox if t.levels[x[0]].leaf[x[1]]]
    for b in leaves:
        u_ref = sorted([c for c in leaves if adj(b, c)], key=lambda x: (x[0], int(t.levels[x[0]].key[x[1]])))
        assert U[b] == u_ref
        cols_b = [(b[0], int(c)) for c in coll[b[0]][b[1]] if c >= 0]
        w_ref = []
        for d in allbox:
            if d[0] <= b[0] or adj(b, d):
                continue
            par = (d[0] - 1, int(t.levels[d[0]].parent[d[1]]))
            if adj(b, par) and any(is_desc(d, c) for c in cols_b):
                w_ref.append(d)
        w_ref.sort(key=lambda x: (x[0], int(t.levels[x[0]].key[x[1]])))
        assert W[b] == w_ref
