"""Octree, Morton keys and interaction lists of the oracle (plain numpy, FP64 + integers).

TEST INFRASTRUCTURE (CPU oracle).  Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import it.

Follows the paper's tree rules:

* Sec. 2 (FMM paragraph): recursive subdivision of the domain into cubes until a
  box size or a particle count is reached; each point is mapped to its box.
* Sec. 3.1: the level count is the smallest integer L with L >= log2(D0/D(L)) + 1
  (D0 = edge of the bounding cube, D(L) = leaf edge) and every point gets a
  Morton-Z key; points are ordered along the Z curve.
* Sec. 2 (near/far rule): two boxes of one level are near if they share a face,
  edge or node; far (the V list) if they are not near but their parents are.
  Near-field sums happen only at the leaves.

Readings where the paper is silent:

* root cube centred on the bounding-box centre; the uniform tree (leaf_max == 0)
  has leaf edge ``leaf_edge`` and root edge leaf_edge * 2^(L-1); the adaptive tree
  (leaf_max > 0) has root edge D0 (1 + 2^-30) and splits a box while it holds more
  than leaf_max points, down to the deepest level whose edge is still >= leaf_edge
  (far-field cutoff) and at most ``max_depth``;
* quantisation u = floor((x - x0) * (2^21 / a_1)) in FP64 (subtract, then multiply),
  clamped to [0, 2^21 - 1]; key bit 3b+0 = bit b of u_x, 3b+1 of u_y, 3b+2 of u_z;
  the box key of a point at level l is key >> 3 (22 - l) (root = level 1);
* points are ordered by (key, original index);
* adaptive lists are the usual U/V/W/X lists; U, W and X interactions are summed
  directly (near field); lists are ordered by source box (level, key).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BITS = 21                       # bits per axis; keys use 63 bits
MAXLEV = BITS + 1               # level 22 resolves single quantisation cells


def spread_bits(u: np.ndarray) -> np.ndarray:
    """Insert two zero bits between the 21 low bits of u (bit b -> bit 3b)."""
    u = u.astype(np.uint64)
    out = np.zeros_like(u)
    for b in range(BITS):
        out |= ((u >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b)
    return out


def compact_bits(k: np.ndarray) -> np.ndarray:
    """Inverse of spread_bits: gather bits 0, 3, 6, ... into bits 0, 1, 2, ..."""
    k = k.astype(np.uint64)
    out = np.zeros_like(k)
    for b in range(BITS):
        out |= ((k >> np.uint64(3 * b)) & np.uint64(1)) << np.uint64(b)
    return out


def morton_encode(ux, uy, uz) -> np.ndarray:
    return spread_bits(np.asarray(ux)) | (spread_bits(np.asarray(uy)) << np.uint64(1)) | \
        (spread_bits(np.asarray(uz)) << np.uint64(2))


def morton_decode(key: np.ndarray):
    key = np.asarray(key, dtype=np.uint64)
    return (compact_bits(key).astype(np.int64), compact_bits(key >> np.uint64(1)).astype(np.int64),
            compact_bits(key >> np.uint64(2)).astype(np.int64))


@dataclass
class Level:
    l: int
    edge: float
    key: np.ndarray            # uint64 [nb], ascending
    begin: np.ndarray          # int64 [nb] first sorted point
    end: np.ndarray            # int64 [nb] one past last
    parent: np.ndarray         # int64 [nb] index at level l-1 (-1 at the root)
    child_begin: np.ndarray    # int64 [nb] first child at level l+1
    child_end: np.ndarray      # int64 [nb]
    leaf: np.ndarray           # bool [nb]
    ijk: np.ndarray            # int64 [nb, 3]
    center: np.ndarray         # float64 [nb, 3]

    @property
    def nbox(self) -> int:
        return int(self.key.shape[0])


@dataclass
class Tree:
    n: int
    leaf_edge: float
    leaf_max: int
    max_depth: int
    lo: np.ndarray
    hi: np.ndarray
    D0: float
    root_center: np.ndarray
    a1: float
    x0: np.ndarray
    scale: float
    nlev: int
    key_unsorted: np.ndarray
    perm: np.ndarray           # sorted position -> original index
    key: np.ndarray            # sorted keys
    levels: list = field(default_factory=list)   # levels[l] for l = 1..nlev (levels[0] unused)


def uniform_level_count(D0: float, leaf_edge: float) -> int:
    """Smallest L with leaf_edge * 2^(L-1) >= D0, i.e. L >= log2(D0/leaf_edge) + 1 (Sec. 3.1)."""
    L = 1
    while leaf_edge * (2.0 ** (L - 1)) < D0:
        L += 1
    return L


def build_tree(points: np.ndarray, leaf_edge: float, leaf_max: int = 0, max_depth: int = 12) -> Tree:
    pts = np.asarray(points, dtype=np.float64)
    if pts.ndim != 2 or pts.shape[1] != 3 or pts.shape[0] < 1:
        raise ValueError("points must be [n, 3] with n >= 1")
    if not np.all(np.isfinite(pts)):
        raise ValueError("non-finite coordinates")
    n = pts.shape[0]
    lo = pts.min(axis=0)
    hi = pts.max(axis=0)
    D0 = float(np.max(hi - lo))
    c = 0.5 * (lo + hi)
    if leaf_max == 0:
        L = uniform_level_count(D0, leaf_edge)
        if L > max_depth:
            raise ValueError(f"uniform tree needs {L} levels > max_depth {max_depth}")
        a1 = leaf_edge * (2.0 ** (L - 1))
        nlev = L
    else:
        a1 = D0 * (1.0 + 2.0 ** -30) if D0 > 0.0 else leaf_edge
        cutoff = 1
        while cutoff < MAXLEV and a1 / (2.0 ** cutoff) >= leaf_edge:
            cutoff += 1
        nlev = min(max_depth, cutoff)
    x0 = c - 0.5 * a1
    scale = (2.0 ** BITS) / a1
    u = np.floor((pts - x0) * scale)
    u = np.clip(u, 0, 2 ** BITS - 1).astype(np.int64)
    key_un = morton_encode(u[:, 0], u[:, 1], u[:, 2])
    perm = np.lexsort((np.arange(n), key_un))      # stable: by (key, original index)
    key = key_un[perm]
    tree = Tree(n=n, leaf_edge=leaf_edge, leaf_max=leaf_max, max_depth=max_depth, lo=lo, hi=hi, D0=D0,
                root_center=c, a1=a1, x0=x0, scale=scale, nlev=nlev, key_unsorted=key_un, perm=perm,
                key=key, levels=[None])

    # Level by level: boxes at level l are the distinct level keys among points whose
    # level-(l-1) box splits.  ``active`` marks those points; ``seg_start`` marks the
    # first point of each split parent, so runs never cross parent boundaries.
    active = np.ones(n, dtype=bool)
    seg_start = np.zeros(n, dtype=bool)
    seg_start[0] = True
    pbox = np.full(n, -1, dtype=np.int64)        # box of each point at the previous level
    for l in range(1, nlev + 1):
        shift = np.uint64(3 * (MAXLEV - l))
        lk = key >> shift
        newrun = seg_start.copy()
        newrun[1:] |= lk[1:] != lk[:-1]
        first = active & newrun
        bb = np.nonzero(first)[0].astype(np.int64)
        # a run ends where the next run starts or where the active stretch ends
        is_end = np.zeros(n, dtype=bool)
        is_end[:-1] = active[:-1] & (newrun[1:] | ~active[1:])
        is_end[-1] = active[-1]
        ee = np.nonzero(is_end)[0].astype(np.int64) + 1
        kk = lk[bb].astype(np.uint64)
        pp = pbox[bb]
        cnt = ee - bb
        if leaf_max == 0:
            split = np.full(kk.shape[0], l < nlev)
        else:
            split = (cnt > leaf_max) & (l < nlev)
        edge = a1 / (2.0 ** (l - 1))
        ix, iy, iz = morton_decode(kk)
        ijk = np.stack([ix, iy, iz], axis=1)
        center = x0[None, :] + (ijk.astype(np.float64) + 0.5) * edge
        lev = Level(l=l, edge=edge, key=kk, begin=bb, end=ee, parent=pp,
                    child_begin=np.zeros(kk.shape[0], dtype=np.int64),
                    child_end=np.zeros(kk.shape[0], dtype=np.int64), leaf=~split, ijk=ijk, center=center)
        tree.levels.append(lev)
        # points of split boxes stay active; each split box starts a new segment
        box_of_pt = np.full(n, -1, dtype=np.int64)
        box_of_pt[bb] = np.arange(bb.shape[0])
        box_of_pt = np.maximum.accumulate(box_of_pt)
        active = active & split[np.maximum(box_of_pt, 0)]
        seg_start = np.zeros(n, dtype=bool)
        seg_start[bb[split]] = True
        pbox = box_of_pt
    # child ranges
    for l in range(1, nlev):
        lev, nxt = tree.levels[l], tree.levels[l + 1]
        if nxt.nbox:
            par = nxt.parent
            first = np.concatenate([[True], par[1:] != par[:-1]])
            last = np.concatenate([par[1:] != par[:-1], [True]])
            lev.child_begin[par[first]] = np.nonzero(first)[0]
            lev.child_end[par[last]] = np.nonzero(last)[0] + 1
    return tree


# ---------------------------------------------------------------------------
# Lists
# ---------------------------------------------------------------------------
_OFF27 = np.array([(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)],
                  dtype=np.int64)


def colleagues(tree: Tree, l: int) -> np.ndarray:
    """[nb, 27] same-level boxes with max |d ijk| <= 1 (incl. self); -1 where absent.

    Slot s holds offset (dx, dy, dz) = _OFF27[s] (dx fastest).
    """
    lev = tree.levels[l]
    nb = lev.nbox
    out = np.full((nb, 27), -1, dtype=np.int64)
    if nb == 0:
        return out
    side = 1 << (l - 1)
    for s, d in enumerate(_OFF27):
        nij = lev.ijk + d[None, :]
        ok = np.all((nij >= 0) & (nij < side), axis=1)
        nk = morton_encode(np.where(ok, nij[:, 0], 0), np.where(ok, nij[:, 1], 0), np.where(ok, nij[:, 2], 0))
        pos = np.searchsorted(lev.key, nk)
        pos_c = np.minimum(pos, nb - 1)
        found = ok & (lev.key[pos_c] == nk)
        out[found, s] = pos_c[found]
    return out


def _to_csr(rows: np.ndarray, cols: np.ndarray, nrows: int):
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    offs = np.zeros(nrows + 1, dtype=np.int64)
    np.add.at(offs, rows + 1, 1)
    return np.cumsum(offs), cols


def v_list_level(tree: Tree, coll: dict, l: int):
    """V lists of level l >= 2 as CSR (offsets [nb+1], source box indices at level l).

    V(b) = children of the colleagues of parent(b) that are not adjacent to b (Sec. 2).
    """
    lev, par = tree.levels[l], tree.levels[l - 1]
    nb = lev.nbox
    pc = coll[l - 1][lev.parent]                       # [nb, 27] parent colleagues
    b_idx = np.repeat(np.arange(nb), 27)
    q = pc.reshape(-1)
    ok = q >= 0
    b_idx, q = b_idx[ok], q[ok]
    cb, ce = par.child_begin[q], par.child_end[q]
    cnt = ce - cb
    rows = np.repeat(b_idx, cnt)
    starts = np.repeat(cb, cnt)
    within = np.arange(rows.shape[0]) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    src = starts + within
    d = np.abs(lev.ijk[src] - lev.ijk[rows]).max(axis=1)
    far = d >= 2
    return _to_csr(rows[far], src[far], nb)


def v_lists(tree: Tree, coll: dict) -> dict:
    """V lists of every level l >= 2 (dict level -> CSR)."""
    return {l: v_list_level(tree, coll, l) for l in range(2, tree.nlev + 1)}


def _adjacent(la: int, ia: np.ndarray, lb: int, ib: np.ndarray) -> bool:
    """Closed cubes of boxes (la, ia) and (lb, ib) touch or overlap."""
    if la > lb:
        la, ia, lb, ib = lb, ib, la, ia
    s = lb - la
    lo = ia * (1 << s)
    hi = (ia + 1) * (1 << s)           # exclusive upper cell at level lb
    return bool(np.all(ib >= lo - 1) and np.all(ib <= hi))


def near_lists_general(tree: Tree, coll: dict):
    """U, W and X lists of the adaptive FMM, by plain per-box loops.

    U(b), b leaf: leaves adjacent to b at any level (incl. b).
    W(b), b leaf: descendants of b's colleagues that are not adjacent to b but
                  whose parent is adjacent to b.
    X(b), any box: leaves c with b in W(c).
    Returns dicts keyed by (level, box) -> list of (level, box), each sorted by (level, key).
    """
    U, W, X = {}, {}, {}
    for l in range(1, tree.nlev + 1):
        lev = tree.levels[l]
        for b in range(lev.nbox):
            X.setdefault((l, b), [])
    for l in range(1, tree.nlev + 1):
        lev = tree.levels[l]
        for b in range(lev.nbox):
            if not lev.leaf[b]:
                continue
            ib = lev.ijk[b]
            u, w = [], []
            # coarser leaves adjacent to b: colleagues of ancestors
            anc = b
            for la in range(l - 1, 0, -1):
                anc = tree.levels[la + 1].parent[anc]
                for q in coll[la][anc]:
                    if q >= 0 and tree.levels[la].leaf[q] and q != anc and \
                            _adjacent(la, tree.levels[la].ijk[q], l, ib):
                        u.append((la, int(q)))
            # same level and finer: walk down from colleagues
            stack = [(l, int(q)) for q in coll[l][b] if q >= 0]
            while stack:
                lq, q = stack.pop()
                levq = tree.levels[lq]
                if lq == l or _adjacent(lq, levq.ijk[q], l, ib):
                    if levq.leaf[q]:
                        u.append((lq, q))
                    else:
                        for c in range(levq.child_begin[q], levq.child_end[q]):
                            stack.append((lq + 1, int(c)))
                else:
                    w.append((lq, q))
            U[(l, b)] = sorted(set(u), key=lambda t: (t[0], int(tree.levels[t[0]].key[t[1]])))
            W[(l, b)] = sorted(set(w), key=lambda t: (t[0], int(tree.levels[t[0]].key[t[1]])))
            for (lw, wb) in W[(l, b)]:
                X[(lw, wb)].append((l, b))
    for kx in X:
        X[kx] = sorted(set(X[kx]), key=lambda t: (t[0], int(tree.levels[t[0]].key[t[1]])))
    return U, W, X


def near_source_ranges(tree: Tree, U, W, X):
    """Per leaf (level, box): sorted list of source boxes summed directly.

    Sources are U(b) and W(b) and X(a) for every ancestor-or-self a of b.
    """
    out = {}
    for (l, b), ul in U.items():
        src = list(ul) + list(W[(l, b)])
        a, la = b, l
        while la >= 1:
            src += X[(la, a)]
            if la == 1:
                break
            a = tree.levels[la].parent[a]
            la -= 1
        out[(l, b)] = sorted(set(src), key=lambda t: (t[0], int(tree.levels[t[0]].key[t[1]])))
    return out


def uniform_u_lists(tree: Tree, coll: dict):
    """U lists of a level-uniform tree: the colleagues of each leaf (all leaves), CSR."""
    l = tree.nlev
    c = coll[l]
    nb = c.shape[0]
    rows = np.repeat(np.arange(nb), 27)
    cols = c.reshape(-1)
    ok = cols >= 0
    return _to_csr(rows[ok], cols[ok], nb)
