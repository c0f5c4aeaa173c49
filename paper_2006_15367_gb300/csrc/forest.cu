// Batched plans over many geometries as one forest.
//
// With level-uniform trees every geometry's leaves have the same edge (the plan's leaf
// edge), so the boxes at the same height above the leaves have the same edge, truncation L,
// sampling grid, translation operators (Sec. 3.2.3) and interpolation maps (Sec. 3.2.2).
// The geometries' trees, built one by one, are merged height by height into one plan: its
// level l holds the boxes of every geometry at height nlev - l (geometry g's level l_g goes
// to l = l_g + (nlev - nlev_g)), with point, box, leaf and list indices shifted by the
// geometry's offsets.  Lists never cross geometries, so the merged plan computes exactly
// what the separate plans do, with one launch per stage and level for all geometries.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace mlfma {

namespace {

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

struct LevOffsets {
    int o[kMaxLev + 2];    // box offset of the geometry at each of its own levels
};

__global__ void k_copy_add(int* __restrict__ dst, const int* __restrict__ src, int64_t n, int add) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[i] + add;
}

// parent indices moved into the forest's parent level (add < 0: the parent level is not in the
// forest, every box is parentless)
__global__ void k_copy_parent(int* __restrict__ dst, const int* __restrict__ src, int64_t n, int add) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (add < 0 || src[i] < 0) ? -1 : src[i] + add;
}

__global__ void k_fill(int* __restrict__ dst, int64_t n, int v) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = v;
}

// M2L list entries (src K) << 32 | mask << 16 | base: the source moves by add_src boxes
__global__ void k_copy_m2l(unsigned long long* __restrict__ dst, const unsigned long long* __restrict__ src, int64_t n,
                           unsigned long long add_hi) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[i] + (add_hi << 32);
}

__global__ void k_copy_tiles(int2* __restrict__ dst, const int2* __restrict__ src, int64_t n, int addx) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = make_int2(src[i].x + addx, src[i].y);
}

// (level, box) pairs of the geometry -> forest (level + shift, box + offset of that level)
__global__ void k_copy_levbox(int* __restrict__ dlev, int* __restrict__ dbox, const int* __restrict__ slev,
                              const int* __restrict__ sbox, int64_t n, int shift, LevOffsets offs) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int l = slev[i];
    dlev[i] = l + shift;
    dbox[i] = sbox[i] + offs.o[l];
}

}  // namespace

bool forest_possible(const std::vector<Plan*>& subs) {
    if (subs.empty()) return false;
    for (const Plan* s : subs)
        if (s->leaf_max != 0 || s->leaf_edge != subs[0]->leaf_edge) return false;
    return true;
}

// Builds P (configured with the batch's n, k, digits, options and caller offsets sub_off)
// as the forest of the already built sub-plans; the sub-plans keep the operator arrays the
// forest points to, their own signatures and scratch are released.
void build_forest(Plan& P) {
    cudaStream_t s = P.stream;
    const int G = (int)P.subs.size();
    int Lmax = 0;
    for (const Plan* sp : P.subs) Lmax = std::max(Lmax, sp->nlev);
    std::vector<int> shift(G);
    int top = 0;
    for (int g = 0; g < G; ++g) {
        const Plan& sp = *P.subs[g];
        shift[g] = Lmax - sp.nlev;
        if (sp.top) top = top ? std::min(top, sp.top + shift[g]) : sp.top + shift[g];
    }
    P.nlev = Lmax;
    P.top = top;
    P.leaf_edge = P.subs[0]->leaf_edge;
    P.off343 = P.subs[0]->off343;
    const size_t cs = csize(P);

    // ---- points: sorted positions per geometry, perm to the caller's batch order
    P.pos = P.mem.make<double>(3 * (size_t)P.n);
    P.perm = P.mem.make<int>(P.n);
    std::vector<int64_t> ptoff(G + 1, 0);
    for (int g = 0; g < G; ++g) ptoff[g + 1] = ptoff[g] + P.subs[g]->n;
    for (int g = 0; g < G; ++g) {
        const Plan& sp = *P.subs[g];
        MLFMA_CUDA(cudaMemcpyAsync(P.pos + 3 * ptoff[g], sp.pos, 3 * sp.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        k_copy_add<<<nblk(sp.n, 256), 256, 0, s>>>(P.perm + ptoff[g], sp.perm, sp.n, (int)P.sub_off[g]);
        MLFMA_LAUNCH_CHECK();
    }

    // ---- which boxes enter the forest: a geometry's levels from one above its top down (the
    // parents that hold the M2L lists of its top level; their G stays zero), only its leaves
    // when it has no far field.  Coarser boxes would only feed interpolation nobody reads.
    auto inc = [&](int g, int l) {
        const Plan& sp = *P.subs[g];
        const int lg = l - shift[g];
        if (lg < 1 || lg > sp.nlev) return false;
        return sp.top ? lg >= sp.top - 1 : lg == sp.nlev;
    };
    // ---- box offsets per geometry and forest level
    std::vector<std::vector<int64_t>> boff(G, std::vector<int64_t>(Lmax + 2, 0));   // by forest level
    for (int l = 1; l <= Lmax; ++l) {
        int64_t acc = 0;
        for (int g = 0; g < G; ++g) {
            const int lg = l - shift[g];
            boff[g][l] = acc;
            if (inc(g, l)) acc += P.subs[g]->lev[lg].nbox;
        }
        P.lev[l].l = l;
        P.lev[l].nbox = acc;
    }
    auto own_offsets = [&](int g) {       // offsets indexed by the geometry's own level
        LevOffsets o;
        for (int i = 0; i < kMaxLev + 2; ++i) o.o[i] = 0;
        for (int lg = 1; lg <= P.subs[g]->nlev; ++lg) o.o[lg] = (int)boff[g][lg + shift[g]];
        return o;
    };

    // ---- per-level box arrays
    for (int l = 1; l <= Lmax; ++l) {
        TreeLevel& T = P.lev[l];
        const int64_t nb = T.nbox;
        T.key = P.mem.make<uint64_t>(std::max<int64_t>(nb, 1));
        T.begin = P.mem.make<int>(std::max<int64_t>(nb, 1));
        T.end = P.mem.make<int>(std::max<int64_t>(nb, 1));
        T.child_begin = P.mem.make<int>(std::max<int64_t>(nb, 1));
        T.child_end = P.mem.make<int>(std::max<int64_t>(nb, 1));
        T.parent = P.mem.make<int>(std::max<int64_t>(nb, 1));
        T.center = P.mem.make<double>(3 * std::max<int64_t>(nb, 1));
        T.m2l_off = P.mem.make<int>(nb + 1);
        int64_t n_small = 0, n_big = 0, n_tiles = 0, m2l_n = 0;
        for (int g = 0; g < G; ++g) {
            const int lg = l - shift[g];
            if (!inc(g, l)) continue;
            const TreeLevel& S = P.subs[g]->lev[lg];
            n_small += S.n_small_leaves;
            n_big += S.n_big_leaves;
            n_tiles += S.n_big_tiles;
            m2l_n += S.m2l_off ? S.m2l_n : 0;
            T.nleaf += S.nleaf;
            T.nv += S.nv;
        }
        T.n_small_leaves = n_small;
        T.n_big_leaves = n_big;
        T.n_big_tiles = n_tiles;
        T.m2l_n = m2l_n;
        T.small_leaves = P.mem.make<int>(std::max<int64_t>(n_small, 1));
        T.big_leaves = P.mem.make<int>(std::max<int64_t>(n_big, 1));
        T.big_tiles = P.mem.make<int2>(std::max<int64_t>(n_tiles, 1));
        T.m2l_src = P.mem.make<unsigned long long>(std::max<int64_t>(m2l_n, 1));
        int64_t o_small = 0, o_big = 0, o_tiles = 0, o_m2l = 0;
        for (int g = 0; g < G; ++g) {
            const int lg = l - shift[g];
            if (!inc(g, l)) continue;
            const Plan& sp = *P.subs[g];
            const TreeLevel& S = sp.lev[lg];
            const int64_t bo = boff[g][l];
            const int64_t nbs = S.nbox;
            if (nbs > 0) {
                MLFMA_CUDA(cudaMemcpyAsync(T.key + bo, S.key, nbs * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
                MLFMA_CUDA(cudaMemcpyAsync(T.center + 3 * bo, S.center, 3 * nbs * sizeof(double), cudaMemcpyDeviceToDevice, s));
                k_copy_add<<<nblk(nbs, 256), 256, 0, s>>>(T.begin + bo, S.begin, nbs, (int)ptoff[g]);
                k_copy_add<<<nblk(nbs, 256), 256, 0, s>>>(T.end + bo, S.end, nbs, (int)ptoff[g]);
                const int cadd = lg < sp.nlev ? (int)boff[g][l + 1] : 0;
                k_copy_add<<<nblk(nbs, 256), 256, 0, s>>>(T.child_begin + bo, S.child_begin, nbs, cadd);
                k_copy_add<<<nblk(nbs, 256), 256, 0, s>>>(T.child_end + bo, S.child_end, nbs, cadd);
                k_copy_parent<<<nblk(nbs, 256), 256, 0, s>>>(T.parent + bo, S.parent, nbs,
                                                             l > 1 && inc(g, l - 1) ? (int)boff[g][l - 1] : -1);
                MLFMA_LAUNCH_CHECK();
                // M2L lists of this level as parent level (sources are children at level l + 1)
                if (S.m2l_off && S.m2l_n > 0) {
                    k_copy_add<<<nblk(nbs, 256), 256, 0, s>>>(T.m2l_off + bo, S.m2l_off, nbs, (int)o_m2l);
                    const unsigned long long addhi =
                        (unsigned long long)(boff[g][l + 1] * (int64_t)sp.far[lg + 1].K);
                    k_copy_m2l<<<nblk(S.m2l_n, 256), 256, 0, s>>>(T.m2l_src + o_m2l, S.m2l_src, S.m2l_n, addhi);
                    o_m2l += S.m2l_n;
                } else {
                    k_fill<<<nblk(nbs, 256), 256, 0, s>>>(T.m2l_off + bo, nbs, (int)o_m2l);
                }
                MLFMA_LAUNCH_CHECK();
            }
            if (S.n_small_leaves > 0) {
                k_copy_add<<<nblk(S.n_small_leaves, 256), 256, 0, s>>>(T.small_leaves + o_small, S.small_leaves,
                                                                       S.n_small_leaves, (int)bo);
                o_small += S.n_small_leaves;
            }
            if (S.n_big_leaves > 0) {
                k_copy_add<<<nblk(S.n_big_leaves, 256), 256, 0, s>>>(T.big_leaves + o_big, S.big_leaves, S.n_big_leaves,
                                                                     (int)bo);
                o_big += S.n_big_leaves;
            }
            if (S.n_big_tiles > 0) {
                k_copy_tiles<<<nblk(S.n_big_tiles, 256), 256, 0, s>>>(T.big_tiles + o_tiles, S.big_tiles,
                                                                      S.n_big_tiles, (int)bo);
                o_tiles += S.n_big_tiles;
            }
            MLFMA_LAUNCH_CHECK();
        }
        k_fill<<<1, 1, 0, s>>>(T.m2l_off + nb, 1, (int)o_m2l);
        MLFMA_LAUNCH_CHECK();
    }

    // ---- parentless boxes per level (L2L adds nothing into them)
    for (int l = 2; l <= Lmax; ++l) {
        std::vector<int2> rg;
        int64_t cnt = 0;
        for (int g = 0; g < G; ++g) {
            const int lg = l - shift[g];
            if (!inc(g, l) || inc(g, l - 1)) continue;
            const int64_t nbs = P.subs[g]->lev[lg].nbox;
            if (nbs > 0) {
                rg.push_back(make_int2((int)boff[g][l], (int)nbs));
                cnt += nbs;
            }
        }
        TreeLevel& T = P.lev[l];
        T.n_orphan_ranges = (int)rg.size();
        T.n_orphans = cnt;
        if (!rg.empty()) {
            T.orphans = P.mem.make<int2>(rg.size());
            MLFMA_CUDA(cudaMemcpyAsync(T.orphans, rg.data(), rg.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
            MLFMA_CUDA(cudaStreamSynchronize(s));            // rg is a host temporary
        }
    }

    // ---- leaf table, near lists, P2P work
    int64_t nleaf = 0, nnear = 0, n_small = 0, n_small32 = 0, n_tiles = 0;
    for (const Plan* sp : P.subs) {
        nleaf += sp->nleaf_total;
        nnear += sp->nnear;
        n_small += sp->n_small;
        n_small32 += sp->n_small32;
        n_tiles += sp->n_tiles;
        P.near_pairs += sp->near_pairs;
    }
    P.nleaf_total = nleaf;
    P.nnear = nnear;
    P.n_small = n_small;
    P.n_small32 = n_small32;
    P.n_tiles = n_tiles;
    P.leaf_level = P.mem.make<int>(std::max<int64_t>(nleaf, 1));
    P.leaf_box = P.mem.make<int>(std::max<int64_t>(nleaf, 1));
    P.near_off = P.mem.make<int>(nleaf + 1);
    P.near_lev = P.mem.make<int>(std::max<int64_t>(nnear, 1));
    P.near_box = P.mem.make<int>(std::max<int64_t>(nnear, 1));
    P.p2p_small = P.mem.make<int>(std::max<int64_t>(n_small, 1));
    P.p2p_tiles = P.mem.make<int2>(std::max<int64_t>(n_tiles, 1));
    // small leaves: every geometry's leaves of up to 32 points first, then those of 33 and more
    int64_t o_leaf = 0, o_near = 0, o_small = 0, o_mid = n_small32, o_tiles = 0;
    for (int g = 0; g < G; ++g) {
        const Plan& sp = *P.subs[g];
        const LevOffsets offs = own_offsets(g);
        if (sp.nleaf_total > 0) {
            k_copy_levbox<<<nblk(sp.nleaf_total, 256), 256, 0, s>>>(P.leaf_level + o_leaf, P.leaf_box + o_leaf,
                                                                    sp.leaf_level, sp.leaf_box, sp.nleaf_total, shift[g],
                                                                    offs);
            k_copy_add<<<nblk(sp.nleaf_total, 256), 256, 0, s>>>(P.near_off + o_leaf, sp.near_off, sp.nleaf_total,
                                                                 (int)o_near);
        }
        if (sp.nnear > 0)
            k_copy_levbox<<<nblk(sp.nnear, 256), 256, 0, s>>>(P.near_lev + o_near, P.near_box + o_near, sp.near_lev,
                                                              sp.near_box, sp.nnear, shift[g], offs);
        if (sp.n_small32 > 0)
            k_copy_add<<<nblk(sp.n_small32, 256), 256, 0, s>>>(P.p2p_small + o_small, sp.p2p_small, sp.n_small32,
                                                               (int)o_leaf);
        if (sp.n_small > sp.n_small32)
            k_copy_add<<<nblk(sp.n_small - sp.n_small32, 256), 256, 0, s>>>(
                P.p2p_small + o_mid, sp.p2p_small + sp.n_small32, sp.n_small - sp.n_small32, (int)o_leaf);
        if (sp.n_tiles > 0)
            k_copy_tiles<<<nblk(sp.n_tiles, 256), 256, 0, s>>>(P.p2p_tiles + o_tiles, sp.p2p_tiles, sp.n_tiles,
                                                               (int)o_leaf);
        MLFMA_LAUNCH_CHECK();
        o_leaf += sp.nleaf_total;
        o_near += sp.nnear;
        o_small += sp.n_small32;
        o_mid += sp.n_small - sp.n_small32;
        o_tiles += sp.n_tiles;
    }
    k_fill<<<1, 1, 0, s>>>(P.near_off + nleaf, 1, (int)nnear);
    MLFMA_LAUNCH_CHECK();

    // ---- far levels: operators from a geometry whose far range covers the level, merged
    // signatures and spectral scratch
    if (P.top) {
        for (int l = P.top; l <= Lmax; ++l) {
            int rep = -1;
            for (int g = 0; g < G && rep < 0; ++g) {
                const Plan& sp = *P.subs[g];
                const int lg = l - shift[g];
                if (sp.top && lg >= sp.top && lg <= sp.nlev) rep = g;
            }
            if (rep < 0) fail(MLFMA_ERR_UNSUPPORTED, "forest level %d has no far-field geometry", l);
            const Plan& sp = *P.subs[rep];
            const FarLevel& src = sp.far[l - shift[rep]];
            for (int g = 0; g < G; ++g) {         // every geometry with far level l must agree
                const Plan& sq = *P.subs[g];
                const int lg = l - shift[g];
                if (sq.top && lg >= sq.top && lg <= sq.nlev && sq.far[lg].L != src.L)
                    fail(MLFMA_ERR_UNSUPPORTED, "geometries disagree on the truncation at forest level %d", l);
            }
            FarLevel& F = P.far[l];
            F = src;                               // grid, operators, interpolation (pointers shared)
            F.X = F.Y = nullptr;
            F.F = P.mem.get((size_t)P.lev[l].nbox * F.K * cs);
            F.G = P.mem.get((size_t)P.lev[l].nbox * F.K * cs);
            // the roots of shallower geometries have no parent, so M2L never writes their G:
            // it stays zero (L2L reads it as a parent)
            MLFMA_CUDA(cudaMemsetAsync(F.G, 0, (size_t)P.lev[l].nbox * F.K * cs, s));
            if (l > P.top && (int64_t)P.lev[l].nbox * F.K >= ((int64_t)1 << 32))
                fail(MLFMA_ERR_UNSUPPORTED, "forest level %d holds %lld samples, beyond 32-bit offsets", l,
                     (long long)((int64_t)P.lev[l].nbox * F.K));
        }
        // interpolation pairs (l, l + 1) need the parent-level maps of a geometry whose far
        // range covers both levels: the representative of l (its range reaches the leaves)
        size_t xs = 0, ys = 0;
        for (int l = P.top; l < Lmax; ++l) {
            const FarLevel& Pf = P.far[l];
            const FarLevel& Ch = P.far[l + 1];
            if (!Pf.At) fail(MLFMA_ERR_UNSUPPORTED, "forest level %d lacks interpolation maps", l);
            const size_t nb = (size_t)P.lev[l + 1].nbox;
            xs = std::max(xs, nb * (2 * Ch.L + 1) * Ch.nth);
            ys = std::max(ys, nb * (2 * Ch.L + 1) * Pf.nth);
        }
        if (xs) {
            void* X = P.mem.get(xs * cs);
            void* Y = P.mem.get(ys * cs);
            for (int l = P.top; l <= Lmax; ++l) { P.far[l].X = X; P.far[l].Y = Y; }
        }
    }
    P.dev_err = P.mem.make<int>(1);
    MLFMA_CUDA(cudaMemsetAsync(P.dev_err, 0, sizeof(int), s));
    P.near_dump = P.mem.get(P.n * cs);
    MLFMA_CUDA(cudaStreamSynchronize(s));

    // ---- the sub-plans keep only the operator arrays the forest points to
    std::vector<const void*> keep;
    for (int l = P.top ? P.top : 1; P.top && l <= Lmax; ++l) {
        const FarLevel& F = P.far[l];
        const void* used[] = {F.x,    F.wgl,  F.dirs, F.tw,   F.T,    F.T1,   F.At,   F.Bt, F.AtE,
                              F.AtD,  F.BtE,  F.BtD,  F.AtTc, F.BtTc, F.DmTc, F.DlTc, F.Soct, F.Sz, F.Sxy};
        for (const void* q : used)
            if (q) keep.push_back(q);
    }
    keep.push_back(P.off343);
    for (Plan* sp : P.subs) {
        std::vector<void*> drop;
        for (const auto& a : sp->mem.live)
            if (std::find(keep.begin(), keep.end(), (const void*)a.first) == keep.end()) drop.push_back(a.first);
        for (void* q : drop) sp->mem.drop(q);
        sp->dev_err = nullptr;
        sp->qs = sp->phis = sp->near_dump = sp->grads = nullptr;
        sp->nrhs_cap = sp->nrhs_grad = 0;
    }
}

}  // namespace mlfma
