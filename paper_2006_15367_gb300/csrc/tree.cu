// Octree construction and interaction lists on the device.
//
// Sec. 3.1: bounding cube, level count (smallest L with L >= log2(D0/D(L)) + 1),
// Morton-Z keys and a sort along the Z curve; Sec. 2: boxes of one level are near
// when they share a face, edge or node, far (V list) when not near but their
// parents are; near-field sums only at the leaves.  Adaptive trees use the usual
// U/V/W/X lists with U, W and X summed directly.  All integer work, bit-exact.
#include <cstdio>
#include <cstring>

#include <set>
#include <unordered_map>

#include "common.cuh"

namespace mlfma {

// ============================================================== scan (int32, exclusive)
constexpr int kScanTile = 1024;   // 256 threads x 4 items

int64_t scan_tmp_ints(int64_t n) { return (n + kScanTile - 1) / kScanTile + 2; }

__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// exclusive scan of one value per thread over a 256-thread block; returns the block total in *total
__device__ int block_excl_scan256(int v, int* total) {
    __shared__ int wsum[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = warp_incl_scan(v);
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int s = lane < 8 ? wsum[lane] : 0;
        s = warp_incl_scan(s);
        if (lane < 8) wsum[lane] = s;
    }
    __syncthreads();
    int off = warp > 0 ? wsum[warp - 1] : 0;
    *total = wsum[7];
    __syncthreads();
    return off + inc - v;
}

__global__ void k_scan_reduce(const int* __restrict__ in, int64_t n, int* __restrict__ sums) {
    int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * 4;
    int s = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e)
        if (base + e < n) s += in[base + e];
    int total;
    block_excl_scan256(s, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_scan_sums(int* sums, int nb) {
    // single block of 256 threads; exclusive scan of sums[0..nb), total -> sums[nb]
    int carry = 0;
    for (int base = 0; base < nb; base += 256) {
        int i = base + threadIdx.x;
        int v = i < nb ? sums[i] : 0;
        int total;
        int ex = block_excl_scan256(v, &total);
        if (i < nb) sums[i] = carry + ex;
        carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void k_scan_final(const int* __restrict__ in, int* __restrict__ out, int64_t n, const int* __restrict__ sums) {
    int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * 4;
    int v[4];
    int s = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        v[e] = base + e < n ? in[base + e] : 0;
        s += v[e];
    }
    int total;
    int ex = block_excl_scan256(s, &total) + sums[blockIdx.x];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        if (base + e < n) out[base + e] = ex;
        ex += v[e];
    }
}

int scan_exclusive(const int* in, int* out, int64_t n, int* tmp, cudaStream_t s) {
    if (n <= 0) return 0;
    int nb = (int)((n + kScanTile - 1) / kScanTile);
    k_scan_reduce<<<nb, 256, 0, s>>>(in, n, tmp);
    MLFMA_LAUNCH_CHECK();
    k_scan_sums<<<1, 256, 0, s>>>(tmp, nb);
    MLFMA_LAUNCH_CHECK();
    k_scan_final<<<nb, 256, 0, s>>>(in, out, n, tmp);
    MLFMA_LAUNCH_CHECK();
    int total = 0;
    MLFMA_CUDA(cudaMemcpyAsync(&total, tmp + nb, sizeof(int), cudaMemcpyDeviceToHost, s));
    MLFMA_CUDA(cudaStreamSynchronize(s));
    return total;
}

// ============================================================== bounding box
__global__ void k_bbox_partial(const double* __restrict__ p, int64_t n, double* __restrict__ part, int* bad) {
    __shared__ double smin[3][256], smax[3][256];
    double mn[3] = {1e308, 1e308, 1e308}, mx[3] = {-1e308, -1e308, -1e308};
    bool nonfinite = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double v = p[3 * i + a];
            if (!isfinite(v)) nonfinite = true;
            mn[a] = fmin(mn[a], v);
            mx[a] = fmax(mx[a], v);
        }
    }
    if (nonfinite) atomicExch(bad, 1);
#pragma unroll
    for (int a = 0; a < 3; ++a) { smin[a][threadIdx.x] = mn[a]; smax[a][threadIdx.x] = mx[a]; }
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                smin[a][threadIdx.x] = fmin(smin[a][threadIdx.x], smin[a][threadIdx.x + s]);
                smax[a][threadIdx.x] = fmax(smax[a][threadIdx.x], smax[a][threadIdx.x + s]);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int a = 0; a < 3; ++a) { part[6 * blockIdx.x + a] = smin[a][0]; part[6 * blockIdx.x + 3 + a] = smax[a][0]; }
}

// ============================================================== Morton keys
__host__ __device__ inline uint64_t spread3(uint64_t u) {
    u &= 0x1fffffull;
    u = (u | (u << 32)) & 0x1f00000000ffffull;
    u = (u | (u << 16)) & 0x1f0000ff0000ffull;
    u = (u | (u << 8)) & 0x100f00f00f00f00full;
    u = (u | (u << 4)) & 0x10c30c30c30c30c3ull;
    u = (u | (u << 2)) & 0x1249249249249249ull;
    return u;
}
__host__ __device__ inline uint64_t compact3(uint64_t u) {
    u &= 0x1249249249249249ull;
    u = (u | (u >> 2)) & 0x10c30c30c30c30c3ull;
    u = (u | (u >> 4)) & 0x100f00f00f00f00full;
    u = (u | (u >> 8)) & 0x1f0000ff0000ffull;
    u = (u | (u >> 16)) & 0x1f00000000ffffull;
    u = (u | (u >> 32)) & 0x1fffffull;
    return u;
}
__host__ __device__ inline uint64_t morton(int x, int y, int z) {
    return spread3((uint64_t)x) | (spread3((uint64_t)y) << 1) | (spread3((uint64_t)z) << 2);
}

// u = floor((x - x0) * scale) in FP64 without contraction, clamped to [0, 2^21 - 1]
__global__ void k_keys(const double* __restrict__ p, int64_t n, double x0, double y0, double z0, double scale,
                       uint64_t* __restrict__ key, int* __restrict__ idx) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double o[3] = {x0, y0, z0};
    int u[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double v = floor(__dmul_rn(__dsub_rn(p[3 * i + a], o[a]), scale));
        v = fmin(fmax(v, 0.0), (double)((1 << kBits) - 1));
        u[a] = (int)v;
    }
    key[i] = morton(u[0], u[1], u[2]);
    idx[i] = (int)i;
}

// ============================================================== stable LSD radix sort (8-bit digits)
constexpr int kRadixTile = 1024;

__global__ void k_radix_hist(const uint64_t* __restrict__ keys, int64_t n, int shift, int* __restrict__ counts, int nblocks) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int e = threadIdx.x; e < kRadixTile; e += 256) {
        int64_t i = base + e;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255], 1);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_radix_scatter(const uint64_t* __restrict__ kin, const int* __restrict__ vin, uint64_t* __restrict__ kout,
                                int* __restrict__ vout, int64_t n, int shift, const int* __restrict__ offs, int nblocks) {
    __shared__ int off[256];
    __shared__ int wh[8][257];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    off[threadIdx.x] = offs[(int64_t)threadIdx.x * nblocks + blockIdx.x];
    int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int r = 0; r < kRadixTile / 256; ++r) {
        for (int w = 0; w < 8; ++w) wh[w][threadIdx.x] = 0;
        __syncthreads();
        int64_t i = base + r * 256 + warp * 32 + lane;
        bool valid = i < n;
        uint64_t k = valid ? kin[i] : 0;
        int v = valid ? vin[i] : 0;
        int d = valid ? (int)((k >> shift) & 255) : 256;
        unsigned mask = __match_any_sync(0xffffffffu, d);
        int rank = __popc(mask & ((1u << lane) - 1u));
        if (valid && lane == __ffs(mask) - 1) wh[warp][d] = __popc(mask);
        __syncthreads();
        int run = 0;
        for (int w = 0; w < 8; ++w) { int c = wh[w][threadIdx.x]; wh[w][threadIdx.x] = run; run += c; }
        __syncthreads();
        if (valid) {
            int pos = off[d] + wh[warp][d] + rank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
        off[threadIdx.x] += run;
        __syncthreads();
    }
}

// ============================================================== levels
__global__ void k_level_flags(const uint64_t* __restrict__ key, int64_t n, int shift, const uint8_t* __restrict__ active,
                              const uint8_t* __restrict__ seg_start, int* __restrict__ flag) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool nr = seg_start[i] || i == 0 || (key[i] >> shift) != (key[i - 1] >> shift);
    flag[i] = (active[i] && nr) ? 1 : 0;
}

__global__ void k_level_fill(const uint64_t* __restrict__ key, int64_t n, int shift, const uint8_t* __restrict__ active,
                             const uint8_t* __restrict__ seg_start, const int* __restrict__ flag, const int* __restrict__ scan,
                             const int* __restrict__ pbox_prev, uint64_t* __restrict__ lkey, int* __restrict__ begin,
                             int* __restrict__ end, int* __restrict__ parent, int* __restrict__ box_of_pt) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || !active[i]) return;
    int box = scan[i] + flag[i] - 1;
    box_of_pt[i] = box;
    uint64_t lk = key[i] >> shift;
    if (flag[i]) {
        lkey[box] = lk;
        begin[box] = (int)i;
        parent[box] = pbox_prev[i];
    }
    bool is_end = (i == n - 1) || !active[i + 1] || seg_start[i + 1] || (key[i + 1] >> shift) != lk;
    if (is_end) end[box] = (int)(i + 1);
}

__global__ void k_level_boxes(int64_t nb, int l, int nlev, int leaf_max, double edge, double x0, double y0, double z0,
                              const uint64_t* __restrict__ lkey, const int* __restrict__ begin, const int* __restrict__ end,
                              uint8_t* __restrict__ leaf, int* __restrict__ ijk, double* __restrict__ center) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int cnt = end[b] - begin[b];
    bool split = (l < nlev) && (leaf_max == 0 || cnt > leaf_max);
    leaf[b] = split ? 0 : 1;
    uint64_t k = lkey[b];
    int c[3] = {(int)compact3(k), (int)compact3(k >> 1), (int)compact3(k >> 2)};
    const double o[3] = {x0, y0, z0};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        ijk[3 * b + a] = c[a];
        center[3 * b + a] = __dadd_rn(o[a], __dmul_rn((double)c[a] + 0.5, edge));
    }
}

__global__ void k_level_next(int64_t n, const int* __restrict__ flag, const int* __restrict__ box_of_pt,
                             const uint8_t* __restrict__ leaf, const int* __restrict__ leafidx, uint8_t* __restrict__ active,
                             uint8_t* __restrict__ seg_start, int* __restrict__ leaf_of_pt) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (!active[i]) { seg_start[i] = 0; return; }
    int b = box_of_pt[i];
    bool split = !leaf[b];
    if (!split) leaf_of_pt[i] = leafidx[b];
    seg_start[i] = (flag[i] && split) ? 1 : 0;
    active[i] = split ? 1 : 0;
}

__global__ void k_child_ranges(int64_t nb, const int* __restrict__ parent, int* __restrict__ cbeg, int* __restrict__ cend) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nb) return;
    int p = parent[c];
    if (c == 0 || parent[c - 1] != p) cbeg[p] = (int)c;
    if (c == nb - 1 || parent[c + 1] != p) cend[p] = (int)(c + 1);
}

__global__ void k_leaf_table(int64_t nb, const uint8_t* __restrict__ leaf, const int* __restrict__ scan, int64_t first, int l,
                             int* __restrict__ leafidx, int* __restrict__ leaf_level, int* __restrict__ leaf_box) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    if (leaf[b]) {
        int li = scan[b];
        leafidx[b] = (int)(first + li);   // global leaf-table index
        leaf_level[li] = l;               // per-level slice of the table
        leaf_box[li] = (int)b;
    } else {
        leafidx[b] = -1;
    }
}

__global__ void k_u8_to_int(const uint8_t* __restrict__ a, int64_t n, int* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i];
}

__global__ void k_gather_pos(const double* __restrict__ p, const int* __restrict__ perm, int64_t n, double* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int j = perm[i];
#pragma unroll
    for (int a = 0; a < 3; ++a) out[3 * i + a] = p[3 * (int64_t)j + a];
}

static inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

void build_tree(Plan& p, const double* pts_dev) {
    cudaStream_t s = p.stream;
    const int64_t n = p.n;
    // ---- bounding box and non-finite check
    int nbb = (int)std::min<int64_t>(1024, (n + 255) / 256);
    double* part = p.mem.make<double>(6 * nbb);
    int* bad = p.mem.make<int>(1);
    MLFMA_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    k_bbox_partial<<<nbb, 256, 0, s>>>(pts_dev, n, part, bad);
    MLFMA_LAUNCH_CHECK();
    std::vector<double> hpart(6 * nbb);
    int hbad = 0;
    MLFMA_CUDA(cudaMemcpyAsync(hpart.data(), part, 6 * nbb * sizeof(double), cudaMemcpyDeviceToHost, s));
    MLFMA_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    MLFMA_CUDA(cudaStreamSynchronize(s));
    if (hbad) fail(MLFMA_ERR_INVALID_ARG, "points contain non-finite coordinates");
    double lo[3] = {1e308, 1e308, 1e308}, hi[3] = {-1e308, -1e308, -1e308};
    for (int b = 0; b < nbb; ++b)
        for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], hpart[6 * b + a]); hi[a] = std::max(hi[a], hpart[6 * b + 3 + a]); }
    double D0 = 0;
    for (int a = 0; a < 3; ++a) D0 = std::max(D0, hi[a] - lo[a]);
    p.D0 = D0;
    double c[3];
    for (int a = 0; a < 3; ++a) c[a] = 0.5 * (lo[a] + hi[a]);
    int nlev;
    if (p.leaf_max == 0) {
        int L = 1;
        while (p.leaf_edge * std::ldexp(1.0, L - 1) < D0) ++L;
        if (L > p.max_depth)
            fail(MLFMA_ERR_UNSUPPORTED, "level-uniform tree needs %d levels > max_depth %d", L, p.max_depth);
        p.a1 = p.leaf_edge * std::ldexp(1.0, L - 1);
        nlev = L;
    } else {
        p.a1 = D0 > 0.0 ? D0 * (1.0 + std::ldexp(1.0, -30)) : p.leaf_edge;
        int cutoff = 1;
        while (cutoff < kMaxLev && p.a1 / std::ldexp(1.0, cutoff) >= p.leaf_edge) ++cutoff;
        nlev = std::min(p.max_depth, cutoff);
    }
    p.nlev = nlev;
    for (int a = 0; a < 3; ++a) p.x0[a] = c[a] - 0.5 * p.a1;
    p.scale = std::ldexp(1.0, kBits) / p.a1;

    // ---- keys + stable sort by (key, index)
    uint64_t* k0 = p.mem.make<uint64_t>(n);
    uint64_t* k1 = p.mem.make<uint64_t>(n);
    int* v0 = p.mem.make<int>(n);
    int* v1 = p.mem.make<int>(n);
    k_keys<<<nblk(n, 256), 256, 0, s>>>(pts_dev, n, p.x0[0], p.x0[1], p.x0[2], p.scale, k0, v0);
    MLFMA_LAUNCH_CHECK();
    int nrb = nblk(n, kRadixTile);
    int64_t ncount = (int64_t)256 * nrb;
    int* counts = p.mem.make<int>(ncount);
    int* offs = p.mem.make<int>(ncount);
    int* tmp = p.mem.make<int>(scan_tmp_ints(std::max<int64_t>(ncount, n)) + 8);
    for (int shift = 0; shift < 64; shift += 8) {
        k_radix_hist<<<nrb, 256, 0, s>>>(k0, n, shift, counts, nrb);
        MLFMA_LAUNCH_CHECK();
        scan_exclusive(counts, offs, ncount, tmp, s);
        k_radix_scatter<<<nrb, 256, 0, s>>>(k0, v0, k1, v1, n, shift, offs, nrb);
        MLFMA_LAUNCH_CHECK();
        std::swap(k0, k1);
        std::swap(v0, v1);
    }
    p.keys = k0;
    p.perm = v0;
    p.pos = p.mem.make<double>(3 * n);
    k_gather_pos<<<nblk(n, 256), 256, 0, s>>>(pts_dev, p.perm, n, p.pos);
    MLFMA_LAUNCH_CHECK();

    // ---- levels
    uint8_t* active = p.mem.make<uint8_t>(n);
    uint8_t* seg = p.mem.make<uint8_t>(n);
    int* flag = p.mem.make<int>(n);
    int* scan = p.mem.make<int>(n);
    int* pbox = p.mem.make<int>(n);
    int* cbox = p.mem.make<int>(n);
    p.leaf_of_pt = p.mem.make<int>(n);
    MLFMA_CUDA(cudaMemsetAsync(active, 1, n, s));
    MLFMA_CUDA(cudaMemsetAsync(seg, 0, n, s));
    MLFMA_CUDA(cudaMemsetAsync(seg, 1, 1, s));
    MLFMA_CUDA(cudaMemsetAsync(pbox, 0xff, n * sizeof(int), s));
    std::vector<int*> leafidx(nlev + 1, nullptr);
    std::vector<int64_t> nleaf(nlev + 1, 0);
    p.leaf_first.assign(nlev + 2, 0);
    // leaf table is filled level by level; its size is known only at the end, so keep
    // per-level arrays and concatenate afterwards
    std::vector<int*> lt_level(nlev + 1), lt_box(nlev + 1);
    int64_t leaves_so_far = 0;
    for (int l = 1; l <= nlev; ++l) {
        TreeLevel& L = p.lev[l];
        L.l = l;
        L.edge = p.a1 / std::ldexp(1.0, l - 1);
        int shift = 3 * (kMaxLev - l);
        k_level_flags<<<nblk(n, 256), 256, 0, s>>>(p.keys, n, shift, active, seg, flag);
        MLFMA_LAUNCH_CHECK();
        int nb = scan_exclusive(flag, scan, n, tmp, s);
        L.nbox = nb;
        L.key = p.mem.make<uint64_t>(std::max(nb, 1));
        L.begin = p.mem.make<int>(std::max(nb, 1));
        L.end = p.mem.make<int>(std::max(nb, 1));
        L.parent = p.mem.make<int>(std::max(nb, 1));
        L.child_begin = p.mem.make<int>(std::max(nb, 1));
        L.child_end = p.mem.make<int>(std::max(nb, 1));
        L.leaf = p.mem.make<uint8_t>(std::max(nb, 1));
        L.ijk = p.mem.make<int>(3 * std::max(nb, 1));
        L.center = p.mem.make<double>(3 * std::max(nb, 1));
        MLFMA_CUDA(cudaMemsetAsync(L.child_begin, 0, std::max(nb, 1) * sizeof(int), s));
        MLFMA_CUDA(cudaMemsetAsync(L.child_end, 0, std::max(nb, 1) * sizeof(int), s));
        k_level_fill<<<nblk(n, 256), 256, 0, s>>>(p.keys, n, shift, active, seg, flag, scan, pbox, L.key, L.begin, L.end,
                                                  L.parent, cbox);
        MLFMA_LAUNCH_CHECK();
        if (nb > 0) {
            k_level_boxes<<<nblk(nb, 256), 256, 0, s>>>(nb, l, nlev, p.leaf_max, L.edge, p.x0[0], p.x0[1], p.x0[2], L.key,
                                                        L.begin, L.end, L.leaf, L.ijk, L.center);
            MLFMA_LAUNCH_CHECK();
        }
        // leaf table of this level
        int* lf = p.mem.make<int>(std::max(nb, 1));
        int* lscan = p.mem.make<int>(std::max(nb, 1));
        k_u8_to_int<<<nblk(std::max(nb, 1), 256), 256, 0, s>>>(L.leaf, nb, lf);
        MLFMA_LAUNCH_CHECK();
        int nl = scan_exclusive(lf, lscan, nb, tmp, s);
        L.nleaf = nl;
        nleaf[l] = nl;
        p.leaf_first[l] = leaves_so_far;
        leafidx[l] = lf;  // reuse as per-box leaf index
        lt_level[l] = p.mem.make<int>(std::max(nl, 1));
        lt_box[l] = p.mem.make<int>(std::max(nl, 1));
        if (nb > 0) {
            k_leaf_table<<<nblk(nb, 256), 256, 0, s>>>(nb, L.leaf, lscan, leaves_so_far, l, lf, lt_level[l], lt_box[l]);
            MLFMA_LAUNCH_CHECK();
        }
        k_level_next<<<nblk(n, 256), 256, 0, s>>>(n, flag, cbox, L.leaf, lf, active, seg, p.leaf_of_pt);
        MLFMA_LAUNCH_CHECK();
        leaves_so_far += nl;
        std::swap(pbox, cbox);
        if (l >= 2 && nb > 0) {
            TreeLevel& P = p.lev[l - 1];
            k_child_ranges<<<nblk(nb, 256), 256, 0, s>>>(nb, L.parent, P.child_begin, P.child_end);
            MLFMA_LAUNCH_CHECK();
        }
    }
    p.leaf_first[nlev + 1] = leaves_so_far;
    p.nleaf_total = leaves_so_far;
    p.leaf_level = p.mem.make<int>(std::max<int64_t>(leaves_so_far, 1));
    p.leaf_box = p.mem.make<int>(std::max<int64_t>(leaves_so_far, 1));
    for (int l = 1; l <= nlev; ++l) {
        if (!nleaf[l]) continue;
        MLFMA_CUDA(cudaMemcpyAsync(p.leaf_level + p.leaf_first[l], lt_level[l], nleaf[l] * sizeof(int),
                                   cudaMemcpyDeviceToDevice, s));
        MLFMA_CUDA(cudaMemcpyAsync(p.leaf_box + p.leaf_first[l], lt_box[l], nleaf[l] * sizeof(int),
                                   cudaMemcpyDeviceToDevice, s));
    }
    MLFMA_CUDA(cudaStreamSynchronize(s));
}

// ============================================================== lists
__device__ __forceinline__ int find_key(const uint64_t* __restrict__ keys, int64_t nb, uint64_t k) {
    int64_t lo = 0, hi = nb;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < k) lo = mid + 1; else hi = mid;
    }
    return (lo < nb && keys[lo] == k) ? (int)lo : -1;
}

__global__ void k_colleagues(int64_t nb, int l, const uint64_t* __restrict__ keys, const int* __restrict__ ijk, int* __restrict__ coll) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int side = 1 << (l - 1);
    const int x = ijk[3 * b], y = ijk[3 * b + 1], z = ijk[3 * b + 2];
    for (int s = 0; s < 27; ++s) {
        int nx = x + s % 3 - 1, ny = y + (s / 3) % 3 - 1, nz = z + s / 9 - 1;
        int r = -1;
        if (nx >= 0 && ny >= 0 && nz >= 0 && nx < side && ny < side && nz < side)
            r = find_key(keys, nb, morton(nx, ny, nz));
        coll[27 * b + s] = r;
    }
}

__device__ __forceinline__ int cheb(const int* a, const int* b) {
    return max(abs(a[0] - b[0]), max(abs(a[1] - b[1]), abs(a[2] - b[2])));
}

// sorted list of the valid colleague slots of box q (ascending box index)
__device__ __forceinline__ int sorted_colleagues(const int* __restrict__ coll, int q, int* out) {
    int m = 0;
    for (int s = 0; s < 27; ++s) {
        int v = coll[27 * q + s];
        if (v < 0) continue;
        int j = m++;
        while (j > 0 && out[j - 1] > v) { out[j] = out[j - 1]; --j; }
        out[j] = v;
    }
    return m;
}

// V(b) = children of the colleagues of parent(b) not adjacent to b; counts or writes in ascending order
__global__ void k_vlist(int64_t nb, const int* __restrict__ parent, const int* __restrict__ ijk, const int* __restrict__ pcoll,
                        const int* __restrict__ pcb, const int* __restrict__ pce, const int* __restrict__ off, int* __restrict__ cnt,
                        int* __restrict__ out) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int q[27];
    int m = sorted_colleagues(pcoll, parent[b], q);
    int c = 0;
    const int* mine = ijk + 3 * b;
    int w = off ? off[b] : 0;
    for (int a = 0; a < m; ++a)
        for (int s = pcb[q[a]]; s < pce[q[a]]; ++s)
            if (cheb(ijk + 3 * s, mine) >= 2) {
                if (out) out[w + c] = s;
                ++c;
            }
    if (cnt) cnt[b] = c;
}

// ---- near lists (U, W and X; see the file header)
struct LevelView {
    const int* ijk;
    const int* coll;
    const int* parent;
    const int* cb;
    const int* ce;
    const uint8_t* leaf;
};
struct LevelViews {
    LevelView v[kMaxLev + 1];
};

// closed cubes (la, ia) and (lb, ib) touch or overlap
__device__ __forceinline__ bool adjacent(int la, const int* ia, int lb, const int* ib) {
    if (la > lb) { int t = la; la = lb; lb = t; const int* u = ia; ia = ib; ib = u; }
    int s = lb - la;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int lo = ia[a] << s, hi = (ia[a] + 1) << s;
        if (ib[a] < lo - 1 || ib[a] > hi) return false;
    }
    return true;
}

constexpr int kStack = 256;

// Enumerates the near sources of leaf (l, b): emit(level, box) is called for each.
// Returns false if the traversal stack overflowed.
template <typename Emit>
__device__ bool near_sources(const LevelViews& V, int l, int b, Emit emit) {
    const int* ib = V.v[l].ijk + 3 * b;
    // coarser leaves adjacent to b (U) : colleagues of the ancestors
    int anc = b;
    for (int la = l - 1; la >= 1; --la) {
        anc = V.v[la + 1].parent[anc];
        for (int s = 0; s < 27; ++s) {
            int q = V.v[la].coll[27 * anc + s];
            if (q < 0 || q == anc || !V.v[la].leaf[q]) continue;
            if (adjacent(la, V.v[la].ijk + 3 * q, l, ib)) emit(la, q);
        }
    }
    // X: for each ancestor-or-self a at level >= 2: leaves c at levels < la adjacent to parent(a)
    // but not adjacent to a; c is a colleague of an ancestor of a
    int a = b;
    for (int la = l; la >= 2; --la) {
        int pa = V.v[la].parent[a];
        const int* ia = V.v[la].ijk + 3 * a;
        const int* ipa = V.v[la - 1].ijk + 3 * pa;
        int anc2 = pa;
        for (int lc = la - 1; lc >= 1; --lc) {
            for (int s = 0; s < 27; ++s) {
                int q = V.v[lc].coll[27 * anc2 + s];
                if (q < 0 || q == anc2 || !V.v[lc].leaf[q]) continue;
                const int* iq = V.v[lc].ijk + 3 * q;
                if (adjacent(lc, iq, la - 1, ipa) && !adjacent(lc, iq, la, ia)) emit(lc, q);
            }
            if (lc > 1) anc2 = V.v[lc].parent[anc2];
        }
        a = pa;
    }
    // same level and finer (U and W): descend from the colleagues of b
    int st_l[kStack], st_b[kStack];
    int top = 0;
    for (int s = 0; s < 27; ++s) {
        int q = V.v[l].coll[27 * b + s];
        if (q >= 0) { st_l[top] = l; st_b[top] = q; ++top; }
    }
    while (top > 0) {
        --top;
        int lq = st_l[top], q = st_b[top];
        const LevelView& Lq = V.v[lq];
        if (lq == l || adjacent(lq, Lq.ijk + 3 * q, l, ib)) {
            if (Lq.leaf[q]) {
                emit(lq, q);
            } else {
                for (int c = Lq.cb[q]; c < Lq.ce[q]; ++c) {
                    if (top >= kStack) return false;
                    st_l[top] = lq + 1; st_b[top] = c; ++top;
                }
            }
        } else {
            emit(lq, q);          // W
        }
    }
    return true;
}

__global__ void k_near_count(int64_t nleaf, const int* __restrict__ leaf_level, const int* __restrict__ leaf_box, LevelViews V,
                             int* __restrict__ cnt, int* __restrict__ err) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nleaf) return;
    int c = 0;
    bool ok = near_sources(V, leaf_level[t], leaf_box[t], [&](int, int) { ++c; });
    if (!ok) atomicExch(err, 1);
    cnt[t] = c;
}

__global__ void k_near_fill(int64_t nleaf, const int* __restrict__ leaf_level, const int* __restrict__ leaf_box, LevelViews V,
                            const int* __restrict__ off, int* __restrict__ out_lev, int* __restrict__ out_box) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nleaf) return;
    int w = off[t];
    const int w0 = w;
    near_sources(V, leaf_level[t], leaf_box[t], [&](int lv, int bx) { out_lev[w] = lv; out_box[w] = bx; ++w; });
    // insertion sort by (level, box): box index order equals key order within a level
    for (int i = w0 + 1; i < w; ++i) {
        int kl = out_lev[i], kb = out_box[i];
        int j = i;
        while (j > w0 && (out_lev[j - 1] > kl || (out_lev[j - 1] == kl && out_box[j - 1] > kb))) {
            out_lev[j] = out_lev[j - 1];
            out_box[j] = out_box[j - 1];
            --j;
        }
        out_lev[j] = kl;
        out_box[j] = kb;
    }
}

// point pairs summed directly by each leaf: n_b * sum of source sizes
__global__ void k_near_pairs(int64_t nleaf, const int* __restrict__ leaf_level, const int* __restrict__ leaf_box,
                             const int* __restrict__ off, const int* __restrict__ nl, const int* __restrict__ nbx,
                             const int* const* __restrict__ beg, const int* const* __restrict__ end,
                             unsigned long long* __restrict__ total) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nleaf) return;
    int l = leaf_level[t], b = leaf_box[t];
    long long nb = end[l][b] - beg[l][b];
    long long s = 0;
    for (int i = off[t]; i < off[t + 1]; ++i) s += end[nl[i]][nbx[i]] - beg[nl[i]][nbx[i]];
    atomicAdd(total, (unsigned long long)(nb * s - nb));   // minus the self pairs
}

void build_lists(Plan& p) {
    cudaStream_t s = p.stream;
    int* tmp = p.mem.make<int>(scan_tmp_ints(std::max<int64_t>(p.n, 1 << 20)) + 8);
    for (int l = 1; l <= p.nlev; ++l) {
        TreeLevel& L = p.lev[l];
        L.coll = p.mem.make<int>(27 * std::max<int64_t>(L.nbox, 1));
        if (L.nbox) {
            k_colleagues<<<nblk(L.nbox, 128), 128, 0, s>>>(L.nbox, l, L.key, L.ijk, L.coll);
            MLFMA_LAUNCH_CHECK();
        }
    }
    for (int l = 2; l <= p.nlev; ++l) {
        TreeLevel& L = p.lev[l];
        TreeLevel& P = p.lev[l - 1];
        L.v_off = p.mem.make<int>(L.nbox + 1);
        int* cnt = p.mem.make<int>(L.nbox + 1);
        MLFMA_CUDA(cudaMemsetAsync(cnt, 0, (L.nbox + 1) * sizeof(int), s));
        k_vlist<<<nblk(L.nbox, 128), 128, 0, s>>>(L.nbox, L.parent, L.ijk, P.coll, P.child_begin, P.child_end, nullptr, cnt,
                                                  nullptr);
        MLFMA_LAUNCH_CHECK();
        int tot = scan_exclusive(cnt, L.v_off, L.nbox + 1, tmp, s);
        L.nv = tot;
        L.v_src = p.mem.make<int>(std::max(tot, 1));
        k_vlist<<<nblk(L.nbox, 128), 128, 0, s>>>(L.nbox, L.parent, L.ijk, P.coll, P.child_begin, P.child_end, L.v_off,
                                                  nullptr, L.v_src);
        MLFMA_LAUNCH_CHECK();
    }
    // near lists
    LevelViews V;
    memset(&V, 0, sizeof(V));
    for (int l = 1; l <= p.nlev; ++l) {
        TreeLevel& L = p.lev[l];
        V.v[l] = LevelView{L.ijk, L.coll, L.parent, L.child_begin, L.child_end, L.leaf};
    }
    const int64_t nlf = p.nleaf_total;
    int* cnt = p.mem.make<int>(nlf + 1);
    int* err = p.mem.make<int>(1);
    MLFMA_CUDA(cudaMemsetAsync(cnt, 0, (nlf + 1) * sizeof(int), s));
    MLFMA_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    k_near_count<<<nblk(nlf, 64), 64, 0, s>>>(nlf, p.leaf_level, p.leaf_box, V, cnt, err);
    MLFMA_LAUNCH_CHECK();
    p.near_off = p.mem.make<int>(nlf + 1);
    int tot = scan_exclusive(cnt, p.near_off, nlf + 1, tmp, s);
    int herr = 0;
    MLFMA_CUDA(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) fail(MLFMA_ERR_UNSUPPORTED, "near-list traversal exceeded its stack (%d entries)", kStack);
    p.nnear = tot;
    p.near_lev = p.mem.make<int>(std::max(tot, 1));
    p.near_box = p.mem.make<int>(std::max(tot, 1));
    k_near_fill<<<nblk(nlf, 64), 64, 0, s>>>(nlf, p.leaf_level, p.leaf_box, V, p.near_off, p.near_lev, p.near_box);
    MLFMA_LAUNCH_CHECK();
    // pair count
    const int* hb[kMaxLev + 1] = {nullptr};
    const int* he[kMaxLev + 1] = {nullptr};
    for (int l = 1; l <= p.nlev; ++l) { hb[l] = p.lev[l].begin; he[l] = p.lev[l].end; }
    const int** db = p.mem.make<const int*>(kMaxLev + 1);
    const int** de = p.mem.make<const int*>(kMaxLev + 1);
    unsigned long long* dtot = p.mem.make<unsigned long long>(1);
    MLFMA_CUDA(cudaMemcpyAsync(db, hb, sizeof(hb), cudaMemcpyHostToDevice, s));
    MLFMA_CUDA(cudaMemcpyAsync(de, he, sizeof(he), cudaMemcpyHostToDevice, s));
    MLFMA_CUDA(cudaMemsetAsync(dtot, 0, sizeof(unsigned long long), s));
    k_near_pairs<<<nblk(nlf, 256), 256, 0, s>>>(nlf, p.leaf_level, p.leaf_box, p.near_off, p.near_lev, p.near_box, db, de,
                                                 dtot);
    MLFMA_LAUNCH_CHECK();
    unsigned long long ht = 0;
    MLFMA_CUDA(cudaMemcpyAsync(&ht, dtot, sizeof(ht), cudaMemcpyDeviceToHost, s));
    MLFMA_CUDA(cudaStreamSynchronize(s));
    p.near_pairs = (int64_t)ht;
}

}  // namespace mlfma

namespace mlfma {

// ============================================================== M2L work lists
// For every box P that has children at the next level: the children of P's colleagues
// (other than P) that are far from at least one child of P, in ascending box order,
// packed as (src * K) << 32 | far-children mask << 16 | base,
// src * K being the element offset of the source's samples at that level (< 2^32).  A child t of P and a
// source s of slot (dx, dy, dz) are far when the offset
//   ijk_t - ijk_s = -2 (dx, dy, dz) + bits(t) - bits(s)
// has a component of magnitude >= 2 (they are then in each other's V lists).  The offset's
// raster index (ox+3) + 7 (oy+3) + 49 (oz+3) in the 7^3 cube splits into a source part
//   base = (3 - 2 dx - sx) + 7 (3 - 2 dy - sy) + 49 (3 - 2 dz - sz)     (0 .. 285)
// and a child part tx + 7 ty + 49 tz (0 .. 57), so the M2L kernel finds the translation
// row of every (child, source) pair by one addition.
__device__ __forceinline__ bool far_pair(int slot, int cs, int ct) {
    const int d[3] = {slot % 3 - 1, (slot / 3) % 3 - 1, slot / 9 - 1};
    int m = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) m = max(m, abs(-2 * d[a] + ((ct >> a) & 1) - ((cs >> a) & 1)));
    return m >= 2;
}

__global__ void k_m2l_lists(int64_t nb, const int* __restrict__ coll, const int* __restrict__ cb, const int* __restrict__ ce,
                            const uint64_t* __restrict__ ckey, const int* __restrict__ off, int* __restrict__ cnt,
                            unsigned long long* __restrict__ out, int64_t K) {
    int64_t P = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (P >= nb) return;
    int c = 0;
    if (cb[P] < ce[P]) {
        // colleagues in ascending box order (= ascending key order)
        int q[27], qs[27], m = 0;
        for (int sl = 0; sl < 27; ++sl) {
            int v = coll[27 * P + sl];
            if (v < 0 || v == (int)P) continue;
            int j = m++;
            while (j > 0 && q[j - 1] > v) { q[j] = q[j - 1]; qs[j] = qs[j - 1]; --j; }
            q[j] = v; qs[j] = sl;
        }
        const int w0 = off ? off[P] : 0;
        for (int a = 0; a < m; ++a)
            for (int s = cb[q[a]]; s < ce[q[a]]; ++s) {
                const int cs = (int)(ckey[s] & 7);
                unsigned far_t = 0;   // bit t: child t of P (in box order) is far from s
                for (int t = cb[P]; t < ce[P]; ++t)
                    if (far_pair(qs[a], cs, (int)(ckey[t] & 7))) far_t |= 1u << (t - cb[P]);
                if (!far_t) continue;
                if (out) {
                    const int sl = qs[a];
                    const int base = (3 - 2 * (sl % 3 - 1) - (cs & 1)) + 7 * (3 - 2 * ((sl / 3) % 3 - 1) - ((cs >> 1) & 1)) +
                                     49 * (3 - 2 * (sl / 9 - 1) - ((cs >> 2) & 1));
                    out[w0 + c] = ((unsigned long long)((int64_t)s * K) << 32) | ((unsigned long long)far_t << 16) |
                                  (unsigned long long)base;
                }
                ++c;
            }
    }
    if (cnt) cnt[P] = c;
}

void build_m2l_lists(Plan& p) {
    cudaStream_t s = p.stream;
    int* tmp = p.mem.make<int>(scan_tmp_ints(std::max<int64_t>(p.n, 1 << 20)) + 8);
    for (int l = std::max(p.top, 2); p.top && l <= p.nlev; ++l) {
        TreeLevel& P = p.lev[l - 1];
        TreeLevel& C = p.lev[l];
        int* cnt = p.mem.make<int>(P.nbox + 1);
        MLFMA_CUDA(cudaMemsetAsync(cnt, 0, (P.nbox + 1) * sizeof(int), s));
        if ((int64_t)C.nbox * p.far[l].K >= ((int64_t)1 << 32))
            fail(MLFMA_ERR_UNSUPPORTED, "level %d holds %lld samples, beyond 32-bit offsets", l,
                 (long long)((int64_t)C.nbox * p.far[l].K));
        k_m2l_lists<<<nblk(P.nbox, 128), 128, 0, s>>>(P.nbox, P.coll, P.child_begin, P.child_end, C.key, nullptr, cnt,
                                                      nullptr, p.far[l].K);
        MLFMA_LAUNCH_CHECK();
        P.m2l_off = p.mem.make<int>(P.nbox + 1);
        int tot = scan_exclusive(cnt, P.m2l_off, P.nbox + 1, tmp, s);
        P.m2l_n = tot;
        P.m2l_src = p.mem.make<unsigned long long>(std::max(tot, 1));
        k_m2l_lists<<<nblk(P.nbox, 128), 128, 0, s>>>(P.nbox, P.coll, P.child_begin, P.child_end, C.key, P.m2l_off, nullptr,
                                                      P.m2l_src, p.far[l].K);
        MLFMA_LAUNCH_CHECK();
    }
    MLFMA_CUDA(cudaStreamSynchronize(s));
}

}  // namespace mlfma

namespace mlfma {

// ============================================================== P2P work split
__global__ void k_leaf_sizes(int64_t nleaf, const int* __restrict__ leaf_level, const int* __restrict__ leaf_box,
                             const int* const* __restrict__ beg, const int* const* __restrict__ end, int* __restrict__ out) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nleaf) return;
    const int l = leaf_level[t], b = leaf_box[t];
    out[t] = end[l][b] - beg[l][b];
}

// near-field source points of each leaf (sum of its near boxes' point counts)
__global__ void k_leaf_sources(int64_t nleaf, const int* __restrict__ near_off, const int* __restrict__ near_lev,
                               const int* __restrict__ near_box, const int* const* __restrict__ beg,
                               const int* const* __restrict__ end, long long* __restrict__ out) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nleaf) return;
    long long n = 0;
    for (int e = near_off[t]; e < near_off[t + 1]; ++e) {
        const int l = near_lev[e], b = near_box[e];
        n += end[l][b] - beg[l][b];
    }
    out[t] = n;
}

// Heavy leaves first: the entries whose work is above four times the list's mean, by decreasing
// work, then the others in their (Morton) order.  The near field's launches then end with short
// warps instead of waiting on one with thousands of sources.
template <typename T, typename W>
static void heavy_first(std::vector<T>& v, W work) {
    if (v.size() < 2) return;
    double mean = 0;
    for (const T& x : v) mean += (double)work(x);
    mean /= (double)v.size();
    std::vector<T> heavy, rest;
    for (const T& x : v) ((double)work(x) > 4.0 * mean ? heavy : rest).push_back(x);
    std::stable_sort(heavy.begin(), heavy.end(), [&](const T& a, const T& b) { return work(a) > work(b); });
    heavy.insert(heavy.end(), rest.begin(), rest.end());
    v.swap(heavy);
}

void build_p2p_work(Plan& p) {
    cudaStream_t s = p.stream;
    const int64_t nl = p.nleaf_total;
    const int* hb[kMaxLev + 1] = {nullptr};
    const int* he[kMaxLev + 1] = {nullptr};
    for (int l = 1; l <= p.nlev; ++l) { hb[l] = p.lev[l].begin; he[l] = p.lev[l].end; }
    const int** db = p.mem.make<const int*>(kMaxLev + 1);
    const int** de = p.mem.make<const int*>(kMaxLev + 1);
    int* sizes = p.mem.make<int>(std::max<int64_t>(nl, 1));
    MLFMA_CUDA(cudaMemcpyAsync(db, hb, sizeof(hb), cudaMemcpyHostToDevice, s));
    MLFMA_CUDA(cudaMemcpyAsync(de, he, sizeof(he), cudaMemcpyHostToDevice, s));
    k_leaf_sizes<<<nblk(nl, 256), 256, 0, s>>>(nl, p.leaf_level, p.leaf_box, db, de, sizes);
    MLFMA_LAUNCH_CHECK();
    long long* srcs = p.mem.make<long long>(std::max<int64_t>(nl, 1));
    if (nl > 0) {
        k_leaf_sources<<<nblk(nl, 256), 256, 0, s>>>(nl, p.near_off, p.near_lev, p.near_box, db, de, srcs);
        MLFMA_LAUNCH_CHECK();
    }
    std::vector<int> hs(nl);
    std::vector<long long> hsrc(nl);
    MLFMA_CUDA(cudaMemcpyAsync(hs.data(), sizes, nl * sizeof(int), cudaMemcpyDeviceToHost, s));
    MLFMA_CUDA(cudaMemcpyAsync(hsrc.data(), srcs, nl * sizeof(long long), cudaMemcpyDeviceToHost, s));
    MLFMA_CUDA(cudaStreamSynchronize(s));
    p.mem.drop(srcs);
    std::vector<int> small, small_mid;        // up to 32 points; 33 .. kSmallLeaf (two targets per lane)
    std::vector<int2> tiles;
    for (int64_t t = 0; t < nl; ++t) {
        if (hs[t] <= 32) {
            small.push_back((int)t);
        } else if (hs[t] <= kSmallLeaf) {
            small_mid.push_back((int)t);
        } else {
            for (int o = 0; o < hs[t]; o += kP2PTile) tiles.push_back(make_int2((int)t, o));
        }
    }
    // per level: small / big leaves and the point tiles of the big ones
    std::vector<int> lev_of(nl), box_of(nl);
    MLFMA_CUDA(cudaMemcpyAsync(lev_of.data(), p.leaf_level, nl * sizeof(int), cudaMemcpyDeviceToHost, s));
    MLFMA_CUDA(cudaMemcpyAsync(box_of.data(), p.leaf_box, nl * sizeof(int), cudaMemcpyDeviceToHost, s));
    MLFMA_CUDA(cudaStreamSynchronize(s));
    for (int l = 1; l <= p.nlev; ++l) {
        std::vector<int> sm, bg;
        std::vector<int2> bt;
        for (int64_t t = p.leaf_first[l]; t < p.leaf_first[l + 1]; ++t) {
            if (hs[t] <= kSmallLeaf) {
                sm.push_back(box_of[t]);
            } else {
                bg.push_back(box_of[t]);
                for (int o = 0; o < hs[t]; o += kP2PTile) bt.push_back(make_int2(box_of[t], o));
            }
        }
        TreeLevel& L = p.lev[l];
        L.n_small_leaves = (int64_t)sm.size();
        L.n_big_leaves = (int64_t)bg.size();
        L.n_big_tiles = (int64_t)bt.size();
        L.small_leaves = p.mem.make<int>(std::max<int64_t>(L.n_small_leaves, 1));
        L.big_leaves = p.mem.make<int>(std::max<int64_t>(L.n_big_leaves, 1));
        L.big_tiles = p.mem.make<int2>(std::max<int64_t>(L.n_big_tiles, 1));
        if (!sm.empty()) MLFMA_CUDA(cudaMemcpyAsync(L.small_leaves, sm.data(), sm.size() * sizeof(int), cudaMemcpyHostToDevice, s));
        if (!bg.empty()) MLFMA_CUDA(cudaMemcpyAsync(L.big_leaves, bg.data(), bg.size() * sizeof(int), cudaMemcpyHostToDevice, s));
        if (!bt.empty()) MLFMA_CUDA(cudaMemcpyAsync(L.big_tiles, bt.data(), bt.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
        MLFMA_CUDA(cudaStreamSynchronize(s));
    }
    // ---- symmetric pairs of large leaves: both near to each other (or a leaf with itself),
    // each pair of points evaluated once
    if (!tiles.empty()) {
        std::vector<int> noff(nl + 1), nlev, nbox;
        MLFMA_CUDA(cudaMemcpyAsync(noff.data(), p.near_off, (nl + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
        MLFMA_CUDA(cudaStreamSynchronize(s));
        nlev.resize(noff[nl]);
        nbox.resize(noff[nl]);
        if (noff[nl] > 0) {
            MLFMA_CUDA(cudaMemcpyAsync(nlev.data(), p.near_lev, noff[nl] * sizeof(int), cudaMemcpyDeviceToHost, s));
            MLFMA_CUDA(cudaMemcpyAsync(nbox.data(), p.near_box, noff[nl] * sizeof(int), cudaMemcpyDeviceToHost, s));
            MLFMA_CUDA(cudaStreamSynchronize(s));
        }
        std::unordered_map<long long, int> leaf_at;   // (level, box) -> leaf-table index of large leaves
        for (int64_t t = 0; t < nl; ++t)
            if (hs[t] > kSmallLeaf) leaf_at[((long long)lev_of[t] << 32) | (unsigned)box_of[t]] = (int)t;
        auto big_of = [&](int e) {
            auto f = leaf_at.find(((long long)nlev[e] << 32) | (unsigned)nbox[e]);
            return f == leaf_at.end() ? -1 : f->second;
        };
        std::set<std::pair<int, int>> nearbig;     // (A, B): B a large near box of large leaf A, A != B
        for (int64_t t = 0; t < nl; ++t) {
            if (hs[t] <= kSmallLeaf) continue;
            for (int e = noff[t]; e < noff[t + 1]; ++e) {
                const int b = big_of(e);
                if (b >= 0 && b != (int)t) nearbig.insert({(int)t, b});
            }
        }
        auto mutual = [&](int a, int b) { return nearbig.count({a, b}) && nearbig.count({b, a}); };
        std::vector<int> aoff(nl + 1, 0), alev, abox;
        struct Item { int a, o, b; long long work; };
        std::vector<Item> items;
        for (int64_t t = 0; t < nl; ++t) {
            aoff[t] = (int)alev.size();
            if (hs[t] <= kSmallLeaf) continue;
            for (int e = noff[t]; e < noff[t + 1]; ++e) {
                const int b = big_of(e);
                if (b == (int)t) {                     // the leaf with itself: pairs j > i, once
                    for (int o = 0; o < hs[t]; o += kP2PTile)
                        items.push_back({(int)t, o, b, (long long)std::min(kP2PTile, hs[t] - o) * (hs[t] - o)});
                    continue;
                }
                if (b >= 0 && b != (int)t && mutual((int)t, b)) {
                    if (b > (int)t)
                        for (int o = 0; o < hs[t]; o += kP2PTile)
                            items.push_back({(int)t, o, b, (long long)std::min(kP2PTile, hs[t] - o) * hs[b]});
                    continue;
                }
                alev.push_back(nlev[e]);
                abox.push_back(nbox[e]);
            }
        }
        aoff[nl] = (int)alev.size();
        // scratch offsets, then heavy items first
        std::stable_sort(items.begin(), items.end(), [](const Item& x, const Item& y) { return x.work > y.work; });
        long long scratch = 0;
        std::vector<int4> hitems;
        std::vector<std::vector<int2>> red(nl);
        for (const Item& it : items) {
            hitems.push_back(make_int4(it.a, it.o, it.b, (int)scratch));
            red[it.a].push_back(make_int2((int)scratch, it.o));
            red[it.b].push_back(make_int2((int)scratch, -1));
            scratch += kP2PTile + hs[it.b];
        }
        if (!items.empty() && scratch < (1ll << 31)) {
            std::vector<int> roff(nl + 1, 0);
            std::vector<int2> rflat;
            for (int64_t t = 0; t < nl; ++t) {
                roff[t] = (int)rflat.size();
                rflat.insert(rflat.end(), red[t].begin(), red[t].end());
            }
            roff[nl] = (int)rflat.size();
            p.n_sym_items = (int64_t)hitems.size();
            p.sym_items = p.mem.make<int4>(hitems.size());
            p.sym_buf = p.mem.get((size_t)scratch * csize(p));
            p.asym_off = p.mem.make<int>(nl + 1);
            p.asym_lev = p.mem.make<int>(std::max<size_t>(alev.size(), 1));
            p.asym_box = p.mem.make<int>(std::max<size_t>(abox.size(), 1));
            p.sym_red_off = p.mem.make<int>(nl + 1);
            p.sym_red = p.mem.make<int2>(std::max<size_t>(rflat.size(), 1));
            MLFMA_CUDA(cudaMemcpyAsync(p.sym_items, hitems.data(), hitems.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
            MLFMA_CUDA(cudaMemcpyAsync(p.asym_off, aoff.data(), (nl + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
            if (!alev.empty()) {
                MLFMA_CUDA(cudaMemcpyAsync(p.asym_lev, alev.data(), alev.size() * sizeof(int), cudaMemcpyHostToDevice, s));
                MLFMA_CUDA(cudaMemcpyAsync(p.asym_box, abox.data(), abox.size() * sizeof(int), cudaMemcpyHostToDevice, s));
            }
            MLFMA_CUDA(cudaMemcpyAsync(p.sym_red_off, roff.data(), (nl + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
            MLFMA_CUDA(cudaMemcpyAsync(p.sym_red, rflat.data(), rflat.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
            MLFMA_CUDA(cudaStreamSynchronize(s));
        }
    }
    auto leaf_work = [&](int t) { return (long long)hs[t] * hsrc[t]; };
    heavy_first(small, leaf_work);
    heavy_first(small_mid, leaf_work);
    heavy_first(tiles, [&](const int2& tl) { return (long long)std::min(kP2PTile, hs[tl.x] - tl.y) * hsrc[tl.x]; });
    p.n_small32 = (int64_t)small.size();
    small.insert(small.end(), small_mid.begin(), small_mid.end());
    p.n_small = (int64_t)small.size();
    p.n_tiles = (int64_t)tiles.size();
    p.p2p_small = p.mem.make<int>(std::max<int64_t>(p.n_small, 1));
    p.p2p_tiles = p.mem.make<int2>(std::max<int64_t>(p.n_tiles, 1));
    if (p.n_small)
        MLFMA_CUDA(cudaMemcpyAsync(p.p2p_small, small.data(), small.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    if (p.n_tiles)
        MLFMA_CUDA(cudaMemcpyAsync(p.p2p_tiles, tiles.data(), tiles.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    MLFMA_CUDA(cudaStreamSynchronize(s));
}

}  // namespace mlfma
