// Near-field direct sums (Sec. 2: near-field calculations happen only at the leaves),
// permutation to/from Morton order, the FP64 direct sum used for accuracy checks,
// and the per-right-hand-side apply pipeline.
//
// P2P for a target leaf b sums q_j e^{ikR}/R over the points of its near sources
// (U list; W and X lists of adaptive trees), skipping R = 0 (the point itself and
// coincident points).  One warp per target leaf of up to 64 points; the source points of its
// near boxes are staged through shared memory relative to the target leaf centre (FP64
// difference, then rounded); lanes split (target, source slice) and the slices are combined
// with warp shuffles, or with 33-64 targets every lane takes two.  Larger leaves take tiles of
// 128 targets per CTA.  The FP32 kernels evaluate sin and cos of k R on the SFU after reducing
// k R / pi to [-1, 1] (absolute error about 4e-7).
#include <cstdio>

#include <type_traits>

#include "common.cuh"

namespace mlfma {

static inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

// 1/R from R^2, 0 for coincident points (the excluded self term).  FP32: the SFU's reciprocal
// square root with subnormals flushed (rsqrt.approx.ftz.f32: no subnormal handling around it),
// so a squared distance below the smallest normal float (R < 1.1e-19) counts as coincident.
__device__ __forceinline__ float inv_dist(float r2) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(r2));
    return r2 >= 1.17549435e-38f ? y : 0.f;
}
__device__ __forceinline__ double inv_dist(double r2) { return r2 > 0.0 ? rsqrt(r2) : 0.0; }

// sin and cos of pi * x.  FP32: reduce x to [-1, 1] (x - 2 rint(x / 2)), then the SFU's sine
// and cosine on [-pi, pi] (sin.approx / cos.approx with subnormals flushed: absolute error
// ~4e-7, below the FP32 path's tolerance); FP64: sincospi.
__device__ __forceinline__ void scpi_fast(float x, float& s, float& c) {
    const float a = 3.14159265358979f * (x - 2.0f * rintf(0.5f * x));
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(a));
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(c) : "f"(a));
}
__device__ __forceinline__ void scpi_fast(double x, double& s, double& c) { sincospi(x, &s, &c); }

// a staged source: position relative to the target leaf centre and one more value
template <typename R>
struct __align__(4 * sizeof(R) > 16 ? 16 : 4 * sizeof(R)) SrcPos {
    R x, y, z, w;
};

struct LevelRanges {
    const int* begin[kMaxLev + 1];
    const int* end[kMaxLev + 1];
    const double* center[kMaxLev + 1];
};

// GRAD: also grad phi_i = sum_j q_j e^{ikR} (ikR - 1) / R^3 (r_i - r_j), written to grads[3 i + a].
// The near sources of the leaf are read as one stream over its near boxes: each round the
// lanes take up to 32 boxes, scan their point counts and fill up to kP2PSlots staged
// sources (a lane finds the box of its slot by a binary search over the scanned counts),
// so the loads of many small boxes are in flight together.  (eb, oe) is the stream
// cursor: box entry and points of it already consumed.
constexpr int kP2PSlots = 128;

// NR right-hand sides (charges and potentials sn apart) share each kernel value; GRAD only
// with NR = 1.  TWO: the leaves of the list hold 33 .. 64 points (else at most 32).
template <typename R, typename C, bool GRAD, int NR, bool TWO>
__global__ void __launch_bounds__(128) k_p2p(int64_t nleaf, const int* __restrict__ leaves, const int* __restrict__ leaf_level,
                                             const int* __restrict__ leaf_box, const int* __restrict__ near_off,
                                             const int* __restrict__ near_lev, const int* __restrict__ near_box, LevelRanges LR,
                                             const double* __restrict__ pos, const C* __restrict__ qs, int64_t sn, R kpi,
                                             C* __restrict__ phis, C* __restrict__ grads) {
    static_assert(!GRAD || NR == 1, "gradients take one right-hand side per pass");
    constexpr unsigned FULL = 0xffffffffu;
    __shared__ R sx[4][kP2PSlots], sy[4][kP2PSlots], sz[4][kP2PSlots];
    __shared__ C sq[4][NR][kP2PSlots];
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t wi = (int64_t)blockIdx.x * 4 + wl;
    if (wi >= nleaf) return;
    const int w = leaves[wi];
    const int l = leaf_level[w], b = leaf_box[w];
    const int t0 = LR.begin[l][b], t1 = LR.end[l][b];
    const double* ct = LR.center[l] + 3 * b;
    const double cx = ct[0], cy = ct[1], cz = ct[2];
    const int s_lo = near_off[w], s_hi = near_off[w + 1];
    // up to 32 targets: P lanes (a power of two) take one target each and the S = 32 / P lane
    // groups split the sources; 33 .. 64 targets: every lane takes targets tp and tp + 32, so
    // each staged source feeds two targets and the stream is staged once
    const int nt = t1 - t0;
    const int np = TWO ? 32 : nt;
    int P = 1;
    while (P < np) P <<= 1;
    const int S = 32 / P;
    const int tp = lane & (P - 1), sl = lane / P;
    const int i = t0 + tp, i2 = i + 32;
    const bool has1 = tp < np, has2 = TWO && i2 < t1;
    R x = 0, y = 0, z = 0, x2 = 0, y2 = 0, z2 = 0;
    if (has1) {
        x = (R)(pos[3 * (int64_t)i] - cx);
        y = (R)(pos[3 * (int64_t)i + 1] - cy);
        z = (R)(pos[3 * (int64_t)i + 2] - cz);
    }
    if (has2) {
        x2 = (R)(pos[3 * (int64_t)i2] - cx);
        y2 = (R)(pos[3 * (int64_t)i2 + 1] - cy);
        z2 = (R)(pos[3 * (int64_t)i2 + 2] - cz);
    }
    C acc[NR], acc2[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = acc2[r] = cmake<C>(0, 0);
    C ga[3] = {cmake<C>(0, 0), cmake<C>(0, 0), cmake<C>(0, 0)};
    C gb[3] = {cmake<C>(0, 0), cmake<C>(0, 0), cmake<C>(0, 0)};
    const R kk = kpi * (R)M_PI;
    // one (target, source) term, branch-free: R = 0 (the point itself, coincident points) gives
    // inv = 0 and adds nothing
    auto term = [&](R tx, R ty, R tz, int jj, C (&ac)[NR], C (&gg)[3]) {
        const R dx = tx - sx[wl][jj], dy = ty - sy[wl][jj], dz = tz - sz[wl][jj];
        const R r2 = dx * dx + dy * dy + dz * dz;
        const R inv = inv_dist(r2);
        const R r = r2 * inv;
        R s, c;
        scpi_fast(kpi * r, s, c);
        if (!GRAD) {
            const C g = cmake<C>(c * inv, s * inv);
#pragma unroll
            for (int q = 0; q < NR; ++q) cfma(ac[q], sq[wl][q][jj], g);
        } else {
            const C qe = cmul(sq[wl][0][jj], cmake<C>(c * inv, s * inv));   // q e^{ikR} / R
            ac[0] = cadd(ac[0], qe);
            // q e^{ikR} (ikR - 1) / R^3 = qe (ikR - 1) / R^2
            const R iv2 = inv * inv;
            const C g = cmul(qe, cmake<C>(-iv2, kk * r * iv2));
            gg[0] = cadd(gg[0], cmake<C>(g.x * dx, g.y * dx));
            gg[1] = cadd(gg[1], cmake<C>(g.x * dy, g.y * dy));
            gg[2] = cadd(gg[2], cmake<C>(g.x * dz, g.y * dz));
        }
    };
    int eb = s_lo, oe = 0;
    while (eb < s_hi) {
        const int e = eb + lane;
        int u0 = 0, cnt = 0;
        if (e < s_hi) {
            const int ls = near_lev[e], bs = near_box[e];
            u0 = LR.begin[ls][bs];
            cnt = LR.end[ls][bs] - u0;
        }
        if (lane == 0) { u0 += oe; cnt -= oe; }
        int inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += t;
        }
        const int exc = inc - cnt;
        const int all = __shfl_sync(FULL, inc, 31);
        const int total = min(all, kP2PSlots);
        for (int s0 = 0; s0 < total; s0 += 32) {
            const int sidx = s0 + lane;
            int q = 0;                       // first lane whose inclusive count exceeds sidx
#pragma unroll
            for (int st = 16; st >= 1; st >>= 1) {
                const int v = __shfl_sync(FULL, inc, q + st - 1);
                if (v <= sidx) q += st;
            }
            const int uq = __shfl_sync(FULL, u0, q), xq = __shfl_sync(FULL, exc, q);
            if (sidx < total) {
                const int64_t j = uq + (sidx - xq);
                sx[wl][sidx] = (R)(pos[3 * j] - cx);
                sy[wl][sidx] = (R)(pos[3 * j + 1] - cy);
                sz[wl][sidx] = (R)(pos[3 * j + 2] - cz);
#pragma unroll
                for (int r = 0; r < NR; ++r) sq[wl][r][sidx] = qs[r * sn + j];
            }
        }
        // advance the cursor past the consumed points
        const int qn = __popc(__ballot_sync(FULL, inc <= total));
        if (total == all) {
            eb += 32;
            oe = 0;
        } else {
            const int xn = __shfl_sync(FULL, exc, qn);
            oe = (qn == 0 ? oe : 0) + (total - xn);
            eb += qn;
        }
        __syncwarp();
        if constexpr (TWO) {
            // every lane holds two targets (the second may be absent: its terms are discarded)
            for (int jj = 0; jj < total; ++jj) {
                term(x, y, z, jj, acc, ga);
                term(x2, y2, z2, jj, acc2, gb);
            }
        } else if (has1) {
            for (int jj = sl; jj < total; jj += S) term(x, y, z, jj, acc, ga);
        }
        __syncwarp();
    }
    for (int o = 16; o >= P && S > 1; o >>= 1) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            acc[r].x += __shfl_xor_sync(0xffffffffu, acc[r].x, o);
            acc[r].y += __shfl_xor_sync(0xffffffffu, acc[r].y, o);
        }
        if (GRAD) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                ga[a].x += __shfl_xor_sync(0xffffffffu, ga[a].x, o);
                ga[a].y += __shfl_xor_sync(0xffffffffu, ga[a].y, o);
            }
        }
    }
    if (sl == 0 && has1) {
#pragma unroll
        for (int r = 0; r < NR; ++r) phis[r * sn + i] = acc[r];
        if (GRAD)
#pragma unroll
            for (int a = 0; a < 3; ++a) grads[3 * (int64_t)i + a] = ga[a];
    }
    if (TWO && has2) {
#pragma unroll
        for (int r = 0; r < NR; ++r) phis[r * sn + i2] = acc2[r];
        if (GRAD)
#pragma unroll
            for (int a = 0; a < 3; ++a) grads[3 * (int64_t)i2 + a] = gb[a];
    }
}


// Larger leaves: one CTA per tile of kP2PTile targets, one target per thread; the source
// points of every near box are staged through shared memory (positions relative to the
// target leaf centre, FP64 difference then rounded) in tiles of 2 * kP2PTile.
template <typename R, typename C, bool GRAD, int NR>
__global__ void __launch_bounds__(kP2PTile) k_p2p_tile(const int2* __restrict__ tiles, const int* __restrict__ leaf_level,
                                                       const int* __restrict__ leaf_box, const int* __restrict__ near_off,
                                                       const int* __restrict__ near_lev, const int* __restrict__ near_box,
                                                       LevelRanges LR, const double* __restrict__ pos,
                                                       const C* __restrict__ qs, int64_t sn, R kpi, C* __restrict__ phis,
                                                       C* __restrict__ grads) {
    static_assert(!GRAD || NR == 1, "gradients take one right-hand side per pass");
    constexpr int SRC = 2 * kP2PTile;
    __shared__ R sx[SRC], sy[SRC], sz[SRC];
    __shared__ C sq[NR][SRC];
    const int2 tile = tiles[blockIdx.x];
    const int w = tile.x;
    const int l = leaf_level[w], b = leaf_box[w];
    const int t0 = LR.begin[l][b], t1 = LR.end[l][b];
    const double* ct = LR.center[l] + 3 * b;
    const double cx = ct[0], cy = ct[1], cz = ct[2];
    const int i = t0 + tile.y + threadIdx.x;
    const bool valid = i < t1;
    R x = 0, y = 0, z = 0;
    if (valid) {
        x = (R)(pos[3 * (int64_t)i] - cx);
        y = (R)(pos[3 * (int64_t)i + 1] - cy);
        z = (R)(pos[3 * (int64_t)i + 2] - cz);
    }
    const R kk = kpi * (R)M_PI;
    C acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = cmake<C>(0, 0);
    C ga[3] = {cmake<C>(0, 0), cmake<C>(0, 0), cmake<C>(0, 0)};
    for (int e = near_off[w]; e < near_off[w + 1]; ++e) {
        const int ls = near_lev[e], bs = near_box[e];
        const int u0 = LR.begin[ls][bs], u1 = LR.end[ls][bs];
        for (int k0 = u0; k0 < u1; k0 += SRC) {
            const int cnt = min(SRC, u1 - k0);
            __syncthreads();
            for (int m = threadIdx.x; m < cnt; m += blockDim.x) {
                const int64_t j = k0 + m;
                sx[m] = (R)(pos[3 * j] - cx);
                sy[m] = (R)(pos[3 * j + 1] - cy);
                sz[m] = (R)(pos[3 * j + 2] - cz);
#pragma unroll
                for (int r = 0; r < NR; ++r) sq[r][m] = qs[r * sn + j];
            }
            __syncthreads();
            if (valid) {
#pragma unroll 4
                for (int m = 0; m < cnt; ++m) {
                    const R dx = x - sx[m], dy = y - sy[m], dz = z - sz[m];
                    const R r2 = dx * dx + dy * dy + dz * dz;
                    if (!GRAD) {
                        // branch-free: R = 0 (self / coincident) gives inv = 0 and no contribution
                        const R inv = inv_dist(r2);
                        R s, c;
                        scpi_fast(kpi * (r2 * inv), s, c);
                        const C g = cmake<C>(c * inv, s * inv);
#pragma unroll
                        for (int r = 0; r < NR; ++r) cfma(acc[r], sq[r][m], g);
                    } else {
                        const R inv = inv_dist(r2);
                        const R r = r2 * inv;
                        R s, c;
                        scpi_fast(kpi * r, s, c);
                        const C qe = cmul(sq[0][m], cmake<C>(c * inv, s * inv));
                        acc[0] = cadd(acc[0], qe);
                        const R i2 = inv * inv;
                        const C g = cmul(qe, cmake<C>(-i2, kk * r * i2));
                        ga[0] = cadd(ga[0], cmake<C>(g.x * dx, g.y * dx));
                        ga[1] = cadd(ga[1], cmake<C>(g.x * dy, g.y * dy));
                        ga[2] = cadd(ga[2], cmake<C>(g.x * dz, g.y * dz));
                    }
                }
            }
        }
    }
    if (valid) {
#pragma unroll
        for (int r = 0; r < NR; ++r) phis[r * sn + i] = acc[r];
        if (GRAD)
#pragma unroll
            for (int a = 0; a < 3; ++a) grads[3 * (int64_t)i + a] = ga[a];
    }
}

// Symmetric near field of two mutually near large leaves A and B (the kernel e^{ikR}/R is
// symmetric in its two points), and of a large leaf with itself (B = A: the sources from the
// tile's first point on, pairs j > i only; the reverse sums below o are zero): one CTA per work
// item (A, target offset o in A, B, scratch offset); thread t holds target o + t of A, and each warp meets 32 sources of B at a time in
// 32 rotation steps (lane l takes source (l + s) mod 32 at step s; the chunk is staged twice in a
// row, so that source is entry l + s): the forward term q_j K_ij
// goes to the lane's target sum, the reverse term q_i K_ij to an accumulator that moves to the
// next lower lane after every step, so after the 32 steps lane l holds the warp's sum for source
// l.  The four warps' sums are added in a fixed order.  Writes the forward sums of the item's
// targets to scratch[off .. off + kP2PTile) and the reverse sums of all of B to
// scratch[off + kP2PTile ..); k_p2p_sym_reduce adds them to the potentials.
template <typename R, typename C>
__global__ void __launch_bounds__(kP2PTile) k_p2p_sym(const int4* __restrict__ items, const int* __restrict__ leaf_level,
                                                      const int* __restrict__ leaf_box, LevelRanges LR,
                                                      const double* __restrict__ pos, const C* __restrict__ qs, R kpi,
                                                      C* __restrict__ scratch) {
    constexpr unsigned FULL = 0xffffffffu;
    // the chunk's 32 sources twice in a row, so lane l's source at step s is entry l + s: position
    // and real part of the charge in one record, imaginary part beside it
    __shared__ SrcPos<R> sp[64];
    __shared__ R sqi[64];
    __shared__ C red[kP2PTile / 32][32];
    const int4 it = items[blockIdx.x];
    const int la = leaf_level[it.x], ba = leaf_box[it.x];
    const int lb = leaf_level[it.z], bb = leaf_box[it.z];
    const int t0 = LR.begin[la][ba], t1 = LR.end[la][ba];
    const int u0 = LR.begin[lb][bb], nb = LR.end[lb][bb] - u0;
    const double* ct = LR.center[la] + 3 * ba;
    const double cx = ct[0], cy = ct[1], cz = ct[2];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const bool self = it.x == it.z;             // B = A: pairs j > i only
    const int iu = it.y + (int)threadIdx.x;      // target index within A
    const int i = t0 + iu;
    const bool valid = i < t1;
    R x = 0, y = 0, z = 0;
    C qi = cmake<C>(0, 0);                       // an absent target contributes nothing in reverse
    if (valid) {
        x = (R)(pos[3 * (int64_t)i] - cx);
        y = (R)(pos[3 * (int64_t)i + 1] - cy);
        z = (R)(pos[3 * (int64_t)i + 2] - cz);
        qi = qs[i];
    }
    C fwd = cmake<C>(0, 0);
    C* out = scratch + (unsigned)it.w;
    const int kstart = self ? it.y : 0;          // B = A: sources from the tile's first point on
    for (int j = threadIdx.x; j < kstart; j += blockDim.x) out[kP2PTile + j] = cmake<C>(0, 0);
    for (int k0 = kstart; k0 < nb; k0 += 32) {
        __syncthreads();                         // the previous chunk's sources and sums are consumed
        if (threadIdx.x < 32) {
            const int j = k0 + (int)threadIdx.x;
            SrcPos<R> v{(R)0, (R)0, (R)0, (R)0}; // past the end of B: a zero charge
            R vi = 0;
            if (j < nb) {
                const int64_t jj = u0 + j;
                const C qj = qs[jj];
                v = SrcPos<R>{(R)(pos[3 * jj] - cx), (R)(pos[3 * jj + 1] - cy), (R)(pos[3 * jj + 2] - cz), qj.x};
                vi = qj.y;
            }
            sp[threadIdx.x] = v;
            sp[threadIdx.x + 32] = v;
            sqi[threadIdx.x] = vi;
            sqi[threadIdx.x + 32] = vi;
        }
        __syncthreads();
        C rev = cmake<C>(0, 0);
        const SrcPos<R>* pl = sp + lane;
        const R* ql = sqi + lane;
        // B = A: the chunks that overlap the tile keep only j > i (the chunks above it need no mask,
        // and run a loop without the test)
        auto steps = [&](auto masked) {
#pragma unroll 4
            for (int st = 0; st < 32; ++st) {
                const SrcPos<R> ps = pl[st];
                const R qjy = ql[st];
                const R dx = x - ps.x, dy = y - ps.y, dz = z - ps.z;
                const R r2 = dx * dx + dy * dy + dz * dz;
                R inv = inv_dist(r2);
                if constexpr (decltype(masked)::value)
                    if (k0 + ((lane + st) & 31) <= iu) inv = (R)0;
                R sn, cs;
                scpi_fast(kpi * (r2 * inv), sn, cs);
                const C g = cmake<C>(cs * inv, sn * inv);
                cfma(fwd, cmake<C>(ps.w, qjy), g);
                cfma(rev, qi, g);
                rev.x = __shfl_sync(FULL, rev.x, (lane + 1) & 31);
                rev.y = __shfl_sync(FULL, rev.y, (lane + 1) & 31);
            }
        };
        if (self && k0 < it.y + kP2PTile) steps(std::true_type{});
        else steps(std::false_type{});
        red[wl][lane] = rev;
        __syncthreads();
        if (threadIdx.x < 32 && k0 + (int)threadIdx.x < nb) {
            C sum = red[0][threadIdx.x];
#pragma unroll
            for (int w = 1; w < kP2PTile / 32; ++w) sum = cadd(sum, red[w][threadIdx.x]);
            out[kP2PTile + k0 + threadIdx.x] = sum;
        }
    }
    out[threadIdx.x] = valid ? fwd : cmake<C>(0, 0);
}

// Adds the symmetric pass's partial sums to the potentials of the large leaves' points, one CTA
// per target tile, each point's blocks in the leaf's fixed order (deterministic).
template <typename C>
__global__ void __launch_bounds__(kP2PTile) k_p2p_sym_reduce(const int2* __restrict__ tiles, const int* __restrict__ leaf_level,
                                                             const int* __restrict__ leaf_box, LevelRanges LR,
                                                             const int* __restrict__ red_off, const int2* __restrict__ red,
                                                             const C* __restrict__ scratch, C* __restrict__ phis) {
    const int2 tile = tiles[blockIdx.x];
    const int w = tile.x;
    const int l = leaf_level[w], b = leaf_box[w];
    const int t0 = LR.begin[l][b], t1 = LR.end[l][b];
    const int u = tile.y + threadIdx.x;
    if (t0 + u >= t1) return;
    C acc = cmake<C>(0, 0);
    for (int e = red_off[w]; e < red_off[w + 1]; ++e) {
        const int2 r = red[e];
        const C* blk = scratch + (unsigned)r.x;
        if (r.y < 0) acc = cadd(acc, blk[kP2PTile + u]);
        else if (u >= r.y && u < r.y + kP2PTile) acc = cadd(acc, blk[u - r.y]);
    }
    phis[t0 + u] = cadd(phis[t0 + u], acc);
}

// caller order (rows of stride ld) <-> Morton order (rows of stride n)
template <typename C>
__global__ void k_permute_in(int64_t n, int nrhs, int64_t ld, const int* __restrict__ perm, const C* __restrict__ q,
                             C* __restrict__ qs, int conj) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * nrhs) return;
    int64_t r = idx / n, i = idx % n;
    C v = q[r * ld + perm[i]];
    if (conj) v.y = -v.y;
    qs[idx] = v;
}

template <typename C>
__global__ void k_permute_out(int64_t n, int nrhs, int64_t ld, const int* __restrict__ perm, const C* __restrict__ phis,
                              C* __restrict__ phi, int conj) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * nrhs) return;
    int64_t r = idx / n, i = idx % n;
    C v = phis[idx];
    if (conj) v.y = -v.y;
    phi[r * ld + perm[i]] = v;
}

void permute_in(Plan& p, const void* q, void* qs, int nrhs, bool conj, int64_t ld) {
    int64_t tot = p.n * nrhs;
    if (ld < 0) ld = p.n;
    if (p.prec == MLFMA_PREC_FP64)
        k_permute_in<double2><<<nblk(tot, 256), 256, 0, p.stream>>>(p.n, nrhs, ld, p.perm, (const double2*)q, (double2*)qs, conj);
    else
        k_permute_in<float2><<<nblk(tot, 256), 256, 0, p.stream>>>(p.n, nrhs, ld, p.perm, (const float2*)q, (float2*)qs, conj);
    MLFMA_LAUNCH_CHECK();
}

void permute_out(Plan& p, const void* phis, void* phi, int nrhs, bool conj, int64_t ld) {
    int64_t tot = p.n * nrhs;
    if (ld < 0) ld = p.n;
    if (p.prec == MLFMA_PREC_FP64)
        k_permute_out<double2><<<nblk(tot, 256), 256, 0, p.stream>>>(p.n, nrhs, ld, p.perm, (const double2*)phis, (double2*)phi,
                                                                    conj);
    else
        k_permute_out<float2><<<nblk(tot, 256), 256, 0, p.stream>>>(p.n, nrhs, ld, p.perm, (const float2*)phis, (float2*)phi,
                                                                   conj);
    MLFMA_LAUNCH_CHECK();
}

template <typename R, int NR>
static void near_apply(Plan& p, const void* qs, void* phis, void* grads, bool timed = true) {
    using C = typename Cx<R>::T;
    LevelRanges LR;
    for (int l = 0; l <= kMaxLev; ++l) {
        LR.begin[l] = l <= p.nlev ? p.lev[l].begin : nullptr;
        LR.end[l] = l <= p.nlev ? p.lev[l].end : nullptr;
        LR.center[l] = l <= p.nlev ? p.lev[l].center : nullptr;
    }
    const int64_t n32 = p.n_small32, nmid = p.n_small - p.n_small32, sn = p.n;
    const R kpi = (R)(p.k / M_PI);
    const bool sym_pass = NR == 1 && !grads && p.n_tiles > 0 && p.n_sym_items > 0;
    StageTimer st(p, MLFMA_STAGE_P2P, 0, (n32 > 0) + (nmid > 0) + (p.n_tiles > 0) + 2 * sym_pass, timed);
    // with large leaves, the small leaves' kernels (whose single wave of warps ends on the
    // heaviest leaves) run on their own stream beside the large leaves' kernels, which write
    // other targets; sequential while stage timings are taken
    const cudaStream_t ns = p.stream;
    const bool sfork = p.sstream && !p.profiling && p.n_tiles > 0 && (n32 > 0 || nmid > 0);
    if (sfork) {
        MLFMA_CUDA(cudaEventRecord(p.ev_sfork, ns));
        MLFMA_CUDA(cudaStreamWaitEvent(p.sstream, p.ev_sfork, 0));
    }
    const cudaStream_t ss = sfork ? p.sstream : ns;
    if (n32 > 0) {
        if (grads)
            k_p2p<R, C, true, 1, false><<<nblk(n32, 4), 128, 0, ss>>>(
                n32, p.p2p_small, p.leaf_level, p.leaf_box, p.near_off, p.near_lev, p.near_box, LR, p.pos,
                (const C*)qs, sn, kpi, (C*)phis, (C*)grads);
        else
            k_p2p<R, C, false, NR, false><<<nblk(n32, 4), 128, 0, ss>>>(
                n32, p.p2p_small, p.leaf_level, p.leaf_box, p.near_off, p.near_lev, p.near_box, LR, p.pos,
                (const C*)qs, sn, kpi, (C*)phis, nullptr);
        MLFMA_LAUNCH_CHECK();
    }
    if (nmid > 0) {
        const int* mid = p.p2p_small + n32;
        if (grads)
            k_p2p<R, C, true, 1, true><<<nblk(nmid, 4), 128, 0, ss>>>(
                nmid, mid, p.leaf_level, p.leaf_box, p.near_off, p.near_lev, p.near_box, LR, p.pos, (const C*)qs, sn,
                kpi, (C*)phis, (C*)grads);
        else
            k_p2p<R, C, false, NR, true><<<nblk(nmid, 4), 128, 0, ss>>>(
                nmid, mid, p.leaf_level, p.leaf_box, p.near_off, p.near_lev, p.near_box, LR, p.pos, (const C*)qs, sn,
                kpi, (C*)phis, nullptr);
        MLFMA_LAUNCH_CHECK();
    }
    if (p.n_tiles > 0) {
        // one right-hand side without gradients: pairs of mutually near large leaves go through the
        // symmetric pass, the tiled kernel takes the rest of their near boxes
        const bool sym = NR == 1 && !grads && p.n_sym_items > 0;
        const int* off = sym ? p.asym_off : p.near_off;
        const int* nlv = sym ? p.asym_lev : p.near_lev;
        const int* nbx = sym ? p.asym_box : p.near_box;
        if (grads)
            k_p2p_tile<R, C, true, 1><<<(unsigned)p.n_tiles, kP2PTile, 0, p.stream>>>(
                p.p2p_tiles, p.leaf_level, p.leaf_box, off, nlv, nbx, LR, p.pos, (const C*)qs, sn, kpi, (C*)phis,
                (C*)grads);
        else
            k_p2p_tile<R, C, false, NR><<<(unsigned)p.n_tiles, kP2PTile, 0, p.stream>>>(
                p.p2p_tiles, p.leaf_level, p.leaf_box, off, nlv, nbx, LR, p.pos, (const C*)qs, sn, kpi, (C*)phis, nullptr);
        MLFMA_LAUNCH_CHECK();
        if (sym) {
            k_p2p_sym<R, C><<<(unsigned)p.n_sym_items, kP2PTile, 0, p.stream>>>(p.sym_items, p.leaf_level, p.leaf_box, LR,
                                                                               p.pos, (const C*)qs, kpi, (C*)p.sym_buf);
            MLFMA_LAUNCH_CHECK();
            k_p2p_sym_reduce<C><<<(unsigned)p.n_tiles, kP2PTile, 0, p.stream>>>(
                p.p2p_tiles, p.leaf_level, p.leaf_box, LR, p.sym_red_off, p.sym_red, (const C*)p.sym_buf, (C*)phis);
            MLFMA_LAUNCH_CHECK();
        }
    }
    if (sfork) {
        MLFMA_CUDA(cudaEventRecord(p.ev_sdone, p.sstream));
        MLFMA_CUDA(cudaStreamWaitEvent(ns, p.ev_sdone, 0));
    }
}

void near_only(Plan& p, const void* qs, void* phis, bool timed) {
    if (p.prec == MLFMA_PREC_FP64) near_apply<double, 1>(p, qs, phis, nullptr, timed);
    else near_apply<float, 1>(p, qs, phis, nullptr, timed);
}

// nr right-hand sides (q and phi n apart): 1, or kMaxNR without gradients
// One pass of nr right-hand sides: the near field writes phis (and grads), the far field's L2O
// adds to them.  The two are independent until then, so unless stage timings are being taken
// the near field runs on its own stream beside the far field's upward and downward passes and
// the plan stream waits for it before the first L2O (the fork and the join are events, so a
// captured apply keeps them as graph edges).
void apply_pipeline(Plan& p, const void* qs, void* phis, void* grads, int nr) {
    if (nr != 1 && !(nr == kMaxNR && !grads)) fail(MLFMA_ERR_INVALID_ARG, "right-hand sides per pass %d", nr);
    const bool fork = p.nstream && !p.profiling;
    const cudaStream_t main = p.stream;
    if (fork) {
        MLFMA_CUDA(cudaEventRecord(p.ev_nfork, main));
        MLFMA_CUDA(cudaStreamWaitEvent(p.nstream, p.ev_nfork, 0));
        p.stream = p.nstream;
    }
    try {
        if (nr == kMaxNR) {
            if (p.prec == MLFMA_PREC_FP64) near_apply<double, kMaxNR>(p, qs, phis, nullptr);
            else near_apply<float, kMaxNR>(p, qs, phis, nullptr);
        } else {
            if (p.prec == MLFMA_PREC_FP64) near_apply<double, 1>(p, qs, phis, grads);
            else near_apply<float, 1>(p, qs, phis, grads);
        }
        if (p.near_dump)
            MLFMA_CUDA(cudaMemcpyAsync(p.near_dump, phis, p.n * csize(p), cudaMemcpyDeviceToDevice, p.stream));
        if (fork) MLFMA_CUDA(cudaEventRecord(p.ev_near, p.nstream));
    } catch (...) {
        p.stream = main;
        throw;
    }
    p.stream = main;
    far_apply(p, qs, phis, grads, nr, fork ? p.ev_near : nullptr);
    if (fork) MLFMA_CUDA(cudaStreamWaitEvent(main, p.ev_near, 0));   // no far field: join here
}

template <typename C>
__global__ void k_permute_out3(int64_t n, int nrhs, int64_t ld, const int* __restrict__ perm, const C* __restrict__ gs,
                               C* __restrict__ g) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * nrhs * 3) return;
    int64_t a = idx % 3, t = idx / 3;
    int64_t r = t / n, i = t % n;
    g[(r * ld + perm[i]) * 3 + a] = gs[idx];
}

void permute_out3(Plan& p, const void* gs, void* g, int nrhs, int64_t ld) {
    int64_t tot = p.n * nrhs * 3;
    if (ld < 0) ld = p.n;
    if (p.prec == MLFMA_PREC_FP64)
        k_permute_out3<double2><<<nblk(tot, 256), 256, 0, p.stream>>>(p.n, nrhs, ld, p.perm, (const double2*)gs, (double2*)g);
    else
        k_permute_out3<float2><<<nblk(tot, 256), 256, 0, p.stream>>>(p.n, nrhs, ld, p.perm, (const float2*)gs, (float2*)g);
    MLFMA_LAUNCH_CHECK();
}

// grad_r[i][a] = sum_r Re[conj(g_ri) gphi_ri[a] + q_ri gpsi_ri[a]]: the derivative of a real loss
// with respect to the position r_i (reverse mode of phi = A(r) q; g = dL/dRe phi + i dL/dIm phi,
// psi = A conj(g)).  One thread per (point, component), caller order, FP64 result.
template <typename C>
__global__ void k_position_grad(int64_t n, int nrhs, const C* __restrict__ q, const C* __restrict__ g,
                                const C* __restrict__ gphi, const C* __restrict__ gpsi, double* __restrict__ grad_r) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= 3 * n) return;
    const int64_t i = idx / 3;
    double acc = 0.0;
    for (int r = 0; r < nrhs; ++r) {
        const C gv = g[r * n + i], qv = q[r * n + i];
        const C a = gphi[r * 3 * n + idx], b = gpsi[r * 3 * n + idx];
        // Re(conj(g) a) + Re(q b)
        acc += (double)gv.x * (double)a.x + (double)gv.y * (double)a.y + (double)qv.x * (double)b.x -
               (double)qv.y * (double)b.y;
    }
    grad_r[idx] = acc;
}

void position_grad(const Plan& p, int64_t n, int nrhs, const void* q, const void* g, const void* gphi, const void* gpsi,
                   double* grad_r, cudaStream_t s) {
    const int64_t tot = 3 * n;
    if (p.prec == MLFMA_PREC_FP64)
        k_position_grad<double2><<<nblk(tot, 256), 256, 0, s>>>(n, nrhs, (const double2*)q, (const double2*)g,
                                                                (const double2*)gphi, (const double2*)gpsi, grad_r);
    else
        k_position_grad<float2><<<nblk(tot, 256), 256, 0, s>>>(n, nrhs, (const float2*)q, (const float2*)g,
                                                               (const float2*)gphi, (const float2*)gpsi, grad_r);
    MLFMA_LAUNCH_CHECK();
}

// ============================================================== FP64 direct sum at selected targets
__global__ void k_direct_fp64(const double* __restrict__ pts, int64_t n, const double2* __restrict__ q, double k,
                              const int64_t* __restrict__ tg, double2* __restrict__ phi) {
    __shared__ double sre[256], sim[256];
    const int64_t i = tg[blockIdx.x];
    const double xi = pts[3 * i], yi = pts[3 * i + 1], zi = pts[3 * i + 2];
    double re = 0, im = 0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        if (j == i) continue;
        double dx = xi - pts[3 * j], dy = yi - pts[3 * j + 1], dz = zi - pts[3 * j + 2];
        double r = sqrt(dx * dx + dy * dy + dz * dz);
        if (r == 0.0) continue;
        double s, c;
        sincos(k * r, &s, &c);
        double2 qj = q[j];
        re += (qj.x * c - qj.y * s) / r;
        im += (qj.x * s + qj.y * c) / r;
    }
    sre[threadIdx.x] = re;
    sim[threadIdx.x] = im;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st) { sre[threadIdx.x] += sre[threadIdx.x + st]; sim[threadIdx.x] += sim[threadIdx.x + st]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) phi[blockIdx.x] = make_double2(sre[0], sim[0]);
}

void direct_fp64(const double* pts, int64_t n, const void* q, double k, const int64_t* tg, int64_t nt, void* phi,
                 cudaStream_t s) {
    if (nt <= 0) return;
    k_direct_fp64<<<(unsigned)nt, 256, 0, s>>>(pts, n, (const double2*)q, k, tg, (double2*)phi);
    MLFMA_LAUNCH_CHECK();
}

}  // namespace mlfma
