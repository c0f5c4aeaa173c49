// Far-field stages of the MLFMA apply (Sec. 2, five stages; Sec. 3.2.1-3.2.5).
//
//   C2M  F_b(p)  = sum_{j in b} q_j e^{-ik khat_p.(r_j - c_b)}                  (leaves)
//   M2M  F_P(p') = sum_c e^{-ik khat_p'.(c_c - c_P)} [I_{c->P} F_c](p')          (Alg. 1: interpolate,
//                                                                                 shift, aggregate)
//   M2L  G_t(p)  = sum_{s in V(t)} T_{c_t - c_s}(p) F_s(p)                        (Alg. 2)
//   L2L  G_c    += W_c^{-1} I^T W_P [e^{+ik khat.(c_c - c_P)} G_P]                (shift, anterpolate, add)
//   L2O  phi_i  += (ik/4pi) sum_p w_p e^{ik khat_p.(r_i - c_b)} G_b(p)            (leaves)
//
// Interpolation I_{c->P} (global, per Fourier mode): forward DFT in phi on the child
// grid (modes |m| <= Lc), theta map A_|m| per mode, inverse DFT onto the parent phi
// nodes; both phi transforms are mixed-radix FFTs in shared memory.  The shift to the parent centre factors into a theta-only part
// e^{-ik cos(theta') dz} (applied per mode, before the inverse DFT, which lets the
// two children stacked in z share one inverse DFT) and a theta-phi part applied on
// the parent grid.  Anterpolation is the weighted transpose of the same steps.
#include <cstdio>

#include "common.cuh"

namespace mlfma {

// sin and cos of the leaf phases (C2M, L2O).  complex64: x is reduced to [-pi, pi] by a
// two-constant Cody-Waite step, x - n 2pi with 2pi = hi + lo (hi the float nearest 2pi, lo
// the remainder; the reduction adds less than 1.2e-7 for |x| <= 200, no more than the
// rounding of x itself beyond), then the SFU approximations, whose documented absolute
// error on [-pi, pi] is 2^-21.4.  complex128: the libm-accurate sincos.
__device__ __forceinline__ void sc(float x, float& s, float& c) {
    const float n = rintf(x * 0.159154936671257f);
    float r = fmaf(-n, 6.28318548202514648f, x);
    r = fmaf(-n, -1.74845553146952e-7f, r);
    __sincosf(r, &s, &c);
}
__device__ __forceinline__ void sc(double x, double& s, double& c) { sincos(x, &s, &c); }

static inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

// rows of a tile: as many as fit in ``budget`` complex slots at ``per_row`` each, in [1, nrows]
static inline int tile_rows(int nrows, int budget, int per_row) {
    int r = budget > 0 ? budget / per_row : 1;
    return std::max(1, std::min(nrows, r));
}
// the smallest tile that covers nrows in as many tiles as tiles of rmax do
// per-parent row tiles below this height take the quadrant-sequential kernels
constexpr int kParentMinRows = 16;

static inline int balanced_rows(int nrows, int rmax) {
    const int nt = (nrows + rmax - 1) / rmax;
    return (nrows + nt - 1) / nt;
}

// ============================================================== C2M (warp per leaf)
constexpr int kC2MPass = 4;   // samples per lane per pass

// NR right-hand sides share each exponential: charges qs[r sn + j], signatures F[r sF + b K + p].
// The leaf's points (at most kSmallLeaf) and charges are staged in shared memory once; each
// pass then covers 32 kC2MPass samples with every point.
template <typename R, typename C, int NR>
__global__ void __launch_bounds__(128) k_c2m(int64_t nleaf, const int* __restrict__ leaf_box, const int* __restrict__ begin,
                                             const int* __restrict__ end, const double* __restrict__ center,
                                             const double* __restrict__ pos, const C* __restrict__ qs, int64_t sn,
                                             const R* __restrict__ dirs, int64_t K, R k, C* __restrict__ F, int64_t sF) {
    __shared__ R sp[4][kSmallLeaf][3];
    __shared__ C sq[4][NR][kSmallLeaf];
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t w = (int64_t)blockIdx.x * 4 + wl;
    if (w >= nleaf) return;
    const int b = leaf_box[w];
    const int b0 = begin[b], np = min(end[b] - b0, kSmallLeaf);
    const double cx = center[3 * b], cy = center[3 * b + 1], cz = center[3 * b + 2];
    for (int t = lane; t < np; t += 32) {
        const int64_t j = b0 + t;
        sp[wl][t][0] = (R)(pos[3 * j] - cx);
        sp[wl][t][1] = (R)(pos[3 * j + 1] - cy);
        sp[wl][t][2] = (R)(pos[3 * j + 2] - cz);
#pragma unroll
        for (int r = 0; r < NR; ++r) sq[wl][r][t] = qs[r * sn + j];
    }
    __syncwarp();
    C* Fb = F + (int64_t)b * K;
    for (int64_t p0 = 0; p0 < K; p0 += 32 * kC2MPass) {
        C acc[kC2MPass][NR];
        R d[kC2MPass][3];
#pragma unroll
        for (int u = 0; u < kC2MPass; ++u) {
#pragma unroll
            for (int r = 0; r < NR; ++r) acc[u][r] = cmake<C>(0, 0);
            int64_t p = p0 + lane + 32 * u;
            int64_t pp = p < K ? p : K - 1;
            d[u][0] = -k * dirs[4 * pp]; d[u][1] = -k * dirs[4 * pp + 1]; d[u][2] = -k * dirs[4 * pp + 2];
        }
        for (int t = 0; t < np; ++t) {
            const R x = sp[wl][t][0], y = sp[wl][t][1], z = sp[wl][t][2];
#pragma unroll
            for (int u = 0; u < kC2MPass; ++u) {
                if (p0 + 32 * u >= K) break;              // warp-uniform: no sample of this slot
                R ph = d[u][0] * x + d[u][1] * y + d[u][2] * z;
                R s, c;
                sc(ph, s, c);
                const C e = cmake<C>(c, s);
#pragma unroll
                for (int r = 0; r < NR; ++r) cfma(acc[u][r], sq[wl][r][t], e);
            }
        }
#pragma unroll
        for (int u = 0; u < kC2MPass; ++u) {
            int64_t p = p0 + lane + 32 * u;
            if (p < K)
#pragma unroll
                for (int r = 0; r < NR; ++r) Fb[r * sF + p] = acc[u][r];
        }
    }
}

// ============================================================== L2O (warp per leaf, lanes = point x slice)
// GRAD: also grad phi_i += (ik/4pi) sum_p w_p (ik khat_p) e^{ik khat_p.(r_i - c_b)} G_b(p).
// NR right-hand sides share each exponential (GRAD only with NR = 1): G[r sF + b K + p],
// phis[r sn + j].
template <typename R, typename C, bool GRAD, int NR>
__global__ void __launch_bounds__(128) k_l2o(int64_t nleaf, const int* __restrict__ leaf_box, const int* __restrict__ begin,
                                             const int* __restrict__ end, const double* __restrict__ center,
                                             const double* __restrict__ pos, const R* __restrict__ dirs, int64_t K, R k,
                                             const C* __restrict__ G, int64_t sF, C* __restrict__ phis, int64_t sn,
                                             C* __restrict__ grads) {
    static_assert(!GRAD || NR == 1, "gradients take one right-hand side per pass");
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t w = (int64_t)blockIdx.x * 4 + wl;
    if (w >= nleaf) return;
    (void)wl;
    const int b = leaf_box[w];
    const int b0 = begin[b], b1 = end[b];
    const double cx = center[3 * b], cy = center[3 * b + 1], cz = center[3 * b + 2];
    const C* Gb = G + (int64_t)b * K;
    for (int j0 = b0; j0 < b1; j0 += 32) {
        int np = min(32, b1 - j0);
        int P = 1;
        while (P < np) P <<= 1;
        const int S = 32 / P;
        const int tp = lane & (P - 1), sl = lane / P;
        const int j = j0 + tp;
        R x = 0, y = 0, z = 0;
        if (tp < np) {
            x = (R)(pos[3 * (int64_t)j] - cx);
            y = (R)(pos[3 * (int64_t)j + 1] - cy);
            z = (R)(pos[3 * (int64_t)j + 2] - cz);
        }
        C acc[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[r] = cmake<C>(0, 0);
        C ga[3] = {cmake<C>(0, 0), cmake<C>(0, 0), cmake<C>(0, 0)};
        for (int64_t p = sl; p < K; p += S) {
            R ph = k * (dirs[4 * p] * x + dirs[4 * p + 1] * y + dirs[4 * p + 2] * z);
            R s, c;
            sc(ph, s, c);
            R wp = dirs[4 * p + 3];
            if (!GRAD) {
                const C e = cmake<C>(wp * c, wp * s);
#pragma unroll
                for (int r = 0; r < NR; ++r) cfma(acc[r], e, Gb[r * sF + p]);
            } else {
                const C term = cmul(cmake<C>(wp * c, wp * s), Gb[p]);
                acc[0] = cadd(acc[0], term);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const R d = dirs[4 * p + a];
                    ga[a] = cadd(ga[a], cmake<C>(d * term.x, d * term.y));
                }
            }
        }
        for (int o = 16; o >= P; o >>= 1) {
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
        if (sl == 0 && tp < np) {
            // (ik / 4 pi) * acc
            const R f = k / (R)(4.0 * M_PI);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                C v = phis[r * sn + j];
                v.x += -f * acc[r].y;
                v.y += f * acc[r].x;
                phis[r * sn + j] = v;
            }
            if (GRAD) {
                // (ik / 4 pi) (ik) = -k^2 / (4 pi)
                const R f2 = -k * k / (R)(4.0 * M_PI);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    C g = grads[3 * (int64_t)j + a];
                    g.x += f2 * ga[a].x;
                    g.y += f2 * ga[a].y;
                    grads[3 * (int64_t)j + a] = g;
                }
            }
        }
    }
}


// ============================================================== C2M / L2O for leaves with many points
// C2M: one CTA per (leaf, chunk of 128 samples), one sample per thread, the leaf's points
// staged through shared memory.
template <typename R, typename C, int NR>
__global__ void __launch_bounds__(128) k_c2m_big(const int* __restrict__ leaves, const int* __restrict__ begin,
                                                 const int* __restrict__ end, const double* __restrict__ center,
                                                 const double* __restrict__ pos, const C* __restrict__ qs, int64_t sn,
                                                 const R* __restrict__ dirs, int64_t K, R k, C* __restrict__ F, int64_t sF) {
    __shared__ R sx[256], sy[256], sz[256];
    __shared__ C sq[NR][256];
    const int b = leaves[blockIdx.x];
    const int b0 = begin[b], b1 = end[b];
    const double cx = center[3 * b], cy = center[3 * b + 1], cz = center[3 * b + 2];
    const int64_t p = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    const int64_t pp = p < K ? p : K - 1;
    const R dx = -k * dirs[4 * pp], dy = -k * dirs[4 * pp + 1], dz = -k * dirs[4 * pp + 2];
    C acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = cmake<C>(0, 0);
    for (int j0 = b0; j0 < b1; j0 += 256) {
        const int cnt = min(256, b1 - j0);
        __syncthreads();
        for (int m = threadIdx.x; m < cnt; m += blockDim.x) {
            const int64_t j = j0 + m;
            sx[m] = (R)(pos[3 * j] - cx);
            sy[m] = (R)(pos[3 * j + 1] - cy);
            sz[m] = (R)(pos[3 * j + 2] - cz);
#pragma unroll
            for (int r = 0; r < NR; ++r) sq[r][m] = qs[r * sn + j];
        }
        __syncthreads();
#pragma unroll 4
        for (int m = 0; m < cnt; ++m) {
            R s, c;
            sc(dx * sx[m] + dy * sy[m] + dz * sz[m], s, c);
            const C e = cmake<C>(c, s);
#pragma unroll
            for (int r = 0; r < NR; ++r) cfma(acc[r], sq[r][m], e);
        }
    }
    if (p < K)
#pragma unroll
        for (int r = 0; r < NR; ++r) F[r * sF + (int64_t)b * K + p] = acc[r];
}

// L2O: one CTA per tile of kP2PTile points of a leaf, one point per thread, the leaf's
// samples (direction, weight, G) staged through shared memory.
template <typename R, typename C, bool GRAD, int NR>
__global__ void __launch_bounds__(128) k_l2o_big(const int2* __restrict__ tiles, const int* __restrict__ begin,
                                                 const int* __restrict__ end, const double* __restrict__ center,
                                                 const double* __restrict__ pos, const R* __restrict__ dirs, int64_t K, R k,
                                                 const C* __restrict__ G, int64_t sF, C* __restrict__ phis, int64_t sn,
                                                 C* __restrict__ grads) {
    static_assert(!GRAD || NR == 1, "gradients take one right-hand side per pass");
    __shared__ R sd[256][4];
    __shared__ C sg[NR][256];
    const int2 tile = tiles[blockIdx.x];
    const int b = tile.x;
    const int i = begin[b] + tile.y + threadIdx.x;
    const bool valid = i < end[b];
    const double cx = center[3 * b], cy = center[3 * b + 1], cz = center[3 * b + 2];
    R x = 0, y = 0, z = 0;
    if (valid) {
        x = (R)(pos[3 * (int64_t)i] - cx);
        y = (R)(pos[3 * (int64_t)i + 1] - cy);
        z = (R)(pos[3 * (int64_t)i + 2] - cz);
    }
    const C* Gb = G + (int64_t)b * K;
    C acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = cmake<C>(0, 0);
    C ga[3] = {cmake<C>(0, 0), cmake<C>(0, 0), cmake<C>(0, 0)};
    for (int64_t p0 = 0; p0 < K; p0 += 256) {
        const int cnt = (int)min((int64_t)256, K - p0);
        __syncthreads();
        for (int m = threadIdx.x; m < cnt; m += blockDim.x) {
#pragma unroll
            for (int a = 0; a < 4; ++a) sd[m][a] = dirs[4 * (p0 + m) + a];
#pragma unroll
            for (int r = 0; r < NR; ++r) sg[r][m] = Gb[r * sF + p0 + m];
        }
        __syncthreads();
        for (int m = 0; m < cnt; ++m) {
            R s, c;
            sc(k * (sd[m][0] * x + sd[m][1] * y + sd[m][2] * z), s, c);
            const R wp = sd[m][3];
            if (!GRAD) {
                const C e = cmake<C>(wp * c, wp * s);
#pragma unroll
                for (int r = 0; r < NR; ++r) cfma(acc[r], e, sg[r][m]);
            } else {
                const C term = cmul(cmake<C>(wp * c, wp * s), sg[0][m]);
                acc[0] = cadd(acc[0], term);
#pragma unroll
                for (int a = 0; a < 3; ++a) ga[a] = cadd(ga[a], cmake<C>(sd[m][a] * term.x, sd[m][a] * term.y));
            }
        }
    }
    if (valid) {
        const R f = k / (R)(4.0 * M_PI);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            C v = phis[r * sn + i];
            v.x += -f * acc[r].y;
            v.y += f * acc[r].x;
            phis[r * sn + i] = v;
        }
        if (GRAD) {
            const R f2 = -k * k / (R)(4.0 * M_PI);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                C g = grads[3 * (int64_t)i + a];
                g.x += f2 * ga[a].x;
                g.y += f2 * ga[a].y;
                grads[3 * (int64_t)i + a] = g;
            }
        }
    }
}

// ============================================================== M2L (Eq. 9)
// G_t = sum over s in V(t) of T_{t-s} F_s, organised per parent P: a warp takes P and a
// 32-sample slice of the grid (p = tile * 32 + lane), walks the list of P's colleagues'
// children that are far from some child of P (entries (src * K) << 32 | far-children mask
// << 16 | base), loads each source's samples once and adds them to every child of P.  The
// operators of the slice are staged in shared memory as the full 7^3 offset cube Ts[343][32]
// (the 27 near rows zero), so the row of a (child, source) pair is base(source) + c(child),
// and a child near the source reads a zero row: the child slots need no predicates.  The
// child count NT is a template argument, so each entry costs exactly NT child slots.  NR
// right-hand sides (signatures r sF apart) share every operator load.
constexpr int kM2LParentsPerWarp = 4;

// cp.async of B bytes global -> shared; v = false fills the B bytes with zeros (nothing is read)
template <int B>
__device__ __forceinline__ void cp_async_zfill(void* dst, const void* src, bool v) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    const int n = v ? B : 0;
    if constexpr (B == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(src), "r"(n) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(sa), "l"(src), "n"(B), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <typename C, int NR, int NT>
__device__ __forceinline__ void m2l_parent(int lane, int t0, const uint64_t* __restrict__ ckey,
                                           const unsigned long long* __restrict__ le, int ne, const C* Fp, int64_t sF,
                                           const C* Tl, bool ok, int64_t K, int64_t p0, C* __restrict__ G,
                                           C* red) {
    int cr[NT];     // child part of the row index, times 32
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const int ct = (int)(ckey[t0 + t] & 7);
        cr[t] = ((ct & 1) + 7 * ((ct >> 1) & 1) + 49 * (ct >> 2)) * 32;
    }
    C acc[NT][NR];
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[t][r] = cmake<C>(0, 0);
    // every lane reads each list entry from the same address (one broadcast load); each entry
    // costs NT child slots without predicates: a child that is not far from the source reads one
    // of the 27 zero (near-offset) rows of the cube, which adds exactly nothing
    for (int j = 0; j < ne; ++j) {
        const unsigned long long w = __ldg(le + j);
        const unsigned lo = (unsigned)w;
        const C* fs = Fp + (unsigned)(w >> 32);
        C f[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) f[r] = fs[r * sF];
        const C* Tb = Tl + (lo & 511u) * 32;
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const C tv = Tb[cr[t]];
#pragma unroll
            for (int r = 0; r < NR; ++r) cfma(acc[t][r], tv, f[r]);
        }
    }
    if (red) {                                    // a partial sum over part of the list
#pragma unroll
        for (int t = 0; t < NT; ++t)
#pragma unroll
            for (int r = 0; r < NR; ++r) red[(t * NR + r) * 32 + lane] = acc[t][r];
    } else if (ok) {
#pragma unroll
        for (int t = 0; t < NT; ++t)
#pragma unroll
            for (int r = 0; r < NR; ++r) G[r * sF + (int64_t)(t0 + t) * K + p0 + lane] = acc[t][r];
    }
}

constexpr long long kM2LWaitLimit = 1ll << 22;

__device__ __forceinline__ bool m2l_bar_wait(uint32_t bar, uint32_t phase, long long limit = kM2LWaitLimit) {
    for (long long i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Lagrange weight of node J among the nodes 0 .. kOpOrder - 1: 1 / prod_{m != J} (J - m)
template <int J> __host__ __device__ constexpr double lagrange_c() {
    double d = 1.0;
    for (int m = 0; m < kOpOrder; ++m)
        if (m != J) d *= (double)(J - m);
    return 1.0 / d;
}

// acc += sum_{j <= J} l_j(t) b[j] and acm += sum_{j <= J} l_j(t) bm[-j], l_j(t) = c_j
// prod_{m < j} (t - m) prod_{m > j} (t - m): pre[j] holds the first product, suf the second
// (built from the top node down)
template <typename R, typename C, int J>
__device__ __forceinline__ void lagrange_terms(C& acc, C& acm, const C* __restrict__ b, const C* __restrict__ bm,
                                               const R (&pre)[kOpOrder], R suf, R t) {
    constexpr double c = lagrange_c<J>();
    const R w = pre[J] * suf * (R)c;
    const C v = __ldg(b + J), vm = __ldg(bm - J);
    acc.x = fma(w, v.x, acc.x);
    acc.y = fma(w, v.y, acc.y);
    acm.x = fma(w, vm.x, acm.x);
    acm.y = fma(w, vm.y, acm.y);
    if constexpr (J > 0) lagrange_terms<R, C, J - 1>(acc, acm, b, bm, pre, suf * (t - (R)J), t);
}

// Sampled operators (Sec. 3.2.3, "Translation Operators": sample the operators, interpolate
// them): T of the offset d (box units) and of its antipode -d at the sample direction khat,
// from the row of |d|^2 of the level's table (entry i + kOpOrder: T at psi_i = i pi / S), by the
// kOpOrder-point Lagrange interpolant on the nodes n_j = floor(u) - kOpOrder/2 + 1 + j,
// u = psi S / pi, psi = atan2(|d x khat|, d . khat) (accurate at every angle, unlike acos of the
// dot product).  The antipode's angle is pi - psi: its stencil is the mirror image, nodes S - n_j
// with the same weights, so the angle and the weights serve both.  S / pi = inv_h + inv_lo
// (inv_lo: what rounding inv_h dropped), and the position within the stencil is
// fma(psi, inv_h, -i) + psi inv_lo, so it keeps the accuracy of psi instead of that of u (whose
// rounding at u ~ 10^3 would move the node by 1e-4 spacings in FP32).  The node index is
// clamped to [0, S], the range psi in [0, pi] gives, so every read stays in the row whatever
// the arithmetic returns.
template <typename R, typename C>
__device__ __forceinline__ void sampled_operator_pair(const C* __restrict__ row, int S, R inv_h, R inv_lo, R dx, R dy,
                                                      R dz, R kx, R ky, R kz, C& v, C& vm) {
    const R cx = dy * kz - dz * ky, cy = dz * kx - dx * kz, cz = dx * ky - dy * kx;
    R psi;
    if constexpr (sizeof(R) == 4) psi = atan2f(sqrtf(cx * cx + cy * cy + cz * cz), dx * kx + dy * ky + dz * kz);
    else psi = atan2(sqrt(cx * cx + cy * cy + cz * cz), dx * kx + dy * ky + dz * kz);
    const int i = min(max((int)floor(psi * inv_h), 0), S);
    const R t = fma(psi, inv_h, -(R)i) + psi * inv_lo + (R)(kOpOrder / 2 - 1);   // among the nodes 0 .. kOpOrder - 1
    R pre[kOpOrder];
    pre[0] = 1;
#pragma unroll
    for (int j = 1; j < kOpOrder; ++j) pre[j] = pre[j - 1] * (t - (R)(j - 1));
    v = cmake<C>(0, 0);
    vm = cmake<C>(0, 0);
    const int n0 = i - (kOpOrder / 2 - 1);              // node 0; entry n + kOpOrder holds psi_n
    lagrange_terms<R, C, kOpOrder - 1>(v, vm, row + n0 + kOpOrder, row + (S - n0) + kOpOrder, pre, (R)1, t);
}

// SMP: the level keeps sampled operators (T1, T1n entries per row, inv_h + inv_lo = S / pi,
// sample directions dirs [K][4]); the CTA computes its operator slice from them instead of
// copying it.
template <typename R, typename C, int NR, int NW, bool SMP>
__global__ void __launch_bounds__(32 * NW, 1) k_m2l(int64_t npar, const int* __restrict__ pcb, const int* __restrict__ pce,
                                                   const int* __restrict__ loff, const unsigned long long* __restrict__ lsrc,
                                                   const uint64_t* __restrict__ ckey, const __grid_constant__ CUtensorMap tmT,
                                                   const C* __restrict__ T1, int T1n, R inv_h, R inv_lo,
                                                   const R* __restrict__ dirs,
                                                   const C* __restrict__ F, int64_t K, int64_t sF, C* __restrict__ G,
                                                   int Q, int* __restrict__ err, long long wait_first) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t tbar;
    // operator slice Ts[344][32] at a 128-byte boundary (TMA destination)
    C* Ts = reinterpret_cast<C*>(smem_raw + ((128 - ((uintptr_t)smem_raw & 127)) & 127));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t p0 = (int64_t)blockIdx.y * 32;
    // Q = 1: a warp takes kM2LParentsPerWarp parents in turn.  Q > 1 (levels with few, wide
    // parents): Q warps share a parent, each summing a contiguous Q-th of its list into shared
    // memory after the operator slice, and the first of them adds the Q partial sums.
    const int PPC = Q > 1 ? NW / Q : NW * kM2LParentsPerWarp;    // parents per CTA
    const int64_t P0 = (int64_t)blockIdx.x * PPC;
    if constexpr (SMP) {
        // row r of the slice = offset (r % 7 - 3, r / 7 % 7 - 3, r / 49 - 3), lane = sample p0 + lane;
        // near rows (|d|^2 <= 3), row 343 and samples past K stay zero
        const int64_t ps = p0 + lane;
        R kx = 0, ky = 0, kz = 0;
        if (ps < K) {
            kx = dirs[4 * ps];
            ky = dirs[4 * ps + 1];
            kz = dirs[4 * ps + 2];
        }
        // rows r and 342 - r hold the offsets d and -d (one interpolation stencil); row 171 is
        // the zero offset
        const int S = T1n - 2 * kOpOrder - 1;
        for (int r = warp; r <= 171; r += NW) {
            const int dx = r % 7 - 3, dy = r / 7 % 7 - 3, dz = r / 49 - 3;
            const int d2 = dx * dx + dy * dy + dz * dz;
            C v = cmake<C>(0, 0), vm = cmake<C>(0, 0);
            if (d2 >= 4 && ps < K)
                sampled_operator_pair<R, C>(T1 + (size_t)d2 * T1n, S, inv_h, inv_lo, (R)dx, (R)dy, (R)dz, kx, ky, kz, v,
                                            vm);
            Ts[r * 32 + lane] = v;
            Ts[(342 - r) * 32 + lane] = vm;
        }
        if (warp == 0) Ts[343 * 32 + lane] = cmake<C>(0, 0);
        __syncthreads();
    } else {
        // stage the slice with two TMA boxes of kTBoxRows rows (rows 343 and samples past K read as
        // zero) completing on one mbarrier
        const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&tbar);
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            constexpr uint32_t box = kTBoxRows * 32 * sizeof(C);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(2 * box) : "memory");
            const int x = (int)(p0 * (int64_t)(sizeof(C) / 8));
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const uint32_t dst = (uint32_t)__cvta_generic_to_shared(Ts + b * kTBoxRows * 32);
                asm volatile(
                    "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                    "[%4];\n" ::"r"(dst),
                    "l"(reinterpret_cast<uint64_t>(&tmT)), "r"(x), "r"(b * kTBoxRows), "r"(bar)
                    : "memory");
            }
        }
        if (!__syncthreads_and(m2l_bar_wait(bar, 0, wait_first))) {
            if (threadIdx.x == 0) atomicExch(err, 2);
            m2l_bar_wait(bar, 0);                     // normal limit: let the copies in flight land
            return;
        }
    }
    const bool ok = p0 + lane < K;
    const C* Fp = F + (ok ? p0 + lane : K - 1);       // lane's sample; + (src * K) per source
    const C* Tl = Ts + lane;
    C* red = Q > 1 ? Ts + 2 * kTBoxRows * 32 + (size_t)warp * 8 * NR * 32 : nullptr;   // [warp][8][NR][32]
    const int nround = Q > 1 ? 1 : kM2LParentsPerWarp;
    for (int pw = 0; pw < nround; ++pw) {
        const int64_t P = Q > 1 ? P0 + warp % PPC : P0 + (int64_t)pw * NW + warp;
        if (P >= npar) break;
        const int t0 = pcb[P], nt = pce[P] - t0;
        int e0 = loff[P], ne = loff[P + 1] - e0;
        if (Q > 1) {
            const int q = warp / PPC;
            const int a = (int)((int64_t)ne * q / Q), b = (int)((int64_t)ne * (q + 1) / Q);
            e0 += a;
            ne = b - a;
        }
        const unsigned long long* le = lsrc + e0;
        switch (nt) {
#define M2L_NT(n) case n: m2l_parent<C, NR, n>(lane, t0, ckey, le, ne, Fp, sF, Tl, ok, K, p0, G, red); break;
            M2L_NT(1) M2L_NT(2) M2L_NT(3) M2L_NT(4) M2L_NT(5) M2L_NT(6) M2L_NT(7) M2L_NT(8)
#undef M2L_NT
            default: break;
        }
    }
    if (Q > 1) {
        __syncthreads();
        const int64_t P = P0 + warp;
        if (warp < PPC && P < npar && ok) {
            const int t0 = pcb[P], nt = pce[P] - t0;
            const C* r0 = Ts + 2 * kTBoxRows * 32;
            for (int t = 0; t < nt; ++t)
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    C v = cmake<C>(0, 0);
                    for (int q = 0; q < Q; ++q) {
                        const C u = r0[(((size_t)(q * PPC + warp) * 8 + t) * NR + r) * 32 + lane];
                        v.x += u.x;
                        v.y += u.y;
                    }
                    G[r * sF + (int64_t)(t0 + t) * K + p0 + lane] = v;
                }
        }
    }
}

// warps per CTA sharing the operator slice (88 KB complex64, 176 KB complex128): as many as
// the registers of the accumulators (8 children x NR right-hand sides) allow
template <typename C, int NR> struct M2LShape {
    static constexpr int NW = sizeof(C) == 8 ? (NR == 1 ? 32 : 16) : (NR == 1 ? 16 : 8);
};

template <typename R, typename C>
static size_t m2l_smem() { return (size_t)2 * kTBoxRows * 32 * sizeof(C) + 128; }

// list split of a level (see k_m2l): complex64 levels with K >= 49152 samples (L >= 156: the
// widest top levels, which hold few parents, so most warps of a CTA would idle and each
// source load's latency would be exposed).  The rule depends on K alone, so a level splits
// the same way in every plan that holds it (batched plans stay bit-identical to single ones).
// On the 2^20-point sphere the 8-parent level 3 drops from 305 to 197 us; at the 56-parent
// level 4 (K = 22050) the split was slower (157 -> 301 us: 7x the operator-slice loads).
template <typename C, int NR>
static int m2l_split(int64_t K) { return sizeof(C) == 8 && K >= 49152 ? 4 : 1; }

// ---- the ragged last sample slice (K mod 32 = w samples, 0 < w <= 16, one right-hand side)
// In k_m2l a warp walks a parent's whole list for one 32-sample slice, so a last slice holding
// w valid samples leaves 32 - w lanes idle (on the 2^20 sphere's leaf level, K = 162: 2 of
// 32).  Here lane (g, s) takes sample K - w + s of parent g among 32 / W parents per warp (W:
// the smallest power of two >= w).  Each lane walks its own parent's list, so the warp runs the
// longest of its parents' lists; the child count is a runtime bound over eight predicated
// slots.  The slice of the operators (343 rows x W samples, zero past K) is staged with plain
// loads.  Per sample the list order and the FMA sequence are those of k_m2l, so the results
// are identical.
constexpr int kM2LTailWarps = 8;

template <typename C, int W>
__global__ void __launch_bounds__(32 * kM2LTailWarps) k_m2l_tail(int64_t npar, const int* __restrict__ pcb,
                                                                 const int* __restrict__ pce, const int* __restrict__ loff,
                                                                 const unsigned long long* __restrict__ lsrc,
                                                                 const uint64_t* __restrict__ ckey, const C* __restrict__ T,
                                                                 const C* __restrict__ F, int64_t K, int w,
                                                                 C* __restrict__ G) {
    constexpr int PPW = 32 / W;                      // parents per warp
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* Ts = reinterpret_cast<C*>(smem_raw);          // [343][W]
    const int64_t p0 = K - w;
    for (int idx = threadIdx.x; idx < 343 * W; idx += blockDim.x) {
        const int row = idx / W, sm = idx % W;
        Ts[idx] = sm < w ? T[(int64_t)row * K + p0 + sm] : cmake<C>(0, 0);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane / W, sm = lane % W;
    const int64_t P = (int64_t)blockIdx.x * kM2LTailWarps * PPW + warp * PPW + g;
    if (P >= npar) return;                           // no barrier below
    const int t0 = pcb[P], nt = pce[P] - t0;
    const int e0 = loff[P], ne = loff[P + 1] - e0;
    const bool ok = sm < w;
    int cr[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int ct = t < nt ? (int)(ckey[t0 + t] & 7) : 0;
        cr[t] = ((ct & 1) + 7 * ((ct >> 1) & 1) + 49 * (ct >> 2)) * W;
    }
    C acc[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) acc[t] = cmake<C>(0, 0);
    const C* Fp = F + p0 + (ok ? sm : 0);
    const C* Tl = Ts + sm;
    for (int j = 0; j < ne; ++j) {
        const unsigned long long e = __ldg(lsrc + e0 + j);
        const unsigned lo = (unsigned)e;
        const C f = Fp[(unsigned)(e >> 32)];
        const C* Tb = Tl + (lo & 511u) * W;
#pragma unroll
        for (int t = 0; t < 8; ++t)
            if (t < nt) cfma(acc[t], Tb[cr[t]], f);
    }
    if (ok) {
#pragma unroll
        for (int t = 0; t < 8; ++t)
            if (t < nt) G[(int64_t)(t0 + t) * K + p0 + sm] = acc[t];
    }
}

// samples of the ragged last slice handled by k_m2l_tail (0: k_m2l takes every slice).  The
// tail kernel pays only with many parents and a short ragged slice: each of its warps walks the
// longest list of 32 / W parents serially, so on levels with few parents (long lists, few warps)
// or with w = 8 it was slower than the idle lanes of k_m2l's last slice (2^20 sphere: leaf level,
// w = 2, 69,745 parents: 0.925 -> 0.850 ms; w = 8 levels and the 56-parent level 4 lost 20-50 us
// each).  Both kernels compute the same values, so the choice does not change results.
template <typename C, int NR>
static int m2l_tail(int64_t K, int64_t npar, bool sampled) {
    const int w = (int)(K % 32);
    return NR == 1 && !sampled && m2l_split<C, NR>(K) == 1 && w <= 4 && npar >= 16384 ? w : 0;
}

template <typename C>
static size_t m2l_tail_smem(int W) { return (size_t)343 * W * sizeof(C); }

// kernel launches of one level's M2L
template <typename C, int NR>
static int m2l_launches(int64_t K, int64_t npar, bool sampled) {
    const int w = m2l_tail<C, NR>(K, npar, sampled);
    return (K >= 32 || !w ? 1 : 0) + (w ? 1 : 0);
}

template <typename R, typename C, int NR>
static void launch_m2l(const Plan& p, int l, cudaStream_t s) {
    constexpr int NW = M2LShape<C, NR>::NW;
    const FarLevel& F = p.far[l];
    const TreeLevel& T = p.lev[l];
    const TreeLevel& TP = p.lev[l - 1];
    const int Q = m2l_split<C, NR>(F.K);
    const bool smp = F.T1 != nullptr;
    const int w = m2l_tail<C, NR>(F.K, TP.nbox, smp);
    const int64_t nslices = w ? F.K / 32 : (F.K + 31) / 32;
    if (nslices > 0) {
        const int ppc = Q > 1 ? NW / Q : NW * kM2LParentsPerWarp;
        const size_t sm = m2l_smem<R, C>() + (Q > 1 ? (size_t)NW * 8 * NR * 32 * sizeof(C) : 0);
        const dim3 grid(nblk(TP.nbox, ppc), (unsigned)nslices);
        if (smp)
            k_m2l<R, C, NR, NW, true><<<grid, 32 * NW, sm, s>>>(
                TP.nbox, TP.child_begin, TP.child_end, TP.m2l_off, TP.m2l_src, T.key, F.tmT, (const C*)F.T1, F.T1n,
                (R)F.T1inv_h, (R)(F.T1inv_h - (double)(R)F.T1inv_h), (const R*)F.dirs, (const C*)F.F, F.K, T.nbox * F.K,
                (C*)F.G, Q, p.dev_err, 0);
        else
            k_m2l<R, C, NR, NW, false><<<grid, 32 * NW, sm, s>>>(
                TP.nbox, TP.child_begin, TP.child_end, TP.m2l_off, TP.m2l_src, T.key, F.tmT, nullptr, 0, (R)0, (R)0, nullptr,
                (const C*)F.F, F.K, T.nbox * F.K, (C*)F.G, Q, p.dev_err, std::min(p.wait_first, kM2LWaitLimit));
        MLFMA_LAUNCH_CHECK();
    }
    if (w) {
        int W = 2;
        while (W < w) W *= 2;
        const int ppb = kM2LTailWarps * (32 / W);
        const size_t sm = m2l_tail_smem<C>(W);
        const unsigned nb = (unsigned)nblk(TP.nbox, ppb);
        switch (W) {
#define M2L_TAIL(v)                                                                                                  \
    case v:                                                                                                          \
        k_m2l_tail<C, v><<<nb, 32 * kM2LTailWarps, sm, s>>>(TP.nbox, TP.child_begin, TP.child_end, TP.m2l_off,       \
                                                            TP.m2l_src, T.key, (const C*)F.T, (const C*)F.F, F.K, w, \
                                                            (C*)F.G);                                                \
        break;
            M2L_TAIL(2) M2L_TAIL(4) M2L_TAIL(8) M2L_TAIL(16)
#undef M2L_TAIL
            default: fail(MLFMA_ERR_INVALID_ARG, "tail width %d", W);
        }
        MLFMA_LAUNCH_CHECK();
    }
}

// raise the dynamic shared-memory limit of the M2L kernel once (before any capture)
// ============================================================== phi transforms: mixed-radix FFTs in shared memory
// Stockham autosort FFT of several rows at once (length n = prod of radices 2, 3, 4, 5, 7).
// tw[k] = e^{-2 pi i k / n}; inv = true uses e^{+2 pi i k / n} (no 1/n scaling).
template <typename C>
__device__ __forceinline__ C twid(const C* __restrict__ tw, int idx, bool inv) {
    C t = tw[idx];
    if (inv) t.y = -t.y;
    return t;
}

// e^{-2 pi i k / R} for the radices of the plan (k is a compile-time constant after unrolling)
template <int R, typename T>
__device__ __forceinline__ void root(int k, T& c, T& s) {
    if (R == 2) {
        const T cc[2] = {1, -1};
        c = cc[k]; s = 0;
    } else if (R == 3) {
        const T cc[3] = {1, -0.5, -0.5};
        const T ss[3] = {0, -0.86602540378443865, 0.86602540378443865};
        c = cc[k]; s = ss[k];
    } else if (R == 4) {
        const T cc[4] = {1, 0, -1, 0};
        const T ss[4] = {0, -1, 0, 1};
        c = cc[k]; s = ss[k];
    } else if (R == 5) {
        const T cc[5] = {1, 0.30901699437494742, -0.80901699437494742, -0.80901699437494742, 0.30901699437494742};
        const T ss[5] = {0, -0.95105651629515357, -0.58778525229247313, 0.58778525229247313, 0.95105651629515357};
        c = cc[k]; s = ss[k];
    } else {
        const T cc[7] = {1, 0.62348980185873353, -0.22252093395631440, -0.90096886790241913, -0.90096886790241913,
                         -0.22252093395631440, 0.62348980185873353};
        const T ss[7] = {0, -0.78183148246802981, -0.97492791218182361, -0.43388373911755812, 0.43388373911755812,
                         0.97492791218182361, 0.78183148246802981};
        c = cc[k]; s = ss[k];
    }
}

// one radix-R butterfly of a Stockham stage: inputs a[j + r nb], outputs b[q Ns R + k + kk Ns]
// with q = j / Ns, k = j mod Ns, twiddles tw[k r tstep]
// R-point DFT X_k = sum_r v_r e^{-+2 pi i r k / R} (- forward, + inverse).  Radix 2 and 4 by
// additions (the roots 0, +-1, +-i cost no multiplies); odd radices from the pairs
// a_r = v_r + v_{R-r}, d_r = v_r - v_{R-r}:  A_k = v_0 + sum_r a_r cos(2 pi r k / R),
// B_k = sum_r d_r sin(2 pi r k / R),  X_k = A_k -+ i B_k,  X_{R-k} = A_k +- i B_k.
template <int R, bool INV, typename C>
__device__ __forceinline__ void small_dft(const C (&v)[R], C (&X)[R]) {
    using T = decltype(C::x);
    auto sub = [](C a, C b) { return cmake<C>(a.x - b.x, a.y - b.y); };
    auto mi = [](C a) { return cmake<C>(a.y, -a.x); };          // -i a
    if constexpr (R == 2) {
        X[0] = cadd(v[0], v[1]);
        X[1] = sub(v[0], v[1]);
    } else if constexpr (R == 4) {
        const C s02 = cadd(v[0], v[2]), d02 = sub(v[0], v[2]);
        const C s13 = cadd(v[1], v[3]), d13 = mi(sub(v[1], v[3]));
        X[0] = cadd(s02, s13);
        X[2] = sub(s02, s13);
        X[INV ? 3 : 1] = cadd(d02, d13);
        X[INV ? 1 : 3] = sub(d02, d13);
    } else {
        constexpr int H = (R - 1) / 2;
        C a[H], d[H];
        C x0 = v[0];
#pragma unroll
        for (int r = 1; r <= H; ++r) {
            a[r - 1] = cadd(v[r], v[R - r]);
            d[r - 1] = sub(v[r], v[R - r]);
            x0 = cadd(x0, a[r - 1]);
        }
        X[0] = x0;
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            C A = v[0], B = cmake<C>(0, 0);
#pragma unroll
            for (int r = 1; r <= H; ++r) {
                T c, s;
                root<R, T>((r * k) % R, c, s);         // c = cos, s = -sin of 2 pi r k / R
                crfma(A, c, a[r - 1]);
                crfma(B, -s, d[r - 1]);
            }
            const C miB = mi(B);
            X[INV ? R - k : k] = cadd(A, miB);
            X[INV ? k : R - k] = sub(A, miB);
        }
    }
}

// Radix-R butterflies of one Stockham stage for the same butterfly index j in up to kFftRows
// rows (row, row + 1, ...): inputs a[j + r nb], outputs b[q Ns R + k + kk Ns] with q = j / Ns,
// k = j mod Ns, twiddles tw[k r tstep].  The index arithmetic and the twiddle loads are done
// once for all the rows.
constexpr int kFftRows = 2;

template <int R, bool INV, typename C>
__device__ __forceinline__ void fft_bfly_rows(const C* __restrict__ a, C* __restrict__ b, int nr, int pitch, int j, int nb,
                                              int Ns, int q, int tstep, const C* __restrict__ tw) {
    const int k = j - q * Ns;
    C w[R];
#pragma unroll
    for (int r = 1; r < R; ++r) w[r] = twid(tw, k * r * tstep, INV);
    const int idxD = q * Ns * R + k;
#pragma unroll
    for (int u = 0; u < kFftRows; ++u) {
        if (u < nr) {
            const C* ar = a + u * pitch;
            C* br = b + u * pitch;
            C v[R];
            v[0] = ar[j];
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(ar[j + r * nb], w[r]);
            C X[R];
            small_dft<R, INV>(v, X);
#pragma unroll
            for (int kk = 0; kk < R; ++kk) br[idxD + kk * Ns] = X[kk];
        }
    }
}

// one stage over nrows rows: a thread takes a butterfly index j and a group of kFftRows rows
template <bool INV, typename C>
__device__ __forceinline__ void fft_stage(const C* __restrict__ in, C* __restrict__ out, int nrows, const FftPlan& fp, int st,
                                          const C* __restrict__ tw, int pitch) {
    const int R = fp.r[st], nb = fp.nb[st], Ns = fp.Ns[st], tstep = fp.tstep[st];
    const FastDiv dnb = fp.dnb[st], dNs = fp.dNs[st];
    const int ngroups = (nrows + kFftRows - 1) / kFftRows;
    for (int idx = threadIdx.x; idx < ngroups * nb; idx += blockDim.x) {
        const int g = (int)dnb.div((unsigned)idx), j = idx - g * nb;
        const int q = (int)dNs.div((unsigned)j);
        const int row = g * kFftRows, nr = min(kFftRows, nrows - row);
        const C* a = in + row * pitch;
        C* b = out + row * pitch;
        switch (R) {
            case 2: fft_bfly_rows<2, INV>(a, b, nr, pitch, j, nb, Ns, q, tstep, tw); break;
            case 3: fft_bfly_rows<3, INV>(a, b, nr, pitch, j, nb, Ns, q, tstep, tw); break;
            case 4: fft_bfly_rows<4, INV>(a, b, nr, pitch, j, nb, Ns, q, tstep, tw); break;
            case 5: fft_bfly_rows<5, INV>(a, b, nr, pitch, j, nb, Ns, q, tstep, tw); break;
            default: fft_bfly_rows<7, INV>(a, b, nr, pitch, j, nb, Ns, q, tstep, tw); break;
        }
    }
}

// Transforms nrows rows of length fp.n, pitch elements apart, in buf0; returns the buffer
// holding the result (buf0 or buf1).  All threads of the block take part.  Kernels whose
// gathers or scatters give consecutive threads consecutive rows use the odd pitch n + 1, so
// that those rows start in different shared-memory banks.
template <typename C>
__device__ C* fft_rows(C* buf0, C* buf1, int nrows, const FftPlan& fp, const C* __restrict__ tw, bool inv, int pitch) {
    C* in = buf0;
    C* out = buf1;
    for (int st = 0; st < fp.ns; ++st) {
        if (inv) fft_stage<true>(in, out, nrows, fp, st, tw, pitch);
        else fft_stage<false>(in, out, nrows, fp, st, tw, pitch);
        __syncthreads();
        C* t = in; in = out; out = t;
    }
    return in;
}

__device__ __forceinline__ int wrap(int m, int n) { return m < 0 ? m + n : m; }

// Shared-memory budgets of the interpolation tiles are plan fields: Plan::tile_fft for one
// row-tile FFT CTA (20 KB by default: several resident CTAs per SM) and Plan::tile_parent for
// the per-parent transforms (32 KB: quadrant rows of one parent in fewer row tiles).

// M2M first step: X[mi][c][i] = scale sum_j F[c][i][j] e^{-i m phi_j}, |m| <= Lc, for the rows
// r = c nth + i of all children (rows are contiguous in F; X is mode-major).  dRB divides by RB.
template <typename C, typename R>
__global__ void k_fft_fwd_rows(int nrows_tot, const C* __restrict__ F, int Lc, FftPlan fp, const C* __restrict__ tw,
                               R scale, int RB, FastDiv dRB, C* __restrict__ X) {
    extern __shared__ unsigned char smem_raw[];
    const int n = fp.n, pn = n + 1, nm = 2 * Lc + 1;
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + RB * pn;
    C* stw = buf1 + RB * pn;
    const int r0 = blockIdx.x * RB;
    const int nr = min(RB, nrows_tot - r0);
    const C* src = F + (int64_t)r0 * n;
    for (int idx = threadIdx.x; idx < nr * n; idx += blockDim.x) {
        const int row = (int)fp.dn.div((unsigned)idx), col = idx - row * n;
        cp_async_zfill<sizeof(C)>(buf0 + row * pn + col, src + idx, true);
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) cp_async_zfill<sizeof(C)>(stw + j, tw + j, true);
    cp_async_wait_all();
    __syncthreads();
    const C* res = fft_rows(buf0, buf1, nr, fp, stw, false, pn);
    for (int idx = threadIdx.x; idx < RB * nm; idx += blockDim.x) {
        const int mi = (int)dRB.div((unsigned)idx), row = idx - mi * RB;
        if (row >= nr) continue;
        C v = res[row * pn + wrap(mi - Lc, n)];
        v.x *= scale; v.y *= scale;
        X[(int64_t)mi * nrows_tot + r0 + row] = v;
    }
}

// children of parent P by xy-quadrant q = oct & 3 and z half oct >> 2 (-1: absent); the
// present quadrants in ascending order.  Ends with a barrier.
__device__ __forceinline__ int parent_quadrants(int c0, int c1, const uint64_t* __restrict__ ckey, int (*s_child)[2],
                                                int* s_q, int* s_nq) {
    if (threadIdx.x < 8) s_child[threadIdx.x >> 1][threadIdx.x & 1] = -1;
    __syncthreads();
    if ((int)threadIdx.x < c1 - c0) {
        const int c = c0 + threadIdx.x;
        const int oct = (int)(ckey[c] & 7);
        s_child[oct & 3][oct >> 2] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int nq = 0;
        for (int q = 0; q < 4; ++q)
            if (s_child[q][0] >= 0 || s_child[q][1] >= 0) s_q[nq++] = q;
        *s_nq = nq;
    }
    __syncthreads();
    return *s_nq;
}

// M2M last step, per parent P and tile of RT parent rows i' (the present xy-quadrants q are
// transformed together):
//   W_q[i'][m] = sum_{children c = (q, sz)} Sz[sz][i'] Y[mi][c][i']          (z part of the shift, per mode)
//   F_P[i'][j'] = sum_q Sxy[q][i'][j'] sum_m W_q[i'][m] e^{+i m phi'_j'}     (inverse FFT, xy part of the shift)
// dRT divides by RT, dn by n.
template <typename C>
__global__ void k_m2m_fft_out(const int* __restrict__ cb, const int* __restrict__ ce, const uint64_t* __restrict__ ckey,
                              int nbox_c, const C* __restrict__ Y, int Lc, int nthp, FftPlan fp, const C* __restrict__ tw,
                              const C* __restrict__ Sz, const C* __restrict__ Sxy, int RT, FastDiv dRT, FastDiv dn,
                              C* __restrict__ Fp) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ int s_child[4][2];
    __shared__ int s_q[4], s_nq;
    const int n = fp.n, nm = 2 * Lc + 1;
    const int64_t Kp = (int64_t)nthp * n;
    const int P = blockIdx.x;
    const int c0 = cb[P], c1 = ce[P];
    if (c0 >= c1) return;
    const int i0 = blockIdx.y * RT;
    const int nr = min(RT, nthp - i0);
    const int pn = n + 1;
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + 4 * RT * pn;
    C* stw = buf1 + 4 * RT * pn;
    for (int j = threadIdx.x; j < n; j += blockDim.x) stw[j] = tw[j];
    const int nq = parent_quadrants(c0, c1, ckey, s_child, s_q, &s_nq);
    // rows of the qi-th present quadrant occupy buf0[(qi * nr + r) * pn ...].  A thread takes a
    // (mode, row) item for every present quadrant at once: its z-shift factors and index
    // arithmetic serve them all, and the child indices come from registers; the loads of all
    // quadrants are issued before use.  The columns of the modes beyond Lc are zeroed apart
    // (disjoint from the mode columns, so no barrier between the two).
    int qa[4], qz[4];
#pragma unroll
    for (int qi = 0; qi < 4; ++qi) {
        const int q = qi < nq ? s_q[qi] : 0;
        qa[qi] = qi < nq ? s_child[q][0] : -1;
        qz[qi] = qi < nq ? s_child[q][1] : -1;
    }
    for (int idx = threadIdx.x; idx < nm * RT; idx += blockDim.x) {
        const int mi = (int)dRT.div((unsigned)idx), r = idx - mi * RT;
        if (r >= nr) continue;
        const C sz0 = Sz[i0 + r], sz1 = Sz[nthp + i0 + r];
        const C* Ym = Y + (int64_t)mi * nbox_c * nthp + i0 + r;
        C ya[4], yz[4];
#pragma unroll
        for (int qi = 0; qi < 4; ++qi) {
            ya[qi] = qa[qi] >= 0 ? Ym[(int64_t)qa[qi] * nthp] : cmake<C>(0, 0);
            yz[qi] = qz[qi] >= 0 ? Ym[(int64_t)qz[qi] * nthp] : cmake<C>(0, 0);
        }
        C* dst = buf0 + r * pn + wrap(mi - Lc, n);
#pragma unroll
        for (int qi = 0; qi < 4; ++qi)
            if (qi < nq) {
                C w = cmake<C>(0, 0);
                cfma(w, sz0, ya[qi]);
                cfma(w, sz1, yz[qi]);
                dst[qi * nr * pn] = w;
            }
    }
    const int nz = n - nm;                        // columns Lc + 1 .. n - Lc - 1
    for (int idx = threadIdx.x; idx < nq * nr * nz; idx += blockDim.x) {
        const int row = idx / nz, k = idx - row * nz;
        buf0[row * pn + Lc + 1 + k] = cmake<C>(0, 0);
    }
    __syncthreads();
    const C* res = fft_rows(buf0, buf1, nq * nr, fp, stw, true, pn);
    const C* sxy[4];                                  // xy-shift tables of the present quadrants, from row i0
#pragma unroll
    for (int qi = 0; qi < 4; ++qi) sxy[qi] = Sxy + (int64_t)(qi < nq ? s_q[qi] : 0) * Kp + (int64_t)i0 * n;
    for (int idx = threadIdx.x; idx < nr * n; idx += blockDim.x) {
        const int r = (int)dn.div((unsigned)idx), j = idx - r * n;
        const C* rq = res + r * pn + j;
        C acc = cmake<C>(0, 0);
#pragma unroll
        for (int qi = 0; qi < 4; ++qi)                  // fixed bound: the loads issue together
            if (qi < nq) cfma(acc, sxy[qi][idx], rq[qi * nr * pn]);
        Fp[(int64_t)P * Kp + (int64_t)i0 * n + idx] = acc;
    }
}

// L2L first step, per parent P and tile of RT parent rows i' (present xy-quadrants in one FFT pass):
//   V_q[i'][m] = (1/n) sum_j' conj(Sxy[q][i'][j']) G_P[i'][j'] e^{+i m phi'_j'},  |m| <= Lc
//   Y[mi][c][i'] = conj(Sz[sz][i']) V_q[i'][m] for each child c = (q, sz)
template <typename C, typename R>
__global__ void k_l2l_fft_in(const int* __restrict__ cb, const int* __restrict__ ce, const uint64_t* __restrict__ ckey,
                             int nbox_c, const C* __restrict__ Gp, int Lc, int nthp, FftPlan fp, const C* __restrict__ tw,
                             const C* __restrict__ Sz, const C* __restrict__ Sxy, int RT, FastDiv dRT, FastDiv dn, R inv_n,
                             C* __restrict__ Y) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ int s_child[4][2];
    __shared__ int s_q[4], s_nq;
    const int n = fp.n, nm = 2 * Lc + 1;
    const int64_t Kp = (int64_t)nthp * n;
    const int P = blockIdx.x;
    const int c0 = cb[P], c1 = ce[P];
    if (c0 >= c1) return;
    const int i0 = blockIdx.y * RT;
    const int nr = min(RT, nthp - i0);
    const int pn = n + 1;
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + 4 * RT * pn;
    C* stw = buf1 + 4 * RT * pn;
    for (int j = threadIdx.x; j < n; j += blockDim.x) stw[j] = tw[j];
    // the tile G_P[i0 .. i0 + nr) is contiguous: stage it in buf1 (free until the transform),
    // in flight while the quadrants are scanned
    const C* gsrc = Gp + (int64_t)P * Kp + (int64_t)i0 * n;
    for (int idx = threadIdx.x; idx < nr * n; idx += blockDim.x) cp_async_zfill<sizeof(C)>(buf1 + idx, gsrc + idx, true);
    const int nq = parent_quadrants(c0, c1, ckey, s_child, s_q, &s_nq);
    cp_async_wait_all();
    __syncthreads();
    const C* sxy[4];                                  // xy-shift tables of the present quadrants, from row i0
#pragma unroll
    for (int qi = 0; qi < 4; ++qi) sxy[qi] = Sxy + (int64_t)(qi < nq ? s_q[qi] : 0) * Kp + (int64_t)i0 * n;
    for (int idx = threadIdx.x; idx < nr * n; idx += blockDim.x) {
        const C gv = buf1[idx];
        const int r = (int)dn.div((unsigned)idx), j = idx - r * n;
        C* dst = buf0 + r * pn + j;
#pragma unroll
        for (int qi = 0; qi < 4; ++qi)
            if (qi < nq) dst[qi * nr * pn] = cmul(cconj(sxy[qi][idx]), gv);
    }
    __syncthreads();
    const C* res = fft_rows(buf0, buf1, nq * nr, fp, stw, true, pn);
    // a thread takes a (mode, row) item for every present quadrant: the z-shift factors and the
    // index arithmetic serve them all, the child indices come from registers
    int qa[4], qz[4];
#pragma unroll
    for (int qi = 0; qi < 4; ++qi) {
        const int q = qi < nq ? s_q[qi] : 0;
        qa[qi] = qi < nq ? s_child[q][0] : -1;
        qz[qi] = qi < nq ? s_child[q][1] : -1;
    }
    for (int idx = threadIdx.x; idx < RT * nm; idx += blockDim.x) {
        const int mi = (int)dRT.div((unsigned)idx), r = idx - mi * RT;
        if (r >= nr) continue;
        const C sz0 = cconj(Sz[i0 + r]), sz1 = cconj(Sz[nthp + i0 + r]);
        const C* src = res + r * pn + wrap(mi - Lc, n);
        C* Ym = Y + (int64_t)mi * nbox_c * nthp + i0 + r;
#pragma unroll
        for (int qi = 0; qi < 4; ++qi) {
            if (qi >= nq) break;
            C v = src[qi * nr * pn];
            v.x *= inv_n; v.y *= inv_n;
            if (qa[qi] >= 0) Ym[(int64_t)qa[qi] * nthp] = cmul(sz0, v);
            if (qz[qi] >= 0) Ym[(int64_t)qz[qi] * nthp] = cmul(sz1, v);
        }
    }
}

// ---- coarse level pairs: the present quadrants one after another
// With long parent rows (n up to a few hundred) the four-quadrant buffers above leave room for
// one or two rows per CTA, so the gathers from the mode-major spectral scratch touch one sample
// per 32-byte sector.  These variants hold one quadrant's rows at a time (buffers of RT rows,
// and the parent tile or the output sum of RT rows), so a CTA takes three to four times as many
// rows; each quadrant is transformed in turn.  Per sample the arithmetic and its order are those
// of k_m2m_fft_out / k_l2l_fft_in (quadrants in ascending order), so results are identical.
template <typename C>
__global__ void k_m2m_fft_out_q(const int* __restrict__ cb, const int* __restrict__ ce, const uint64_t* __restrict__ ckey,
                                int nbox_c, const C* __restrict__ Y, int Lc, int nthp, FftPlan fp, const C* __restrict__ tw,
                                const C* __restrict__ Sz, const C* __restrict__ Sxy, int RT, FastDiv dRT, FastDiv dn,
                                FastDiv dnz, C* __restrict__ Fp) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ int s_child[4][2];
    __shared__ int s_q[4], s_nq;
    const int n = fp.n, nm = 2 * Lc + 1;
    const int64_t Kp = (int64_t)nthp * n;
    const int P = blockIdx.x;
    const int c0 = cb[P], c1 = ce[P];
    if (c0 >= c1) return;
    const int i0 = blockIdx.y * RT;
    const int nr = min(RT, nthp - i0);
    const int pn = n + 1;
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + RT * pn;
    C* stw = buf1 + RT * pn;
    C* sum = stw + n;                                 // [nr][n]: F_P rows accumulated over quadrants
    for (int j = threadIdx.x; j < n; j += blockDim.x) stw[j] = tw[j];
    const int nq = parent_quadrants(c0, c1, ckey, s_child, s_q, &s_nq);
    const int nz = n - nm;
    for (int qi = 0; qi < nq; ++qi) {
        const int q = s_q[qi];
        const int ca = s_child[q][0], cz = s_child[q][1];
        for (int idx = threadIdx.x; idx < nm * RT; idx += blockDim.x) {
            const int mi = (int)dRT.div((unsigned)idx), r = idx - mi * RT;
            if (r >= nr) continue;
            const C* Ym = Y + (int64_t)mi * nbox_c * nthp + i0 + r;
            const C ya = ca >= 0 ? Ym[(int64_t)ca * nthp] : cmake<C>(0, 0);
            const C yz = cz >= 0 ? Ym[(int64_t)cz * nthp] : cmake<C>(0, 0);
            C w = cmake<C>(0, 0);
            cfma(w, Sz[i0 + r], ya);
            cfma(w, Sz[nthp + i0 + r], yz);
            buf0[r * pn + wrap(mi - Lc, n)] = w;
        }
        for (int idx = threadIdx.x; idx < nr * nz; idx += blockDim.x) {
            const int row = (int)dnz.div((unsigned)idx), k = idx - row * nz;
            buf0[row * pn + Lc + 1 + k] = cmake<C>(0, 0);
        }
        __syncthreads();
        const C* res = fft_rows(buf0, buf1, nr, fp, stw, true, pn);
        const C* sq = Sxy + (int64_t)q * Kp + (int64_t)i0 * n;
        for (int idx = threadIdx.x; idx < nr * n; idx += blockDim.x) {
            const int r = (int)dn.div((unsigned)idx), j = idx - r * n;
            C acc = qi ? sum[idx] : cmake<C>(0, 0);
            cfma(acc, sq[idx], res[r * pn + j]);
            sum[idx] = acc;
        }
        __syncthreads();                              // buf0 / buf1 are refilled for the next quadrant
    }
    C* out = Fp + (int64_t)P * Kp + (int64_t)i0 * n;
    for (int idx = threadIdx.x; idx < nr * n; idx += blockDim.x) out[idx] = sum[idx];
}

template <typename C, typename R>
__global__ void k_l2l_fft_in_q(const int* __restrict__ cb, const int* __restrict__ ce, const uint64_t* __restrict__ ckey,
                               int nbox_c, const C* __restrict__ Gp, int Lc, int nthp, FftPlan fp, const C* __restrict__ tw,
                               const C* __restrict__ Sz, const C* __restrict__ Sxy, int RT, FastDiv dRT, FastDiv dn,
                               R inv_n, C* __restrict__ Y) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ int s_child[4][2];
    __shared__ int s_q[4], s_nq;
    const int n = fp.n, nm = 2 * Lc + 1;
    const int64_t Kp = (int64_t)nthp * n;
    const int P = blockIdx.x;
    const int c0 = cb[P], c1 = ce[P];
    if (c0 >= c1) return;
    const int i0 = blockIdx.y * RT;
    const int nr = min(RT, nthp - i0);
    const int pn = n + 1;
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + RT * pn;
    C* stw = buf1 + RT * pn;
    C* gs = stw + n;                                  // [nr][n]: the parent tile G_P[i0 .. i0 + nr)
    for (int j = threadIdx.x; j < n; j += blockDim.x) stw[j] = tw[j];
    const C* gsrc = Gp + (int64_t)P * Kp + (int64_t)i0 * n;
    for (int idx = threadIdx.x; idx < nr * n; idx += blockDim.x) cp_async_zfill<sizeof(C)>(gs + idx, gsrc + idx, true);
    const int nq = parent_quadrants(c0, c1, ckey, s_child, s_q, &s_nq);
    cp_async_wait_all();
    __syncthreads();
    for (int qi = 0; qi < nq; ++qi) {
        const int q = s_q[qi];
        const int ca = s_child[q][0], cz = s_child[q][1];
        const C* sq = Sxy + (int64_t)q * Kp + (int64_t)i0 * n;
        for (int idx = threadIdx.x; idx < nr * n; idx += blockDim.x) {
            const int r = (int)dn.div((unsigned)idx), j = idx - r * n;
            buf0[r * pn + j] = cmul(cconj(sq[idx]), gs[idx]);
        }
        __syncthreads();
        const C* res = fft_rows(buf0, buf1, nr, fp, stw, true, pn);
        for (int idx = threadIdx.x; idx < RT * nm; idx += blockDim.x) {
            const int mi = (int)dRT.div((unsigned)idx), r = idx - mi * RT;
            if (r >= nr) continue;
            C v = res[r * pn + wrap(mi - Lc, n)];
            v.x *= inv_n; v.y *= inv_n;
            C* Ym = Y + (int64_t)mi * nbox_c * nthp + i0 + r;
            if (ca >= 0) Ym[(int64_t)ca * nthp] = cmul(cconj(Sz[i0 + r]), v);
            if (cz >= 0) Ym[(int64_t)cz * nthp] = cmul(cconj(Sz[nthp + i0 + r]), v);
        }
        __syncthreads();                              // buf0 / buf1 are refilled for the next quadrant
    }
}

// L2L last step: G[c][i][j] += sum_m H[mi][c][i] e^{-i m phi_j} for the rows r = c nth + i of all children.
template <typename C>
__global__ void k_l2l_fft_out(int nrows_tot, const C* __restrict__ H, int Lc, FftPlan fp, const C* __restrict__ tw, int RB,
                              FastDiv dRB, C* __restrict__ G) {
    extern __shared__ unsigned char smem_raw[];
    const int n = fp.n, nm = 2 * Lc + 1;
    const int pn = n + 1;
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + RB * pn;
    C* stw = buf1 + RB * pn;
    const int r0 = blockIdx.x * RB;
    const int nr = min(RB, nrows_tot - r0);
    for (int idx = threadIdx.x; idx < nr * pn; idx += blockDim.x) buf0[idx] = cmake<C>(0, 0);
    for (int j = threadIdx.x; j < n; j += blockDim.x) stw[j] = tw[j];
    __syncthreads();
    // the zero fill above is complete (barrier) before the copies overwrite the mode columns
    for (int idx = threadIdx.x; idx < RB * nm; idx += blockDim.x) {
        const int mi = (int)dRB.div((unsigned)idx), row = idx - mi * RB;
        if (row >= nr) continue;
        cp_async_zfill<sizeof(C)>(buf0 + row * pn + wrap(mi - Lc, n), H + (int64_t)mi * nrows_tot + r0 + row, true);
    }
    cp_async_wait_all();
    __syncthreads();
    const C* res = fft_rows(buf0, buf1, nr, fp, stw, false, pn);
    C* g0 = G + (int64_t)r0 * n;
#pragma unroll 4
    for (int idx = threadIdx.x; idx < nr * n; idx += blockDim.x) {
        const int row = (int)fp.dn.div((unsigned)idx), col = idx - row * n;
        g0[idx] = cadd(g0[idx], res[row * pn + col]);
    }
}

// ============================================================== fused phi transform + theta map (fine levels)
// For level pairs whose child rows fit in shared memory a CTA takes CPB (2 ... 16, a power
// of two) consecutive child boxes and keeps the spectral rows on chip between the phi transform and
// the theta map.  The theta map is register-blocked over the CTA's children and split by
// parity like k_theta_map_par: a thread owns one mode, one output row o and its mirror n'-1-o,
// with an even and an odd accumulator per child, so each entry of the map's halves is loaded
// once per CTA and the spectral samples are shared-memory broadcasts.
constexpr int kMaxCPB = 16;

// M2M first two steps:  Y[mi][c][i'] = scale sum_i At[|m|][i][i'] sum_j F[c][i][j] e^{-i m phi_j}
// (At applied as its parity halves AtE, AtD).
// dnh divides by (nthp + 1) / 2.
template <typename C, typename R, int CPB>
__global__ void k_m2m_in(int nbox_c, const C* __restrict__ F, int Lc, int nthc, int nthp, FftPlan fp,
                         const C* __restrict__ tw, R scale, const R* __restrict__ AtE, const R* __restrict__ AtD,
                         FastDiv dnh, C* __restrict__ Y) {
    extern __shared__ unsigned char smem_raw[];
    const int n = fp.n, nm = 2 * Lc + 1;
    // unpadded rows: no loop here walks across rows with consecutive threads
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + CPB * nthc * n;
    C* stw = buf1 + CPB * nthc * n;
    const int c0 = blockIdx.x * CPB;
    const int ncb = min(CPB, nbox_c - c0);
    const int nr = ncb * nthc;
    const C* src = F + (int64_t)c0 * nthc * n;
    for (int idx = threadIdx.x; idx < nr * n; idx += blockDim.x) cp_async_zfill<sizeof(C)>(buf0 + idx, src + idx, true);
    for (int j = threadIdx.x; j < n; j += blockDim.x) cp_async_zfill<sizeof(C)>(stw + j, tw + j, true);
    cp_async_wait_all();
    __syncthreads();
    const C* res = fft_rows(buf0, buf1, nr, fp, stw, false, n);
    const int rowc = nthc * n;                     // stride between children in res
    // a thread takes output row o and its mirror nthp - 1 - o of one mode, from the parity
    // halves of the map (even part on e_i = x_i + x_{n-1-i}, odd part on d_i = x_i - x_{n-1-i})
    const int nh = (nthp + 1) >> 1, hin = (nthc + 1) >> 1;
    for (int idx = threadIdx.x; idx < nm * nh; idx += blockDim.x) {
        const int mi = (int)dnh.div((unsigned)idx), o = idx - mi * nh;
        const int m = abs(mi - Lc);
        const R* Em = AtE + (int64_t)m * hin * nh + o;
        const R* Dm = AtD + (int64_t)m * hin * nh + o;
        const C* xr = res + wrap(mi - Lc, n);
        C ae[CPB], ad[CPB];
#pragma unroll
        for (int c = 0; c < CPB; ++c) ae[c] = ad[c] = cmake<C>(0, 0);
        for (int i = 0; i < hin; ++i) {
            const R e = Em[i * nh], d = Dm[i * nh];
            const C* xl = xr + i * n;
            const C* xh = xr + (nthc - 1 - i) * n;
#pragma unroll
            for (int c = 0; c < CPB; ++c)
                if (c < ncb) {
                    const C lo = xl[c * rowc], hi = xh[c * rowc];
                    crfma(ae[c], e, cmake<C>(lo.x + hi.x, lo.y + hi.y));
                    crfma(ad[c], d, cmake<C>(lo.x - hi.x, lo.y - hi.y));
                }
        }
        C* yo = Y + ((int64_t)mi * nbox_c + c0) * nthp;
        const bool mirror = nthp - 1 - o != o;
#pragma unroll
        for (int c = 0; c < CPB; ++c)
            if (c < ncb) {
                yo[c * nthp + o] = cmake<C>((ae[c].x + ad[c].x) * scale, (ae[c].y + ad[c].y) * scale);
                if (mirror) yo[c * nthp + nthp - 1 - o] = cmake<C>((ae[c].x - ad[c].x) * scale, (ae[c].y - ad[c].y) * scale);
            }
    }
}

// L2L last two steps:  G[c][i][j] += sum_m e^{-i m phi_j} sum_i' Bt[|m|][i'][i] H[mi][c][i']
// (Bt applied as its parity halves BtE, BtD).
// The CTA's slice of H is staged in shared memory first.  dnh divides by (nthc + 1) / 2, dhrow
// by ncb nthp (dhfull: CPB nthp, the value for every CTA but the last).
template <typename C, typename R, int CPB>
__global__ void k_l2l_out(int nbox_c, const C* __restrict__ H, int Lc, int nthc, int nthp, FftPlan fp,
                          const C* __restrict__ tw, const R* __restrict__ BtE, const R* __restrict__ BtD, FastDiv dnh,
                          FastDiv dhrow,
                          FastDiv dhfull, C* __restrict__ G) {
    extern __shared__ unsigned char smem_raw[];
    const int n = fp.n, nm = 2 * Lc + 1;
    const int pn = n + 1, hp = CPB * nthp + 1;     // padded pitches of the FFT rows and of hs
    // hs is read only by the theta map, before the FFT needs buf1: the two share their space
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* stw = buf0 + CPB * nthc * pn;
    C* buf1 = stw + n;
    C* hs = buf1;                                  // [nm][hp]: the CPB children's rows of one mode
    const int c0 = blockIdx.x * CPB;
    const int ncb = min(CPB, nbox_c - c0);
    const int nr = ncb * nthc;
    const int hrow = ncb * nthp;                   // contiguous run of the CTA's children in one mode
    for (int idx = threadIdx.x; idx < nm * hrow; idx += blockDim.x) {
        const int mi = (int)(ncb == CPB ? dhfull : dhrow).div((unsigned)idx), t = idx - mi * hrow;
        cp_async_zfill<sizeof(C)>(hs + mi * hp + t, H + ((int64_t)mi * nbox_c + c0) * nthp + t, true);
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) cp_async_zfill<sizeof(C)>(stw + j, tw + j, true);
    for (int idx = threadIdx.x; idx < nr * pn; idx += blockDim.x) buf0[idx] = cmake<C>(0, 0);
    cp_async_wait_all();
    __syncthreads();
    // a thread takes child row i and its mirror nthc - 1 - i of one mode, from the parity halves
    const int nh = (nthc + 1) >> 1, hin = (nthp + 1) >> 1;
    for (int idx = threadIdx.x; idx < nm * nh; idx += blockDim.x) {
        const int mi = (int)dnh.div((unsigned)idx), i = idx - mi * nh;
        const int m = abs(mi - Lc);
        const R* Em = BtE + (int64_t)m * hin * nh + i;
        const R* Dm = BtD + (int64_t)m * hin * nh + i;
        const C* hm = hs + mi * hp;
        C ae[CPB], ad[CPB];
#pragma unroll
        for (int c = 0; c < CPB; ++c) ae[c] = ad[c] = cmake<C>(0, 0);
        for (int ip = 0; ip < hin; ++ip) {
            const R e = Em[ip * nh], d = Dm[ip * nh];
#pragma unroll
            for (int c = 0; c < CPB; ++c)
                if (c < ncb) {
                    const C lo = hm[c * nthp + ip], hi = hm[c * nthp + nthp - 1 - ip];
                    crfma(ae[c], e, cmake<C>(lo.x + hi.x, lo.y + hi.y));
                    crfma(ad[c], d, cmake<C>(lo.x - hi.x, lo.y - hi.y));
                }
        }
        const int col = wrap(mi - Lc, n);
        const bool mirror = nthc - 1 - i != i;
#pragma unroll
        for (int c = 0; c < CPB; ++c)
            if (c < ncb) {
                buf0[(c * nthc + i) * pn + col] = cmake<C>(ae[c].x + ad[c].x, ae[c].y + ad[c].y);
                if (mirror) buf0[(c * nthc + nthc - 1 - i) * pn + col] = cmake<C>(ae[c].x - ad[c].x, ae[c].y - ad[c].y);
            }
    }
    __syncthreads();
    const C* res = fft_rows(buf0, buf1, nr, fp, stw, false, pn);
    C* g0 = G + (int64_t)c0 * nthc * n;
    for (int idx = threadIdx.x; idx < nr * n; idx += blockDim.x) {
        const int row = (int)fp.dn.div((unsigned)idx), col = idx - row * n;
        g0[idx] = cadd(g0[idx], res[row * pn + col]);
    }
}

// Y[mi][c][i'] = 0 for the boxes c of the given ranges (forest boxes without a parent: the
// L2L out-stage then adds nothing to them); one thread per (range, box, mode, row) in turn
template <typename C>
__global__ void k_zero_orphans(const int2* __restrict__ ranges, int nranges, int64_t total, int nbox_c, int nm, int nthp,
                               C* __restrict__ Y) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= total * nm * nthp) return;
    const int ip = (int)(idx % nthp);
    const int64_t t = idx / nthp;
    const int mi = (int)(t % nm);
    int64_t b = t / nm;                       // orphan ordinal
    int g = 0;
    while (g < nranges && b >= ranges[g].y) {
        b -= ranges[g].y;
        ++g;
    }
    if (g >= nranges) return;
    Y[((int64_t)mi * nbox_c + ranges[g].x + b) * nthp + ip] = cmake<C>(0, 0);
}

// children per CTA of the fused kernels, a power of two in [2, kMaxCPB] (0: the level pair
// takes the three-kernel path); extra = complex elements per child staged besides the two
// FFT buffers (rows of ``pitch`` elements), fixed = elements per CTA besides the twiddles
// (budget: Plan::tile_fused, 40 KB by default)
static int fused_children(size_t budget, int nthc, int n, int pitch, int extra, int fixed, size_t csz) {
    // counted as separate areas, although k_l2l_out overlays the extra rows on its second FFT
    // buffer: sized by the overlaid footprint, the 2^20 sphere's 6 -> 7 pair became a fused pair
    // of two children per CTA, slower than the three-kernel path (9.33 vs 9.28 ms per matvec)
    const size_t per = ((size_t)2 * nthc * pitch + extra) * csz;
    if (budget < (size_t)(n + fixed) * csz) return 0;
    const size_t avail = budget - (size_t)(n + fixed) * csz;
    int c = 0;
    for (int t = 2; t <= kMaxCPB; t *= 2)
        if ((size_t)t * per <= avail) c = t;
    return c;
}

template <typename C, typename R>
static void launch_m2m_in(int CPB, int nbox_c, const C* F, int Lc, int nthc, int nthp, const FftPlan& fp, const C* tw,
                          R scale, const R* AtE, const R* AtD, C* Y, cudaStream_t s) {
    const size_t sm = ((size_t)2 * CPB * nthc * fp.n + fp.n) * sizeof(C);
    const FastDiv d = FastDiv::make((nthp + 1) / 2);
    switch (CPB) {
#define M2M_IN(c) case c: k_m2m_in<C, R, c><<<nblk(nbox_c, c), 128, sm, s>>>(nbox_c, F, Lc, nthc, nthp, fp, tw, scale, AtE, AtD, d, Y); break;
        M2M_IN(2) M2M_IN(4) M2M_IN(8) M2M_IN(16)
#undef M2M_IN
        default: fail(MLFMA_ERR_INVALID_ARG, "children per CTA %d", CPB);
    }
    MLFMA_LAUNCH_CHECK();
}

template <typename C, typename R>
static void launch_l2l_out(int CPB, int nbox_c, const C* H, int Lc, int nthc, int nthp, const FftPlan& fp, const C* tw,
                           const R* BtE, const R* BtD, C* G, cudaStream_t s) {
    const size_t rows = (size_t)CPB * nthc * (fp.n + 1), hsz = (size_t)(2 * Lc + 1) * (CPB * nthp + 1);
    const size_t sm = (rows + fp.n + std::max(rows, hsz)) * sizeof(C);
    const FastDiv d = FastDiv::make((nthc + 1) / 2);
    const int tail = nbox_c % CPB ? nbox_c % CPB : CPB;      // children of the last CTA
    const FastDiv dt = FastDiv::make(tail * nthp), df = FastDiv::make(CPB * nthp);
    switch (CPB) {
#define L2L_OUT(c) case c: k_l2l_out<C, R, c><<<nblk(nbox_c, c), 128, sm, s>>>(nbox_c, H, Lc, nthc, nthp, fp, tw, BtE, BtD, d, dt, df, G); break;
        L2L_OUT(2) L2L_OUT(4) L2L_OUT(8) L2L_OUT(16)
#undef L2L_OUT
        default: fail(MLFMA_ERR_INVALID_ARG, "children per CTA %d", CPB);
    }
    MLFMA_LAUNCH_CHECK();
}

// ============================================================== theta maps
// Per Fourier mode, a batched GEMM (complex x real):
//   out[mi][c][o] = sum_i M[|m|][i][o] in[mi][c][i],   m = mi - Lc
// Tile BM boxes x BN outputs per CTA (BM * BN = 4096), 256 threads, 4 x 4 per thread; the
// reduction runs in chunks of BK (16 complex64, 8 complex128) staged in shared memory by
// cp.async, double-buffered so that the next chunk loads while this one is multiplied (three
// stages measured no better than two).
template <typename C> __device__ __forceinline__ void ld4c(const C* p, C (&v)[4]) {
    if constexpr (sizeof(C) == 8) {            // two 16-byte loads
        const float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 2);
        v[0] = cmake<C>(a.x, a.y); v[1] = cmake<C>(a.z, a.w); v[2] = cmake<C>(b.x, b.y); v[3] = cmake<C>(b.z, b.w);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = p[q];
    }
}
template <typename R> __device__ __forceinline__ void ld4r(const R* p, R (&v)[4]) {
    if constexpr (sizeof(R) == 4) {
        const float4 a = *reinterpret_cast<const float4*>(p);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    } else {
        const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
}

// The same GEMM by parity.  Gauss-Legendre nodes come in pairs (x, -x) and every map is
// centrosymmetric, M[n-1-i][n'-1-o] = M[i][o], so with e_i = in[i] + in[n-1-i] and
// d_i = in[i] - in[n-1-i] (i < ceil(n/2)) the halves
//   oe[o] = sum_i ME[i][o] e_i,   od[o] = sum_i MD[i][o] d_i   (o < ceil(n'/2))
// give out[o] = oe + od and out[n'-1-o] = oe - od: two GEMMs of a quarter of the size, half the
// multiply-adds of the full map.  ME and MD are built at plan creation from the even and odd
// terms of the Legendre sums (k_interp_par; ME's middle row halved, because e takes the middle
// sample twice).  The CTA stages the rows in[i] and in[n-1-i] of its chunk and forms e and d
// in registers as it multiplies.
template <typename R, typename C, int BN>
struct MapParShape {
    static constexpr int BM = 4096 / BN, BK = sizeof(C) == 8 ? 16 : 8, AP = BM + 2;
    static constexpr size_t smem = 2 * (2 * (size_t)BK * AP * sizeof(C) + 2 * (size_t)BK * BN * sizeof(R));
};

template <typename R, typename C, int BN>
__global__ void __launch_bounds__(256) k_theta_map_par(int nbox, int Lc, int nin, int nout, const R* __restrict__ ME,
                                                       const R* __restrict__ MD, const C* __restrict__ in,
                                                       C* __restrict__ out) {
    using S = MapParShape<R, C, BN>;
    constexpr int BM = S::BM, BK = S::BK, AP = S::AP;
    constexpr int TX = BN / 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* Al = reinterpret_cast<C*>(smem_raw);                    // [2][BK][AP] in[i]
    C* Ah = Al + 2 * BK * AP;                                  // [2][BK][AP] in[nin-1-i]
    R* Be = reinterpret_cast<R*>(Ah + 2 * BK * AP);            // [2][BK][BN]
    R* Bd = Be + 2 * BK * BN;                                  // [2][BK][BN]
    const int hin = (nin + 1) / 2, hout = (nout + 1) / 2;
    const int mi = blockIdx.z;
    const int m = abs(mi - Lc);
    const int c0 = blockIdx.x * BM, o0 = blockIdx.y * BN;
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const C* inm = in + (int64_t)mi * nbox * nin;
    const R* Em = ME + (int64_t)m * hin * hout;
    const R* Dm = MD + (int64_t)m * hin * hout;
    auto stage = [&](int buf, int k0) {
        C* al = Al + buf * BK * AP;
        C* ah = Ah + buf * BK * AP;
        for (int idx = threadIdx.x; idx < BM * BK; idx += 256) {
            const int cl = idx / BK, kk = idx % BK;
            const int c = c0 + cl, i = k0 + kk;
            const bool v = c < nbox && i < hin;
            const C* row = inm + (int64_t)c * nin;
            cp_async_zfill<sizeof(C)>(al + kk * AP + cl, v ? row + i : inm, v);
            cp_async_zfill<sizeof(C)>(ah + kk * AP + cl, v ? row + (nin - 1 - i) : inm, v);
        }
        R* be = Be + buf * BK * BN;
        R* bd = Bd + buf * BK * BN;
        for (int idx = threadIdx.x; idx < BK * BN; idx += 256) {
            const int kk = idx / BN, ol = idx % BN;
            const int i = k0 + kk, o = o0 + ol;
            const bool v = i < hin && o < hout;
            const int64_t e = (int64_t)i * hout + o;
            cp_async_zfill<sizeof(R)>(be + kk * BN + ol, v ? Em + e : Em, v);
            cp_async_zfill<sizeof(R)>(bd + kk * BN + ol, v ? Dm + e : Dm, v);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    C ae[4][4], ad[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) ae[a][b] = ad[a][b] = cmake<C>(0, 0);
    const int nch = (hin + BK - 1) / BK;
    stage(0, 0);
    for (int ch = 0; ch < nch; ++ch) {
        if (ch + 1 < nch) {
            stage((ch + 1) & 1, (ch + 1) * BK);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncthreads();
        const C* al = Al + (ch & 1) * BK * AP;
        const C* ah = Ah + (ch & 1) * BK * AP;
        const R* be = Be + (ch & 1) * BK * BN;
        const R* bd = Bd + (ch & 1) * BK * BN;
        auto mac = [&](int kk) {
            C lo[4], hi[4];
            R ev[4], dv[4];
            ld4c(al + kk * AP + ty * 4, lo);
            ld4c(ah + kk * AP + ty * 4, hi);
            ld4r(be + kk * BN + tx * 4, ev);
            ld4r(bd + kk * BN + tx * 4, dv);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const C e = cmake<C>(lo[i].x + hi[i].x, lo[i].y + hi[i].y);
                const C d = cmake<C>(lo[i].x - hi[i].x, lo[i].y - hi[i].y);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    crfma(ae[i][j], ev[j], e);
                    crfma(ad[i][j], dv[j], d);
                }
            }
        };
        const int kc = hin - ch * BK;
        if (kc >= BK) {
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) mac(kk);
        } else {                                  // the last, partial chunk: skip its zero fill
#pragma unroll 2
            for (int kk = 0; kk < kc; ++kk) mac(kk);
        }
        __syncthreads();                          // the buffer is restaged two chunks later
    }
    C* outm = out + (int64_t)mi * nbox * nout;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int c = c0 + ty * 4 + i;
        if (c >= nbox) continue;
        C* row = outm + (int64_t)c * nout;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int o = o0 + tx * 4 + j;
            if (o >= hout) continue;
            const C e = ae[i][j], d = ad[i][j];
            row[o] = cmake<C>(e.x + d.x, e.y + d.y);
            if (nout - 1 - o != o) row[nout - 1 - o] = cmake<C>(e.x - d.x, e.y - d.y);
        }
    }
}

// Mtc: the pre-split form of M for the tensor-core precisions; ME, MD: its parity halves
template <typename R, typename C>
static void launch_theta_map(const Plan& p, int64_t nbox, int Lc, int nin, int nout, const R* M, const void* Mtc,
                             const R* ME, const R* MD, const C* in, C* out, cudaStream_t s) {
    if constexpr (sizeof(C) == 8) {
        if (p.prec == MLFMA_PREC_FP32_TF32X3 || p.prec == MLFMA_PREC_FP32_BF16X3) {
            launch_theta_map_tc(p, nbox, Lc, nin, nout, Mtc, (const float2*)in, (float2*)out, s);
            return;
        }
    }
    const int nm = 2 * Lc + 1;
    const int hout = (nout + 1) / 2;
    if (hout <= 32) {
        k_theta_map_par<R, C, 32><<<dim3(nblk(nbox, 128), nblk(hout, 32), nm), 256, MapParShape<R, C, 32>::smem, s>>>(
            (int)nbox, Lc, nin, nout, ME, MD, in, out);
    } else {
        k_theta_map_par<R, C, 64><<<dim3(nblk(nbox, 64), nblk(hout, 64), nm), 256, MapParShape<R, C, 64>::smem, s>>>(
            (int)nbox, Lc, nin, nout, ME, MD, in, out);
    }
    MLFMA_LAUNCH_CHECK();
}

// ============================================================== pipeline
// One pass of the far field for NR right-hand sides (charges qs[r n + j], potentials
// phis[r n + j]; signatures of level l r nbox_l K_l apart).  C2M, M2L and L2O take all NR
// at once; the interpolation steps run per right-hand side on the shared spectral scratch.
// Upward pass (with each level's M2L beside it once the level's F is complete), then L2L down
// the levels, then L2O at every level with leaves (after near_done, when the near field runs
// on another stream: L2O adds to what it wrote; each level's local signatures stay in place
// after its L2L, so L2O can come last).
template <typename R, int NR>
static void far_pipeline(Plan& p, const void* qs_v, void* phis_v, void* grads_v, cudaEvent_t near_done) {
    using C = typename Cx<R>::T;
    cudaStream_t s = p.stream;
    const C* qs = (const C*)qs_v;
    C* phis = (C*)phis_v;
    const R k = (R)p.k;
    const int64_t sn = p.n;
    auto sF = [&](int l) { return p.lev[l].nbox * p.far[l].K; };
    // M2L of a level needs only that level's F: unless stage timings are being taken, it runs
    // on its own stream as soon as the upward pass has completed F (the fork and join are
    // events, kept as graph edges in a captured apply); the downward pass starts after the
    // last of them
    const bool mfork = p.mstream && !p.profiling;
    // ---- upward pass: C2M at every far level's leaves, M2M from the deepest level up
    auto upward = [&](int l) {
        FarLevel& F = p.far[l];
        TreeLevel& T = p.lev[l];
        if (T.nleaf > 0) {
            StageTimer st(p, MLFMA_STAGE_C2M, l, (T.n_small_leaves > 0) + (T.n_big_leaves > 0));
            if (T.n_small_leaves > 0) {
                k_c2m<R, C, NR><<<nblk(T.n_small_leaves, 4), 128, 0, s>>>(T.n_small_leaves, T.small_leaves, T.begin,
                                                                        T.end, T.center, p.pos, qs, sn, (const R*)F.dirs,
                                                                        F.K, k, (C*)F.F, sF(l));
                MLFMA_LAUNCH_CHECK();
            }
            if (T.n_big_leaves > 0) {
                k_c2m_big<R, C, NR><<<dim3((unsigned)T.n_big_leaves, nblk(F.K, 128)), 128, 0, s>>>(
                    T.big_leaves, T.begin, T.end, T.center, p.pos, qs, sn, (const R*)F.dirs, F.K, k, (C*)F.F, sF(l));
                MLFMA_LAUNCH_CHECK();
            }
        }
        if (l == p.nlev) return;
        FarLevel& Ch = p.far[l + 1];
        TreeLevel& TC = p.lev[l + 1];
        if (F.dense) {
            // fine pair on the tensor cores: one dense map per right-hand side
            StageTimer st(p, MLFMA_STAGE_M2M, l, NR);
            for (int r = 0; r < NR; ++r)
                launch_dense_m2m_tc(p, TC.nbox, (int)Ch.K, (int)F.K, F.DmTc, TC.parent, TC.key, (const float2*)F.Soct,
                                    (const float2*)Ch.F + r * sF(l + 1), (float2*)F.F + r * sF(l), s);
            return;
        }
        const int Lc = Ch.L;
        const int64_t rows_c = TC.nbox * (int64_t)Ch.nth;
        const int budget = (int)(p.tile_fft / sizeof(C));
        const int CPB = fused_children(p.tile_fused, Ch.nth, Ch.nph, Ch.nph, 0, 0, sizeof(C));
        StageTimer st(p, MLFMA_STAGE_M2M, l, NR * (CPB ? 2 : 3));
        for (int r = 0; r < NR; ++r) {
            const C* Fc = (const C*)Ch.F + r * sF(l + 1);
            C* Fp = (C*)F.F + r * sF(l);
            size_t sm;
            if (CPB) {
                // A+B: forward FFT of the children's rows and theta maps, on chip
                launch_m2m_in<C, R>(CPB, (int)TC.nbox, Fc, Lc, Ch.nth, F.nth, Ch.fft, (const C*)Ch.tw,
                                    (R)(1.0 / Ch.nph), (const R*)F.AtE, (const R*)F.AtD, (C*)F.Y, s);
            } else {
                // A: forward FFT of the children's rows, modes |m| <= Lc
                int RB = tile_rows((int)std::min<int64_t>(rows_c, 1 << 20), budget - Ch.nph, 2 * (Ch.nph + 1));
                sm = ((size_t)2 * RB * (Ch.nph + 1) + Ch.nph) * sizeof(C);
                k_fft_fwd_rows<C, R><<<nblk(rows_c, RB), 128, sm, s>>>((int)rows_c, Fc, Lc, Ch.fft, (const C*)Ch.tw,
                                                                          (R)(1.0 / Ch.nph), RB, FastDiv::make(RB),
                                                                          (C*)F.X);
                MLFMA_LAUNCH_CHECK();
                // B: theta maps per mode
                launch_theta_map<R, C>(p, TC.nbox, Lc, Ch.nth, F.nth, (const R*)F.At, F.AtTc, (const R*)F.AtE,
                                       (const R*)F.AtD, (const C*)F.X, (C*)F.Y, s);
            }
            // C: z-shift per mode, inverse FFT, xy-shift, sum over children
            const int pbudget = (int)(p.tile_parent / sizeof(C));
            const int RT = balanced_rows(F.nth, tile_rows(F.nth, pbudget - F.nph, 8 * (F.nph + 1)));
            if (RT < kParentMinRows && RT < F.nth) {   // coarse pair: quadrants in turn, taller row tiles
                const int RQ = balanced_rows(F.nth, tile_rows(F.nth, pbudget - F.nph, 3 * F.nph + 2));
                sm = ((size_t)3 * RQ * (F.nph + 1) + F.nph) * sizeof(C);
                k_m2m_fft_out_q<C><<<dim3((unsigned)T.nbox, nblk(F.nth, RQ)), 128, sm, s>>>(
                    T.child_begin, T.child_end, TC.key, (int)TC.nbox, (const C*)F.Y, Lc, F.nth, F.fft, (const C*)F.tw,
                    (const C*)F.Sz, (const C*)F.Sxy, RQ, FastDiv::make(RQ), FastDiv::make(F.nph),
                    FastDiv::make(F.nph - (2 * Lc + 1)), Fp);
            } else {
                sm = ((size_t)8 * RT * (F.nph + 1) + F.nph) * sizeof(C);
                k_m2m_fft_out<C><<<dim3((unsigned)T.nbox, nblk(F.nth, RT)), 128, sm, s>>>(
                    T.child_begin, T.child_end, TC.key, (int)TC.nbox, (const C*)F.Y, Lc, F.nth, F.fft, (const C*)F.tw,
                    (const C*)F.Sz, (const C*)F.Sxy, RT, FastDiv::make(RT), FastDiv::make(F.nph), Fp);
            }
            MLFMA_LAUNCH_CHECK();
        }
    };
    for (int l = p.nlev; l >= p.top; --l) {
        upward(l);
        if (mfork) {
            MLFMA_CUDA(cudaEventRecord(p.ev_mfork, s));
            MLFMA_CUDA(cudaStreamWaitEvent(p.mstream, p.ev_mfork, 0));
            launch_m2l<R, C, NR>(p, l, p.mstream);
        }
    }
    if (mfork) {
        MLFMA_CUDA(cudaEventRecord(p.ev_mdone, p.mstream));
        MLFMA_CUDA(cudaStreamWaitEvent(s, p.ev_mdone, 0));
    }
    // ---- downward pass: M2L (unless it ran beside the upward pass), L2L, L2O
    for (int l = p.top; l <= p.nlev; ++l) {
        FarLevel& F = p.far[l];
        TreeLevel& T = p.lev[l];
        TreeLevel& TP = p.lev[l - 1];
        if (!mfork) {
            StageTimer st(p, MLFMA_STAGE_M2L, l, m2l_launches<C, NR>(F.K, TP.nbox, F.T1 != nullptr));
            launch_m2l<R, C, NR>(p, l, s);
        }
        if (l > p.top && p.far[l - 1].dense) {
            // fine pair on the tensor cores: one dense map per right-hand side, added to G
            FarLevel& Pf = p.far[l - 1];
            StageTimer st(p, MLFMA_STAGE_L2L, l, NR);
            for (int r = 0; r < NR; ++r)
                launch_dense_l2l_tc(p, T.nbox, (int)Pf.K, (int)F.K, Pf.DlTc, T.parent, T.key, (const float2*)Pf.Soct,
                                    (const float2*)Pf.G + r * sF(l - 1), (float2*)F.G + r * sF(l), s);
        } else if (l > p.top) {
            FarLevel& Pf = p.far[l - 1];
            const int Lc = F.L;
            const int CPB =
                fused_children(p.tile_fused, F.nth, F.nph, F.nph + 1, (2 * Lc + 1) * Pf.nth, 2 * Lc + 1, sizeof(C));
            StageTimer st(p, MLFMA_STAGE_L2L, l, NR * ((CPB ? 2 : 3) + (T.n_orphans > 0)));
            const int budget = (int)(p.tile_fft / sizeof(C));
            const int pbudget = (int)(p.tile_parent / sizeof(C));
            const int RT = balanced_rows(Pf.nth, tile_rows(Pf.nth, pbudget - Pf.nph, 8 * (Pf.nph + 1)));
            for (int r = 0; r < NR; ++r) {
                const C* Gp = (const C*)Pf.G + r * sF(l - 1);
                C* Gc = (C*)F.G + r * sF(l);
                size_t sm;
                if (RT < kParentMinRows && RT < Pf.nth) {   // coarse pair: quadrants in turn, taller row tiles
                    const int RQ = balanced_rows(Pf.nth, tile_rows(Pf.nth, pbudget - Pf.nph, 3 * Pf.nph + 2));
                    sm = ((size_t)3 * RQ * (Pf.nph + 1) + Pf.nph) * sizeof(C);
                    k_l2l_fft_in_q<C, R><<<dim3((unsigned)TP.nbox, nblk(Pf.nth, RQ)), 128, sm, s>>>(
                        TP.child_begin, TP.child_end, T.key, (int)T.nbox, Gp, Lc, Pf.nth, Pf.fft, (const C*)Pf.tw,
                        (const C*)Pf.Sz, (const C*)Pf.Sxy, RQ, FastDiv::make(RQ), FastDiv::make(Pf.nph),
                        (R)(1.0 / Pf.nph), (C*)Pf.Y);
                } else {
                    sm = ((size_t)8 * RT * (Pf.nph + 1) + Pf.nph) * sizeof(C);
                    k_l2l_fft_in<C, R><<<dim3((unsigned)TP.nbox, nblk(Pf.nth, RT)), 128, sm, s>>>(
                        TP.child_begin, TP.child_end, T.key, (int)T.nbox, Gp, Lc, Pf.nth, Pf.fft, (const C*)Pf.tw,
                        (const C*)Pf.Sz, (const C*)Pf.Sxy, RT, FastDiv::make(RT), FastDiv::make(Pf.nph),
                        (R)(1.0 / Pf.nph), (C*)Pf.Y);
                }
                MLFMA_LAUNCH_CHECK();
                if (T.n_orphans > 0) {
                    const int64_t tot = T.n_orphans * (2 * Lc + 1) * Pf.nth;
                    k_zero_orphans<C><<<nblk(tot, 256), 256, 0, s>>>(T.orphans, T.n_orphan_ranges, T.n_orphans,
                                                                     (int)T.nbox, 2 * Lc + 1, Pf.nth, (C*)Pf.Y);
                    MLFMA_LAUNCH_CHECK();
                }
                if (CPB) {
                    // theta maps and inverse FFT of the children's rows, on chip; added to G
                    launch_l2l_out<C, R>(CPB, (int)T.nbox, (const C*)Pf.Y, Lc, F.nth, Pf.nth, F.fft, (const C*)F.tw,
                                         (const R*)Pf.BtE, (const R*)Pf.BtD, Gc, s);
                } else {
                    launch_theta_map<R, C>(p, T.nbox, Lc, Pf.nth, F.nth, (const R*)Pf.Bt, Pf.BtTc, (const R*)Pf.BtE,
                                           (const R*)Pf.BtD, (const C*)Pf.Y, (C*)Pf.X, s);
                    const int64_t rows_c = T.nbox * (int64_t)F.nth;
                    int RB = tile_rows((int)std::min<int64_t>(rows_c, 1 << 20), budget - F.nph, 2 * (F.nph + 1));
                    sm = ((size_t)2 * RB * (F.nph + 1) + F.nph) * sizeof(C);
                    k_l2l_fft_out<C><<<nblk(rows_c, RB), 128, sm, s>>>((int)rows_c, (const C*)Pf.X, Lc, F.fft,
                                                                        (const C*)F.tw, RB, FastDiv::make(RB), Gc);
                    MLFMA_LAUNCH_CHECK();
                }
            }
        }
    }
    // ---- L2O at every level with leaves (after the near field)
    if (near_done) MLFMA_CUDA(cudaStreamWaitEvent(s, near_done, 0));
    for (int l = p.top; l <= p.nlev; ++l) {
        FarLevel& F = p.far[l];
        TreeLevel& T = p.lev[l];
        if (T.nleaf > 0) {
            StageTimer st(p, MLFMA_STAGE_L2O, l, (T.n_small_leaves > 0) + (T.n_big_tiles > 0));
            if (T.n_small_leaves > 0) {
                if (grads_v)
                    k_l2o<R, C, true, 1><<<nblk(T.n_small_leaves, 4), 128, 0, s>>>(
                        T.n_small_leaves, T.small_leaves, T.begin, T.end, T.center, p.pos, (const R*)F.dirs, F.K, k,
                        (const C*)F.G, sF(l), phis, sn, (C*)grads_v);
                else
                    k_l2o<R, C, false, NR><<<nblk(T.n_small_leaves, 4), 128, 0, s>>>(
                        T.n_small_leaves, T.small_leaves, T.begin, T.end, T.center, p.pos, (const R*)F.dirs, F.K, k,
                        (const C*)F.G, sF(l), phis, sn, nullptr);
                MLFMA_LAUNCH_CHECK();
            }
            if (T.n_big_tiles > 0) {
                if (grads_v)
                    k_l2o_big<R, C, true, 1><<<(unsigned)T.n_big_tiles, 128, 0, s>>>(
                        T.big_tiles, T.begin, T.end, T.center, p.pos, (const R*)F.dirs, F.K, k, (const C*)F.G, sF(l), phis,
                        sn, (C*)grads_v);
                else
                    k_l2o_big<R, C, false, NR><<<(unsigned)T.n_big_tiles, 128, 0, s>>>(
                        T.big_tiles, T.begin, T.end, T.center, p.pos, (const R*)F.dirs, F.K, k, (const C*)F.G, sF(l), phis,
                        sn, nullptr);
                MLFMA_LAUNCH_CHECK();
            }
        }
    }
}

// allow a kernel the device's opt-in shared memory per block minus its static shared memory
template <typename K>
static void allow_max_smem(K kernel) {
    int dev = 0, optin = 0;
    MLFMA_CUDA(cudaGetDevice(&dev));
    MLFMA_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    MLFMA_CUDA(cudaFuncGetAttributes(&fa, kernel));
    MLFMA_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes));
}

template <typename C, typename R>
static void prepare_fft_kernels() {
    // one row tile of a long transform (e.g. 9 n complex128 for n = 400) can exceed 48 KB
    allow_max_smem(k_m2m_fft_out<C>);
    allow_max_smem(k_l2l_fft_in<C, R>);
    allow_max_smem(k_m2m_fft_out_q<C>);
    allow_max_smem(k_l2l_fft_in_q<C, R>);
    allow_max_smem(k_fft_fwd_rows<C, R>);
    // fused level pairs: budgets above 48 KB (autotuner candidates) need the opt-in limit
    allow_max_smem(k_m2m_in<C, R, 2>);
    allow_max_smem(k_m2m_in<C, R, 4>);
    allow_max_smem(k_m2m_in<C, R, 8>);
    allow_max_smem(k_m2m_in<C, R, 16>);
    allow_max_smem(k_l2l_out<C, R, 2>);
    allow_max_smem(k_l2l_out<C, R, 4>);
    allow_max_smem(k_l2l_out<C, R, 8>);
    allow_max_smem(k_l2l_out<C, R, 16>);
    allow_max_smem(k_l2l_fft_out<C>);
    allow_max_smem(k_theta_map_par<R, C, 32>);
    allow_max_smem(k_theta_map_par<R, C, 64>);
}

void prepare_kernels(Plan& p) {
    if (p.prec == MLFMA_PREC_FP64) prepare_fft_kernels<double2, double>();
    else prepare_fft_kernels<float2, float>();
    if (p.prec == MLFMA_PREC_FP32_TF32X3 || p.prec == MLFMA_PREC_FP32_BF16X3) {
        prepare_theta_tc();
        prepare_dense_tc();
    }
    if (p.prec == MLFMA_PREC_FP64) {
        allow_max_smem(k_m2l<double, double2, 1, M2LShape<double2, 1>::NW, false>);
        allow_max_smem(k_m2l<double, double2, kMaxNR, M2LShape<double2, kMaxNR>::NW, false>);
        allow_max_smem(k_m2l<double, double2, 1, M2LShape<double2, 1>::NW, true>);
        allow_max_smem(k_m2l<double, double2, kMaxNR, M2LShape<double2, kMaxNR>::NW, true>);
        allow_max_smem(k_m2l_tail<double2, 16>);
    } else {
        allow_max_smem(k_m2l<float, float2, 1, M2LShape<float2, 1>::NW, false>);
        allow_max_smem(k_m2l<float, float2, kMaxNR, M2LShape<float2, kMaxNR>::NW, false>);
        allow_max_smem(k_m2l<float, float2, 1, M2LShape<float2, 1>::NW, true>);
        allow_max_smem(k_m2l<float, float2, kMaxNR, M2LShape<float2, kMaxNR>::NW, true>);
    }
}

void far_apply(Plan& p, const void* qs, void* phis, void* grads, int nr, cudaEvent_t near_done) {
    if (!p.top) return;
    if (nr != 1 && nr != kMaxNR) fail(MLFMA_ERR_INVALID_ARG, "right-hand sides per pass %d", nr);
    if (p.prec == MLFMA_PREC_FP64) {
        if (nr == 1) far_pipeline<double, 1>(p, qs, phis, grads, near_done);
        else far_pipeline<double, kMaxNR>(p, qs, phis, nullptr, near_done);
    } else {
        if (nr == 1) far_pipeline<float, 1>(p, qs, phis, grads, near_done);
        else far_pipeline<float, kMaxNR>(p, qs, phis, nullptr, near_done);
    }
}

}  // namespace mlfma
