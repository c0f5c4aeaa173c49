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
// nodes.  The shift to the parent centre factors into a theta-only part
// e^{-ik cos(theta') dz} (applied per mode, before the inverse DFT, which lets the
// two children stacked in z share one inverse DFT) and a theta-phi part applied on
// the parent grid.  Anterpolation is the weighted transpose of the same steps.
#include <cstdio>

#include "common.cuh"

namespace mlfma {

__device__ __forceinline__ void sc(float x, float& s, float& c) { sincosf(x, &s, &c); }
__device__ __forceinline__ void sc(double x, double& s, double& c) { sincos(x, &s, &c); }

static inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

// rows of a tile: as many as fit in ``budget`` complex slots at ``per_row`` each, in [1, nrows]
static inline int tile_rows(int nrows, int budget, int per_row) {
    int r = budget > 0 ? budget / per_row : 1;
    return std::max(1, std::min(nrows, r));
}

// ============================================================== C2M (warp per leaf)
constexpr int kC2MPass = 4;   // samples per lane per pass

template <typename R, typename C>
__global__ void __launch_bounds__(128) k_c2m(int64_t nleaf, const int* __restrict__ leaf_box, const int* __restrict__ begin,
                                             const int* __restrict__ end, const double* __restrict__ center,
                                             const double* __restrict__ pos, const C* __restrict__ qs,
                                             const R* __restrict__ dirs, int64_t K, R k, C* __restrict__ F) {
    __shared__ R sp[4][32][3];
    __shared__ C sq[4][32];
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t w = (int64_t)blockIdx.x * 4 + wl;
    if (w >= nleaf) return;
    const int b = leaf_box[w];
    const int b0 = begin[b], b1 = end[b];
    const double cx = center[3 * b], cy = center[3 * b + 1], cz = center[3 * b + 2];
    C* Fb = F + (int64_t)b * K;
    for (int64_t p0 = 0; p0 < K; p0 += 32 * kC2MPass) {
        C acc[kC2MPass];
        R d[kC2MPass][3];
#pragma unroll
        for (int u = 0; u < kC2MPass; ++u) {
            acc[u] = cmake<C>(0, 0);
            int64_t p = p0 + lane + 32 * u;
            int64_t pp = p < K ? p : K - 1;
            d[u][0] = -k * dirs[4 * pp]; d[u][1] = -k * dirs[4 * pp + 1]; d[u][2] = -k * dirs[4 * pp + 2];
        }
        for (int j0 = b0; j0 < b1; j0 += 32) {
            int j = j0 + lane;
            if (j < b1) {
                sp[wl][lane][0] = (R)(pos[3 * (int64_t)j] - cx);
                sp[wl][lane][1] = (R)(pos[3 * (int64_t)j + 1] - cy);
                sp[wl][lane][2] = (R)(pos[3 * (int64_t)j + 2] - cz);
                sq[wl][lane] = qs[j];
            }
            __syncwarp();
            int cnt = min(32, b1 - j0);
            for (int t = 0; t < cnt; ++t) {
                R x = sp[wl][t][0], y = sp[wl][t][1], z = sp[wl][t][2];
                C q = sq[wl][t];
#pragma unroll
                for (int u = 0; u < kC2MPass; ++u) {
                    R ph = d[u][0] * x + d[u][1] * y + d[u][2] * z;
                    R s, c;
                    sc(ph, s, c);
                    cfma(acc[u], q, cmake<C>(c, s));
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int u = 0; u < kC2MPass; ++u) {
            int64_t p = p0 + lane + 32 * u;
            if (p < K) Fb[p] = acc[u];
        }
    }
}

// ============================================================== L2O (warp per leaf, lanes = point x slice)
template <typename R, typename C>
__global__ void __launch_bounds__(128) k_l2o(int64_t nleaf, const int* __restrict__ leaf_box, const int* __restrict__ begin,
                                             const int* __restrict__ end, const double* __restrict__ center,
                                             const double* __restrict__ pos, const R* __restrict__ dirs, int64_t K, R k,
                                             const C* __restrict__ G, C* __restrict__ phis) {
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
        C acc = cmake<C>(0, 0);
        for (int64_t p = sl; p < K; p += S) {
            R ph = k * (dirs[4 * p] * x + dirs[4 * p + 1] * y + dirs[4 * p + 2] * z);
            R s, c;
            sc(ph, s, c);
            R wp = dirs[4 * p + 3];
            cfma(acc, cmake<C>(wp * c, wp * s), Gb[p]);
        }
        for (int o = 16; o >= P; o >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        }
        if (sl == 0 && tp < np) {
            // (ik / 4 pi) * acc
            const R f = k / (R)(4.0 * M_PI);
            C v = phis[j];
            v.x += -f * acc.y;
            v.y += f * acc.x;
            phis[j] = v;
        }
    }
}

// ============================================================== M2L (CTA per parent: its children are the targets)
constexpr int kMaxSrc = 26 * 8;

template <typename R, typename C>
__global__ void __launch_bounds__(256) k_m2l(const int* __restrict__ pcb, const int* __restrict__ pce, const int* __restrict__ pcoll,
                                             const int* __restrict__ ijk, const int* __restrict__ off343,
                                             const C* __restrict__ F, const C* __restrict__ T, int64_t K, C* __restrict__ G) {
    __shared__ int s_src[kMaxSrc];
    __shared__ signed short s_oi[kMaxSrc][8];
    __shared__ int s_ns;
    const int P = blockIdx.x;
    const int t0 = pcb[P], t1 = pce[P];
    if (t0 >= t1) return;
    const int nt = t1 - t0;
    if (threadIdx.x == 0) {
        int ns = 0;
        for (int sl = 0; sl < 27; ++sl) {
            int q = pcoll[27 * P + sl];
            if (q < 0 || q == P) continue;
            for (int s = pcb[q]; s < pce[q]; ++s) s_src[ns++] = s;
        }
        s_ns = ns;
    }
    __syncthreads();
    const int ns = s_ns;
    for (int idx = threadIdx.x; idx < ns * 8; idx += blockDim.x) {
        int si = idx >> 3, t = idx & 7;
        int oi = -1;
        if (t < nt) {
            int s = s_src[si];
            int dx = ijk[3 * (t0 + t)] - ijk[3 * s], dy = ijk[3 * (t0 + t) + 1] - ijk[3 * s + 1],
                dz = ijk[3 * (t0 + t) + 2] - ijk[3 * s + 2];
            if (max(abs(dx), max(abs(dy), abs(dz))) >= 2) oi = off343[(dx + 3) + 7 * (dy + 3) + 49 * (dz + 3)];
        }
        s_oi[si][t] = (signed short)oi;
    }
    __syncthreads();
    const int64_t p = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    if (p >= K) return;
    C acc[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) acc[t] = cmake<C>(0, 0);
    for (int si = 0; si < ns; ++si) {
        const C f = F[(int64_t)s_src[si] * K + p];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            int oi = s_oi[si][t];
            if (oi >= 0) cfma(acc[t], T[(int64_t)oi * K + p], f);
        }
    }
#pragma unroll
    for (int t = 0; t < 8; ++t)
        if (t < nt) G[(int64_t)(t0 + t) * K + p] = acc[t];
}

// ============================================================== interpolation building blocks
// forward DFT in phi of the rows of one box: X[b][mi][i] = scale sum_j F[b][i][j] tw[(sgn m j) mod nph]
template <typename C>
__global__ void k_dft_rows(int64_t nbox, const C* __restrict__ F, int nth, int nph, int L, int sgn, const C* __restrict__ tw,
                           typename std::conditional<sizeof(C) == 8, float, double>::type scale, int RT, C* __restrict__ X,
                           const C* __restrict__ pre, int pre_q) {
    extern __shared__ unsigned char smem_raw[];
    C* rows = reinterpret_cast<C*>(smem_raw);
    const int ld = nph + 1;
    C* stw = rows + RT * ld;
    const int64_t b = blockIdx.x;
    const int i0 = blockIdx.y * RT;
    const int nr = min(RT, nth - i0);
    const int64_t K = (int64_t)nth * nph;
    for (int idx = threadIdx.x; idx < nr * nph; idx += blockDim.x) {
        int r = idx / nph, j = idx % nph;
        C v = F[b * K + (int64_t)(i0 + r) * nph + j];
        if (pre) v = cmul(cconj(pre[(int64_t)pre_q * K + (int64_t)(i0 + r) * nph + j]), v);
        rows[r * ld + j] = v;
    }
    for (int j = threadIdx.x; j < nph; j += blockDim.x) stw[j] = tw[j];
    __syncthreads();
    const int nm = 2 * L + 1;
    for (int idx = threadIdx.x; idx < nr * nm; idx += blockDim.x) {
        int r = idx % nr, mi = idx / nr;
        int m = mi - L;
        int step = ((sgn * m) % nph + nph) % nph;
        int kk = 0;
        C acc = cmake<C>(0, 0);
        const C* row = rows + r * ld;
        for (int j = 0; j < nph; ++j) {
            cfma(acc, row[j], stw[kk]);
            kk += step;
            if (kk >= nph) kk -= nph;
        }
        acc.x *= scale; acc.y *= scale;
        X[(b * nm + mi) * nth + i0 + r] = acc;
    }
}

// theta map per mode: out[c][mi][o] = sum_in M[|m|][in][o] in[c][mi][in]
constexpr int kMapCB = 8;

template <typename R, typename C>
__global__ void k_theta_map(int64_t nbox, int Lc, int nin, int nout, const R* __restrict__ M, const C* __restrict__ in,
                            C* __restrict__ out) {
    extern __shared__ unsigned char smem_raw[];
    C* xin = reinterpret_cast<C*>(smem_raw);
    const int mi = blockIdx.y;
    const int nm = 2 * Lc + 1;
    const int m = abs(mi - Lc);
    const int64_t c0 = (int64_t)blockIdx.x * kMapCB;
    const int nc = (int)((nbox - c0) < kMapCB ? (nbox - c0) : kMapCB);
    for (int idx = threadIdx.x; idx < nc * nin; idx += blockDim.x) {
        int cl = idx / nin, i = idx % nin;
        xin[cl * nin + i] = in[((c0 + cl) * nm + mi) * nin + i];
    }
    __syncthreads();
    const R* Mm = M + (int64_t)m * nin * nout;
    for (int idx = threadIdx.x; idx < nc * nout; idx += blockDim.x) {
        int cl = idx / nout, o = idx % nout;
        C acc = cmake<C>(0, 0);
        const C* x = xin + cl * nin;
        for (int i = 0; i < nin; ++i) crfma(acc, Mm[(int64_t)i * nout + o], x[i]);
        out[((c0 + cl) * nm + mi) * nout + o] = acc;
    }
}

// M2M final step: F[P][i'][j'] = sum_q Sxy[q][i'][j'] sum_mi e^{i m phi'_j'} W_q[i'][mi],
// W_q[i'][mi] = sum_{children c = (q, sz)} Sz[sz][i'] Y[c][mi][i'].  Non-leaf parents only.
template <typename C>
__global__ void k_m2m_out(const int* __restrict__ cb, const int* __restrict__ ce, const uint64_t* __restrict__ ckey,
                          const C* __restrict__ Y, int Lc, int nthp, int nphp, const C* __restrict__ tw, const C* __restrict__ Sz,
                          const C* __restrict__ Sxy, int RT, C* __restrict__ Fp) {
    extern __shared__ unsigned char smem_raw[];
    const int nm = 2 * Lc + 1;
    C* W = reinterpret_cast<C*>(smem_raw);           // [4][RT][nm]
    C* stw = W + 4 * RT * nm;                         // [nphp]
    __shared__ int s_has[4];
    const int P = blockIdx.x;
    const int c0 = cb[P], c1 = ce[P];
    if (c0 >= c1) return;
    const int i0 = blockIdx.y * RT;
    const int nr = min(RT, nthp - i0);
    if (threadIdx.x < 4) s_has[threadIdx.x] = 0;
    for (int idx = threadIdx.x; idx < 4 * RT * nm; idx += blockDim.x) W[idx] = cmake<C>(0, 0);
    for (int j = threadIdx.x; j < nphp; j += blockDim.x) stw[j] = tw[j];
    __syncthreads();
    for (int c = c0; c < c1; ++c) {
        const int oct = (int)(ckey[c] & 7);
        const int q = oct & 3, sz = oct >> 2;
        if (threadIdx.x == 0) s_has[q] = 1;
        for (int idx = threadIdx.x; idx < nr * nm; idx += blockDim.x) {
            int r = idx % nr, mi = idx / nr;
            C y = Y[((int64_t)c * nm + mi) * nthp + i0 + r];
            cfma(W[(q * RT + r) * nm + mi], Sz[sz * nthp + i0 + r], y);
        }
        __syncthreads();
    }
    const int64_t Kp = (int64_t)nthp * nphp;
    for (int idx = threadIdx.x; idx < nr * nphp; idx += blockDim.x) {
        int r = idx / nphp, j = idx % nphp;
        C acc = cmake<C>(0, 0);
        for (int q = 0; q < 4; ++q) {
            if (!s_has[q]) continue;
            const C* w = W + (q * RT + r) * nm;
            // e^{+i m phi_j} = tw[(-m j) mod n]; start at m = -Lc
            int step = j;                       // index increment per unit m for e^{+i m phi_j}: tw[-j]
            int kk = (int)(((int64_t)Lc * j) % nphp);   // (-(-Lc) j) ... tw index of e^{+i(-Lc) phi_j} = tw[Lc j]
            C s = cmake<C>(0, 0);
            for (int mi = 0; mi < nm; ++mi) {
                cfma(s, w[mi], stw[kk]);
                kk -= step;
                if (kk < 0) kk += nphp;
            }
            cfma(acc, Sxy[(int64_t)q * Kp + (int64_t)(i0 + r) * nphp + j], s);
        }
        Fp[(int64_t)P * Kp + (int64_t)(i0 + r) * nphp + j] = acc;
    }
}

// L2L first step (per parent, per xy-quadrant q present):
//   V_q[i'][mi] = (1/nph_p) sum_j' conj(Sxy[q][i'][j']) G_P[i'][j'] e^{+i m phi'_j'}
//   Yc[c][mi][i'] = conj(Sz[sz][i']) V_q[i'][mi] for each child c = (q, sz)
template <typename C>
__global__ void k_l2l_in(const int* __restrict__ cb, const int* __restrict__ ce, const uint64_t* __restrict__ ckey,
                         const C* __restrict__ Gp, int Lc, int nthp, int nphp, const C* __restrict__ tw, const C* __restrict__ Sz,
                         const C* __restrict__ Sxy, int RT, C* __restrict__ Y) {
    extern __shared__ unsigned char smem_raw[];
    const int nm = 2 * Lc + 1;
    const int ld = nphp + 1;
    C* rows = reinterpret_cast<C*>(smem_raw);        // [RT][ld]
    C* stw = rows + RT * ld;
    __shared__ int s_child[4][2];
    const int P = blockIdx.x;
    const int c0 = cb[P], c1 = ce[P];
    if (c0 >= c1) return;
    const int i0 = blockIdx.y * RT;
    const int nr = min(RT, nthp - i0);
    const int64_t Kp = (int64_t)nthp * nphp;
    if (threadIdx.x < 8) s_child[threadIdx.x >> 1][threadIdx.x & 1] = -1;
    for (int j = threadIdx.x; j < nphp; j += blockDim.x) stw[j] = tw[j];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int c = c0; c < c1; ++c) {
            int oct = (int)(ckey[c] & 7);
            s_child[oct & 3][oct >> 2] = c;
        }
    const typename std::conditional<sizeof(C) == 8, float, double>::type inv = 1.0 / nphp;
    for (int q = 0; q < 4; ++q) {
        __syncthreads();
        if (s_child[q][0] < 0 && s_child[q][1] < 0) continue;
        for (int idx = threadIdx.x; idx < nr * nphp; idx += blockDim.x) {
            int r = idx / nphp, j = idx % nphp;
            int64_t g = (int64_t)(i0 + r) * nphp + j;
            rows[r * ld + j] = cmul(cconj(Sxy[(int64_t)q * Kp + g]), Gp[(int64_t)P * Kp + g]);
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < nr * nm; idx += blockDim.x) {
            int r = idx % nr, mi = idx / nr;
            int m = mi - Lc;
            int step = ((-m) % nphp + nphp) % nphp;      // e^{+i m phi_j} = tw[(-m j) mod n]
            int kk = 0;
            C acc = cmake<C>(0, 0);
            const C* row = rows + r * ld;
            for (int j = 0; j < nphp; ++j) {
                cfma(acc, row[j], stw[kk]);
                kk += step;
                if (kk >= nphp) kk -= nphp;
            }
            acc.x *= inv; acc.y *= inv;
            for (int sz = 0; sz < 2; ++sz) {
                int c = s_child[q][sz];
                if (c < 0) continue;
                Y[((int64_t)c * nm + mi) * nthp + i0 + r] = cmul(cconj(Sz[sz * nthp + i0 + r]), acc);
            }
        }
    }
}

// L2L last step: G_c[i][j] += sum_mi H[c][mi][i] e^{-i m phi_j}
template <typename C>
__global__ void k_l2l_out(int64_t nbox, const C* __restrict__ H, int Lc, int nth, int nph, const C* __restrict__ tw, int RT,
                          C* __restrict__ G) {
    extern __shared__ unsigned char smem_raw[];
    const int nm = 2 * Lc + 1;
    C* h = reinterpret_cast<C*>(smem_raw);            // [RT][nm]
    C* stw = h + RT * nm;
    const int64_t c = blockIdx.x;
    const int i0 = blockIdx.y * RT;
    const int nr = min(RT, nth - i0);
    for (int idx = threadIdx.x; idx < nr * nm; idx += blockDim.x) {
        int r = idx % nr, mi = idx / nr;
        h[r * nm + mi] = H[(c * nm + mi) * nth + i0 + r];
    }
    for (int j = threadIdx.x; j < nph; j += blockDim.x) stw[j] = tw[j];
    __syncthreads();
    const int64_t K = (int64_t)nth * nph;
    for (int idx = threadIdx.x; idx < nr * nph; idx += blockDim.x) {
        int r = idx / nph, j = idx % nph;
        // e^{-i m phi_j} = tw[(m j) mod n], m from -Lc
        int kk = (int)((((int64_t)(-Lc) * j) % nph + nph) % nph);
        C acc = cmake<C>(0, 0);
        const C* hr = h + r * nm;
        for (int mi = 0; mi < nm; ++mi) {
            cfma(acc, hr[mi], stw[kk]);
            kk += j;
            if (kk >= nph) kk -= nph;
        }
        int64_t g = c * K + (int64_t)(i0 + r) * nph + j;
        G[g] = cadd(G[g], acc);
    }
}

// ============================================================== pipeline
template <typename R>
static void far_pipeline(Plan& p, const void* qs_v, void* phis_v) {
    using C = typename Cx<R>::T;
    cudaStream_t s = p.stream;
    const C* qs = (const C*)qs_v;
    C* phis = (C*)phis_v;
    const R k = (R)p.k;
    const size_t smem_cap = 96 * 1024;
    // ---- upward pass: C2M at every far level's leaves, M2M from the deepest level up
    for (int l = p.nlev; l >= p.top; --l) {
        FarLevel& F = p.far[l];
        TreeLevel& T = p.lev[l];
        if (T.nleaf > 0) {
            k_c2m<R, C><<<nblk(T.nleaf, 4), 128, 0, s>>>(T.nleaf, p.leaf_box + p.leaf_first[l], T.begin, T.end, T.center, p.pos,
                                                       qs, (const R*)F.dirs, F.K, k, (C*)F.F);
            MLFMA_LAUNCH_CHECK();
        }
        if (l == p.nlev) continue;
        FarLevel& Ch = p.far[l + 1];
        TreeLevel& TC = p.lev[l + 1];
        const int Lc = Ch.L, nm = 2 * Lc + 1;
        // A: forward DFT of the children's rows
        int RT = tile_rows(Ch.nth, (int)(40 * 1024 / sizeof(C)) - Ch.nph, Ch.nph + 1);
        size_t sm = ((size_t)RT * (Ch.nph + 1) + Ch.nph) * sizeof(C);
        k_dft_rows<C><<<dim3((unsigned)TC.nbox, nblk(Ch.nth, RT)), 128, sm, s>>>(TC.nbox, (const C*)Ch.F, Ch.nth, Ch.nph, Lc,
                                                                                   1, (const C*)Ch.tw, (R)(1.0 / Ch.nph), RT,
                                                                                   (C*)F.X, nullptr, 0);
        MLFMA_LAUNCH_CHECK();
        // B: theta maps per mode
        sm = (size_t)kMapCB * Ch.nth * sizeof(C);
        k_theta_map<R, C><<<dim3(nblk(TC.nbox, kMapCB), nm), 128, sm, s>>>(TC.nbox, Lc, Ch.nth, F.nth, (const R*)F.At,
                                                                              (const C*)F.X, (C*)F.Y);
        MLFMA_LAUNCH_CHECK();
        // C: z-shift per mode, inverse DFT, xy-shift, sum over children
        RT = tile_rows(F.nth, (int)(40 * 1024 / sizeof(C)) - F.nph, 4 * nm);
        sm = ((size_t)4 * RT * nm + F.nph) * sizeof(C);
        if (sm > smem_cap) fail(MLFMA_ERR_UNSUPPORTED, "M2M tile needs %zu bytes of shared memory", sm);
        k_m2m_out<C><<<dim3((unsigned)T.nbox, nblk(F.nth, RT)), 128, sm, s>>>(T.child_begin, T.child_end, TC.key, (const C*)F.Y,
                                                                              Lc, F.nth, F.nph, (const C*)F.tw, (const C*)F.Sz,
                                                                              (const C*)F.Sxy, RT, (C*)F.F);
        MLFMA_LAUNCH_CHECK();
    }
    // ---- downward pass: M2L, L2L, L2O
    for (int l = p.top; l <= p.nlev; ++l) {
        FarLevel& F = p.far[l];
        TreeLevel& T = p.lev[l];
        TreeLevel& TP = p.lev[l - 1];
        {
            int tb = (int)std::min<int64_t>(256, ((F.K + 31) / 32) * 32);
            int ny = nblk(F.K, tb);
            k_m2l<R, C><<<dim3((unsigned)TP.nbox, ny), tb, 0, s>>>(TP.child_begin, TP.child_end, TP.coll, T.ijk, p.off343,
                                                                  (const C*)F.F, (const C*)F.T, F.K, (C*)F.G);
            MLFMA_LAUNCH_CHECK();
        }
        if (l > p.top) {
            FarLevel& Pf = p.far[l - 1];
            const int Lc = F.L, nm = 2 * Lc + 1;
            int RT = tile_rows(Pf.nth, (int)(40 * 1024 / sizeof(C)) - Pf.nph, Pf.nph + 1);
            size_t sm = ((size_t)RT * (Pf.nph + 1) + Pf.nph) * sizeof(C);
            k_l2l_in<C><<<dim3((unsigned)TP.nbox, nblk(Pf.nth, RT)), 128, sm, s>>>(TP.child_begin, TP.child_end, T.key,
                                                                                   (const C*)Pf.G, Lc, Pf.nth, Pf.nph,
                                                                                   (const C*)Pf.tw, (const C*)Pf.Sz,
                                                                                   (const C*)Pf.Sxy, RT, (C*)Pf.Y);
            MLFMA_LAUNCH_CHECK();
            sm = (size_t)kMapCB * Pf.nth * sizeof(C);
            k_theta_map<R, C><<<dim3(nblk(T.nbox, kMapCB), nm), 128, sm, s>>>(T.nbox, Lc, Pf.nth, F.nth, (const R*)Pf.Bt,
                                                                                (const C*)Pf.Y, (C*)Pf.X);
            MLFMA_LAUNCH_CHECK();
            RT = tile_rows(F.nth, (int)(40 * 1024 / sizeof(C)) - F.nph, nm);
            sm = ((size_t)RT * nm + F.nph) * sizeof(C);
            k_l2l_out<C><<<dim3((unsigned)T.nbox, nblk(F.nth, RT)), 128, sm, s>>>(T.nbox, (const C*)Pf.X, Lc, F.nth, F.nph,
                                                                                  (const C*)F.tw, RT, (C*)F.G);
            MLFMA_LAUNCH_CHECK();
        }
        if (T.nleaf > 0) {
            k_l2o<R, C><<<nblk(T.nleaf, 4), 128, 0, s>>>(T.nleaf, p.leaf_box + p.leaf_first[l], T.begin, T.end, T.center, p.pos,
                                                       (const R*)F.dirs, F.K, k, (const C*)F.G, phis);
            MLFMA_LAUNCH_CHECK();
        }
    }
}

void far_apply(Plan& p, const void* qs, void* phis) {
    if (!p.top) return;
    if (p.prec == MLFMA_PREC_FP64) far_pipeline<double>(p, qs, phis);
    else far_pipeline<float>(p, qs, phis);
}

}  // namespace mlfma
