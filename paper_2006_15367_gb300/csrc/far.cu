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

// ============================================================== phi transforms: mixed-radix FFTs in shared memory
// Stockham autosort FFT of several rows at once (length n = prod of radices 2, 3, 4, 5, 7).
// tw[k] = e^{-2 pi i k / n}; inv = true uses e^{+2 pi i k / n} (no 1/n scaling).
template <typename C>
__device__ __forceinline__ C twid(const C* __restrict__ tw, int idx, bool inv) {
    C t = tw[idx];
    if (inv) t.y = -t.y;
    return t;
}

template <int R, typename C>
__device__ __forceinline__ void fft_bfly(const C* __restrict__ a, C* __restrict__ b, int j, int Ns, int n,
                                         const C* __restrict__ tw, bool inv) {
    const int nb = n / R;
    const int k = j % Ns;
    const int tstep = n / (Ns * R);
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        C x = a[j + r * nb];
        if (r > 0) x = cmul(x, twid(tw, k * r * tstep, inv));
        v[r] = x;
    }
    const int idxD = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int kk = 0; kk < R; ++kk) {
        C s = v[0];
#pragma unroll
        for (int r = 1; r < R; ++r) cfma(s, v[r], twid(tw, ((r * kk) % R) * nb, inv));
        b[idxD + kk * Ns] = s;
    }
}

// Transforms nrows rows of length fp.n stored contiguously in buf0; returns the buffer
// holding the result (buf0 or buf1).  All threads of the block take part.
template <typename C>
__device__ C* fft_rows(C* buf0, C* buf1, int nrows, const FftPlan& fp, const C* __restrict__ tw, bool inv) {
    const int n = fp.n;
    C* in = buf0;
    C* out = buf1;
    int Ns = 1;
    for (int st = 0; st < fp.ns; ++st) {
        const int R = fp.r[st];
        const int nb = n / R;
        for (int idx = threadIdx.x; idx < nrows * nb; idx += blockDim.x) {
            const int row = idx / nb, j = idx - row * nb;
            const C* a = in + row * n;
            C* b = out + row * n;
            switch (R) {
                case 2: fft_bfly<2>(a, b, j, Ns, n, tw, inv); break;
                case 3: fft_bfly<3>(a, b, j, Ns, n, tw, inv); break;
                case 4: fft_bfly<4>(a, b, j, Ns, n, tw, inv); break;
                case 5: fft_bfly<5>(a, b, j, Ns, n, tw, inv); break;
                default: fft_bfly<7>(a, b, j, Ns, n, tw, inv); break;
            }
        }
        __syncthreads();
        C* t = in; in = out; out = t;
        Ns *= R;
    }
    return in;
}

__device__ __forceinline__ int wrap(int m, int n) { return m < 0 ? m + n : m; }

// M2M first step: X[c][mi][i] = scale sum_j F[c][i][j] e^{-i m phi_j}, |m| <= Lc, for the rows
// (c, i) of all children (rows are contiguous in F).
template <typename C, typename R>
__global__ void k_fft_fwd_rows(int64_t nrows_tot, const C* __restrict__ F, int nth, int Lc, FftPlan fp,
                               const C* __restrict__ tw, R scale, int RB, C* __restrict__ X) {
    extern __shared__ unsigned char smem_raw[];
    const int n = fp.n, nm = 2 * Lc + 1;
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + RB * n;
    C* stw = buf1 + RB * n;
    const int64_t r0 = (int64_t)blockIdx.x * RB;
    const int nr = (int)((nrows_tot - r0) < RB ? (nrows_tot - r0) : RB);
    for (int idx = threadIdx.x; idx < nr * n; idx += blockDim.x) buf0[idx] = F[r0 * n + idx];
    for (int j = threadIdx.x; j < n; j += blockDim.x) stw[j] = tw[j];
    __syncthreads();
    const C* res = fft_rows(buf0, buf1, nr, fp, stw, false);
    for (int idx = threadIdx.x; idx < nr * nm; idx += blockDim.x) {
        const int row = idx % nr, mi = idx / nr;
        const int64_t r = r0 + row;
        const int64_t c = r / nth;
        const int i = (int)(r - c * nth);
        C v = res[row * n + wrap(mi - Lc, n)];
        v.x *= scale; v.y *= scale;
        X[(c * nm + mi) * nth + i] = v;
    }
}

// M2M last step, per parent P and tile of parent rows i':
//   W_q[i'][m] = sum_{children c = (q, sz)} Sz[sz][i'] Y[c][mi][i']          (z part of the shift, per mode)
//   F_P[i'][j'] = sum_q Sxy[q][i'][j'] sum_m W_q[i'][m] e^{+i m phi'_j'}     (inverse FFT, xy part of the shift)
template <typename C>
__global__ void k_m2m_fft_out(const int* __restrict__ cb, const int* __restrict__ ce, const uint64_t* __restrict__ ckey,
                              const C* __restrict__ Y, int Lc, int nthp, FftPlan fp, const C* __restrict__ tw,
                              const C* __restrict__ Sz, const C* __restrict__ Sxy, int RT, C* __restrict__ Fp) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ int s_child[4][2];
    const int n = fp.n, nm = 2 * Lc + 1;
    const int64_t Kp = (int64_t)nthp * n;
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + RT * n;
    C* acc = buf1 + RT * n;
    C* stw = acc + RT * n;
    const int P = blockIdx.x;
    const int c0 = cb[P], c1 = ce[P];
    if (c0 >= c1) return;
    const int i0 = blockIdx.y * RT;
    const int nr = min(RT, nthp - i0);
    if (threadIdx.x < 8) s_child[threadIdx.x >> 1][threadIdx.x & 1] = -1;
    for (int j = threadIdx.x; j < n; j += blockDim.x) stw[j] = tw[j];
    for (int idx = threadIdx.x; idx < nr * n; idx += blockDim.x) acc[idx] = cmake<C>(0, 0);
    __syncthreads();
    if (threadIdx.x == 0)
        for (int c = c0; c < c1; ++c) {
            const int oct = (int)(ckey[c] & 7);
            s_child[oct & 3][oct >> 2] = c;
        }
    __syncthreads();
    for (int q = 0; q < 4; ++q) {
        const int ca = s_child[q][0], cz = s_child[q][1];
        if (ca < 0 && cz < 0) continue;
        for (int idx = threadIdx.x; idx < nr * n; idx += blockDim.x) buf0[idx] = cmake<C>(0, 0);
        __syncthreads();
        for (int idx = threadIdx.x; idx < nr * nm; idx += blockDim.x) {
            const int r = idx % nr, mi = idx / nr;
            C w = cmake<C>(0, 0);
            if (ca >= 0) cfma(w, Sz[i0 + r], Y[((int64_t)ca * nm + mi) * nthp + i0 + r]);
            if (cz >= 0) cfma(w, Sz[nthp + i0 + r], Y[((int64_t)cz * nm + mi) * nthp + i0 + r]);
            buf0[r * n + wrap(mi - Lc, n)] = w;
        }
        __syncthreads();
        const C* res = fft_rows(buf0, buf1, nr, fp, stw, true);
        for (int idx = threadIdx.x; idx < nr * n; idx += blockDim.x) {
            const int r = idx / n, j = idx - r * n;
            cfma(acc[idx], Sxy[(int64_t)q * Kp + (int64_t)(i0 + r) * n + j], res[idx]);
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < nr * n; idx += blockDim.x) Fp[(int64_t)P * Kp + (int64_t)i0 * n + idx] = acc[idx];
}

// L2L first step, per parent P, tile of parent rows i' and xy-quadrant q with children:
//   V_q[i'][m] = (1/n) sum_j' conj(Sxy[q][i'][j']) G_P[i'][j'] e^{+i m phi'_j'},  |m| <= Lc
//   Y[c][mi][i'] = conj(Sz[sz][i']) V_q[i'][m] for each child c = (q, sz)
template <typename C, typename R>
__global__ void k_l2l_fft_in(const int* __restrict__ cb, const int* __restrict__ ce, const uint64_t* __restrict__ ckey,
                             const C* __restrict__ Gp, int Lc, int nthp, FftPlan fp, const C* __restrict__ tw,
                             const C* __restrict__ Sz, const C* __restrict__ Sxy, int RT, R inv_n, C* __restrict__ Y) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ int s_child[4][2];
    const int n = fp.n, nm = 2 * Lc + 1;
    const int64_t Kp = (int64_t)nthp * n;
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + RT * n;
    C* stw = buf1 + RT * n;
    const int P = blockIdx.x;
    const int c0 = cb[P], c1 = ce[P];
    if (c0 >= c1) return;
    const int i0 = blockIdx.y * RT;
    const int nr = min(RT, nthp - i0);
    if (threadIdx.x < 8) s_child[threadIdx.x >> 1][threadIdx.x & 1] = -1;
    for (int j = threadIdx.x; j < n; j += blockDim.x) stw[j] = tw[j];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int c = c0; c < c1; ++c) {
            const int oct = (int)(ckey[c] & 7);
            s_child[oct & 3][oct >> 2] = c;
        }
    __syncthreads();
    for (int q = 0; q < 4; ++q) {
        const int ca = s_child[q][0], cz = s_child[q][1];
        if (ca < 0 && cz < 0) continue;
        for (int idx = threadIdx.x; idx < nr * n; idx += blockDim.x) {
            const int64_t g = (int64_t)i0 * n + idx;
            buf0[idx] = cmul(cconj(Sxy[(int64_t)q * Kp + g]), Gp[(int64_t)P * Kp + g]);
        }
        __syncthreads();
        const C* res = fft_rows(buf0, buf1, nr, fp, stw, true);
        for (int idx = threadIdx.x; idx < nr * nm; idx += blockDim.x) {
            const int r = idx % nr, mi = idx / nr;
            C v = res[r * n + wrap(mi - Lc, n)];
            v.x *= inv_n; v.y *= inv_n;
            if (ca >= 0) Y[((int64_t)ca * nm + mi) * nthp + i0 + r] = cmul(cconj(Sz[i0 + r]), v);
            if (cz >= 0) Y[((int64_t)cz * nm + mi) * nthp + i0 + r] = cmul(cconj(Sz[nthp + i0 + r]), v);
        }
        __syncthreads();
    }
}

// L2L last step: G[c][i][j] += sum_m H[c][mi][i] e^{-i m phi_j} for the rows (c, i) of all children.
template <typename C>
__global__ void k_l2l_fft_out(int64_t nrows_tot, const C* __restrict__ H, int nth, int Lc, FftPlan fp,
                              const C* __restrict__ tw, int RB, C* __restrict__ G) {
    extern __shared__ unsigned char smem_raw[];
    const int n = fp.n, nm = 2 * Lc + 1;
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + RB * n;
    C* stw = buf1 + RB * n;
    const int64_t r0 = (int64_t)blockIdx.x * RB;
    const int nr = (int)((nrows_tot - r0) < RB ? (nrows_tot - r0) : RB);
    for (int idx = threadIdx.x; idx < nr * n; idx += blockDim.x) buf0[idx] = cmake<C>(0, 0);
    for (int j = threadIdx.x; j < n; j += blockDim.x) stw[j] = tw[j];
    __syncthreads();
    for (int idx = threadIdx.x; idx < nr * nm; idx += blockDim.x) {
        const int row = idx % nr, mi = idx / nr;
        const int64_t r = r0 + row;
        const int64_t c = r / nth;
        const int i = (int)(r - c * nth);
        buf0[row * n + wrap(mi - Lc, n)] = H[(c * nm + mi) * nth + i];
    }
    __syncthreads();
    const C* res = fft_rows(buf0, buf1, nr, fp, stw, false);
    for (int idx = threadIdx.x; idx < nr * n; idx += blockDim.x) {
        C* g = G + r0 * n + idx;
        *g = cadd(*g, res[idx]);
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

// ============================================================== pipeline
template <typename R>
static void far_pipeline(Plan& p, const void* qs_v, void* phis_v) {
    using C = typename Cx<R>::T;
    cudaStream_t s = p.stream;
    const C* qs = (const C*)qs_v;
    C* phis = (C*)phis_v;
    const R k = (R)p.k;
    // ---- upward pass: C2M at every far level's leaves, M2M from the deepest level up
    for (int l = p.nlev; l >= p.top; --l) {
        FarLevel& F = p.far[l];
        TreeLevel& T = p.lev[l];
        if (T.nleaf > 0) {
            StageTimer st(p, MLFMA_STAGE_C2M, l, 1);
            k_c2m<R, C><<<nblk(T.nleaf, 4), 128, 0, s>>>(T.nleaf, p.leaf_box + p.leaf_first[l], T.begin, T.end, T.center, p.pos,
                                                       qs, (const R*)F.dirs, F.K, k, (C*)F.F);
            MLFMA_LAUNCH_CHECK();
        }
        if (l == p.nlev) continue;
        FarLevel& Ch = p.far[l + 1];
        TreeLevel& TC = p.lev[l + 1];
        const int Lc = Ch.L, nm = 2 * Lc + 1;
        StageTimer st(p, MLFMA_STAGE_M2M, l, 3);
        const int64_t rows_c = TC.nbox * (int64_t)Ch.nth;
        const int budget = (int)(44 * 1024 / sizeof(C));
        // A: forward FFT of the children's rows, modes |m| <= Lc
        int RB = tile_rows((int)std::min<int64_t>(rows_c, 1 << 20), budget - Ch.nph, 2 * Ch.nph);
        size_t sm = ((size_t)2 * RB * Ch.nph + Ch.nph) * sizeof(C);
        k_fft_fwd_rows<C, R><<<nblk(rows_c, RB), 128, sm, s>>>(rows_c, (const C*)Ch.F, Ch.nth, Lc, Ch.fft,
                                                                  (const C*)Ch.tw, (R)(1.0 / Ch.nph), RB, (C*)F.X);
        MLFMA_LAUNCH_CHECK();
        // B: theta maps per mode
        sm = (size_t)kMapCB * Ch.nth * sizeof(C);
        k_theta_map<R, C><<<dim3(nblk(TC.nbox, kMapCB), nm), 128, sm, s>>>(TC.nbox, Lc, Ch.nth, F.nth, (const R*)F.At,
                                                                              (const C*)F.X, (C*)F.Y);
        MLFMA_LAUNCH_CHECK();
        // C: z-shift per mode, inverse FFT, xy-shift, sum over children
        int RT = tile_rows(F.nth, budget - F.nph, 3 * F.nph);
        sm = ((size_t)3 * RT * F.nph + F.nph) * sizeof(C);
        k_m2m_fft_out<C><<<dim3((unsigned)T.nbox, nblk(F.nth, RT)), 128, sm, s>>>(T.child_begin, T.child_end, TC.key,
                                                                                  (const C*)F.Y, Lc, F.nth, F.fft,
                                                                                  (const C*)F.tw, (const C*)F.Sz,
                                                                                  (const C*)F.Sxy, RT, (C*)F.F);
        MLFMA_LAUNCH_CHECK();
    }
    // ---- downward pass: M2L, L2L, L2O
    for (int l = p.top; l <= p.nlev; ++l) {
        FarLevel& F = p.far[l];
        TreeLevel& T = p.lev[l];
        TreeLevel& TP = p.lev[l - 1];
        {
            StageTimer st(p, MLFMA_STAGE_M2L, l, 1);
            int tb = (int)std::min<int64_t>(256, ((F.K + 31) / 32) * 32);
            int ny = nblk(F.K, tb);
            k_m2l<R, C><<<dim3((unsigned)TP.nbox, ny), tb, 0, s>>>(TP.child_begin, TP.child_end, TP.coll, T.ijk, p.off343,
                                                                  (const C*)F.F, (const C*)F.T, F.K, (C*)F.G);
            MLFMA_LAUNCH_CHECK();
        }
        if (l > p.top) {
            FarLevel& Pf = p.far[l - 1];
            const int Lc = F.L, nm = 2 * Lc + 1;
            StageTimer st(p, MLFMA_STAGE_L2L, l, 3);
            const int budget = (int)(44 * 1024 / sizeof(C));
            int RT = tile_rows(Pf.nth, budget - Pf.nph, 2 * Pf.nph);
            size_t sm = ((size_t)2 * RT * Pf.nph + Pf.nph) * sizeof(C);
            k_l2l_fft_in<C, R><<<dim3((unsigned)TP.nbox, nblk(Pf.nth, RT)), 128, sm, s>>>(
                TP.child_begin, TP.child_end, T.key, (const C*)Pf.G, Lc, Pf.nth, Pf.fft, (const C*)Pf.tw, (const C*)Pf.Sz,
                (const C*)Pf.Sxy, RT, (R)(1.0 / Pf.nph), (C*)Pf.Y);
            MLFMA_LAUNCH_CHECK();
            sm = (size_t)kMapCB * Pf.nth * sizeof(C);
            k_theta_map<R, C><<<dim3(nblk(T.nbox, kMapCB), nm), 128, sm, s>>>(T.nbox, Lc, Pf.nth, F.nth, (const R*)Pf.Bt,
                                                                                (const C*)Pf.Y, (C*)Pf.X);
            MLFMA_LAUNCH_CHECK();
            const int64_t rows_c = T.nbox * (int64_t)F.nth;
            int RB = tile_rows((int)std::min<int64_t>(rows_c, 1 << 20), budget - F.nph, 2 * F.nph);
            sm = ((size_t)2 * RB * F.nph + F.nph) * sizeof(C);
            k_l2l_fft_out<C><<<nblk(rows_c, RB), 128, sm, s>>>(rows_c, (const C*)Pf.X, F.nth, Lc, F.fft, (const C*)F.tw, RB,
                                                                (C*)F.G);
            MLFMA_LAUNCH_CHECK();
        }
        if (T.nleaf > 0) {
            StageTimer st(p, MLFMA_STAGE_L2O, l, 1);
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
