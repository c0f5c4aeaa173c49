// Per-level sampling grids, translation operators, interpolation matrices and shift
// tables, all computed on the device in FP64 and stored in the apply precision.
//
// Sec. 3.2.3 (translation operators are precomputed per level and offset), Sec. 3.2.2
// and 3.2.4 (global interpolation / anterpolation between the grids of two levels).
// The grid of a level with truncation L is (L+1) Gauss-Legendre nodes in cos(theta)
// (ascending) times nph uniform phi nodes (nph = smallest even 7-smooth number
// >= 2L+2, so that the phi transforms are mixed-radix FFTs), sample p = i nph + j,
// weight w_p = w_i 2 pi / nph.  Translation operator for the box offset X = c_t - c_s:
//   T_X(khat) = sum_{n=0}^{L} i^n (2n+1) h_n(k|X|) P_n(khat . Xhat),
// the diagonal plane-wave form of the Gegenbauer addition theorem.
// Interpolation child (Lc) -> parent (Lp), per Fourier mode m (|m| <= Lc):
//   A_m[i'][i] = sum_{n=|m|}^{Lc} Pbar_n^m(x'_i') Pbar_n^m(x_i) w_i
// (Pbar orthonormal on [-1, 1]); anterpolation uses the weighted transpose
//   B_m[i][i'] = A_m[i'][i] w'_i' / w_i.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "common.cuh"

namespace mlfma {

// smallest even number >= m whose prime factors are all in {2, 3, 5, 7}
int smooth_even(int m) {
    for (;; ++m) {
        int t = m;
        for (int r : {2, 3, 5, 7})
            while (t % r == 0) t /= r;
        if (t == 1 && m % 2 == 0) return m;
    }
}

FftPlan make_fft_plan(int n) {
    FftPlan p;
    p.n = n;
    int m = n;
    for (int r : {7, 5, 3, 4, 2})   // odd radices first: their strided writes are conflict-free
        while (m % r == 0) {
            if (p.ns >= 16) fail(MLFMA_ERR_UNSUPPORTED, "FFT length %d has too many factors", n);
            p.r[p.ns++] = r;
            m /= r;
        }
    if (m != 1) fail(MLFMA_ERR_UNSUPPORTED, "FFT length %d is not 7-smooth", n);
    p.dn = FastDiv::make((unsigned)n);
    int Ns = 1;
    for (int st = 0; st < p.ns; ++st) {
        p.Ns[st] = Ns;
        p.nb[st] = n / p.r[st];
        p.tstep[st] = n / (Ns * p.r[st]);
        p.dNs[st] = FastDiv::make((unsigned)Ns);
        p.dnb[st] = FastDiv::make((unsigned)p.nb[st]);
        Ns *= p.r[st];
    }
    return p;
}

// TMA descriptor of a level's operators T[343][K] (complex as 8-byte elements: K or 2 K per
// row), box of 32 complex samples x kTBoxRows rows; out-of-range samples and rows read as zero
void encode_translation_map(FarLevel& F, size_t csz) {
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Encode encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        MLFMA_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !fn) fail(MLFMA_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
        encode = (Encode)fn;
    }
    const cuuint64_t per = csz / 8;                      // 8-byte elements per complex sample
    const cuuint64_t dims[2] = {(cuuint64_t)F.K * per, 343};
    const cuuint64_t strides[1] = {(cuuint64_t)F.K * csz};
    const cuuint32_t box[2] = {(cuuint32_t)(32 * per), (cuuint32_t)kTBoxRows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(&F.tmT, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, F.T, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) fail(MLFMA_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) for K = %lld", (int)r, (long long)F.K);
}

int truncation_L(double edge, double k, int digits, int margin) {
    double kD = k * std::sqrt(3.0) * edge;
    double d0 = (double)(digits + margin);
    return (int)std::ceil(kD + 1.8 * std::pow(d0, 2.0 / 3.0) * std::pow(kD, 1.0 / 3.0));
}

static void offsets_table(int* off343, int* dxyz /* [316][3] */) {
    int c = 0;
    for (int dz = -3; dz <= 3; ++dz)
        for (int dy = -3; dy <= 3; ++dy)
            for (int dx = -3; dx <= 3; ++dx) {
                int idx = (dx + 3) + 7 * (dy + 3) + 49 * (dz + 3);
                if (std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz))) <= 1) {
                    off343[idx] = -1;
                } else {
                    off343[idx] = c;
                    dxyz[3 * c] = dx; dxyz[3 * c + 1] = dy; dxyz[3 * c + 2] = dz;
                    ++c;
                }
            }
}

// ---------------------------------------------------------------- Gauss-Legendre (Newton on P_n)
__global__ void k_gauss_legendre(int npts, double* __restrict__ x, double* __restrict__ w) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npts) return;
    // ascending nodes: x_i = -cos(pi (i + 3/4) / (n + 1/2)) as the starting guess
    double z = -cos(M_PI * (i + 0.75) / (npts + 0.5));
    double p0 = 1, p1 = z;
    for (int it = 0; it < 100; ++it) {
        p0 = 1.0; p1 = z;
        for (int n = 1; n < npts; ++n) {
            double p2 = ((2 * n + 1) * z * p1 - n * p0) / (n + 1);
            p0 = p1; p1 = p2;
        }
        double dp = npts * (z * p1 - p0) / (z * z - 1.0);
        double dz = p1 / dp;
        z -= dz;
        if (fabs(dz) < 1e-16) break;
    }
    p0 = 1.0; p1 = z;
    for (int n = 1; n < npts; ++n) {
        double p2 = ((2 * n + 1) * z * p1 - n * p0) / (n + 1);
        p0 = p1; p1 = p2;
    }
    double dp = npts * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
}

// khat_p and w_p in the apply precision
template <typename R>
__global__ void k_dirs(const double* __restrict__ x, const double* __restrict__ wgl, int nth, int nph, R* __restrict__ dirs) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= (int64_t)nth * nph) return;
    int i = (int)(p / nph), j = (int)(p % nph);
    double sp, cp;
    sincospi(2.0 * j / nph, &sp, &cp);
    double st = sqrt(1.0 - x[i] * x[i]);
    dirs[4 * p + 0] = (R)(st * cp);
    dirs[4 * p + 1] = (R)(st * sp);
    dirs[4 * p + 2] = (R)x[i];
    dirs[4 * p + 3] = (R)(wgl[i] * 2.0 * M_PI / nph);
}

template <typename C>
__global__ void k_twiddle(int nph, C* __restrict__ tw) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nph) return;
    double s, c;
    sincospi(-2.0 * j / nph, &s, &c);
    tw[j] = cmake<C>(c, s);
}

// ---------------------------------------------------------------- spherical Hankel functions per offset
// h_n(x), n = 0..L, x = k |X_o|: y_n by upward recurrence; j_n upward while n < x
// (stable there), else by Miller's downward recurrence normalised with
// sum_n (2n+1) j_n^2 = 1.
constexpr int kMillerMax = 2048;

__global__ void k_hankel(int noff, int L, double k, double edge, const int* __restrict__ dxyz, double2* __restrict__ hn,
                         double* __restrict__ work) {
    int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= noff) return;
    double X[3] = {dxyz[3 * o] * edge, dxyz[3 * o + 1] * edge, dxyz[3 * o + 2] * edge};
    double x = k * sqrt(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
    double2* h = hn + (size_t)o * (L + 1);
    // y_n
    double sx, cx;
    sincos(x, &sx, &cx);
    double ym1 = -cx / x, y0 = -cx / (x * x) - sx / x;
    h[0].y = ym1;
    if (L >= 1) h[1].y = y0;
    for (int n = 1; n < L; ++n) {
        double y1 = (2 * n + 1) / x * y0 - ym1;
        h[n + 1].y = y1;
        ym1 = y0; y0 = y1;
    }
    // j_n
    if (x > L + 1) {
        double jm1 = sx / x, j0 = sx / (x * x) - cx / x;
        h[0].x = jm1;
        if (L >= 1) h[1].x = j0;
        for (int n = 1; n < L; ++n) {
            double j1 = (2 * n + 1) / x * j0 - jm1;
            h[n + 1].x = j1;
            jm1 = j0; j0 = j1;
        }
    } else {
        double* v = work + (size_t)o * (kMillerMax + 2);
        int ns = (int)fmax((double)L, x) + 40 + (int)(2.0 * sqrt(fmax((double)L, x)));
        if (ns > kMillerMax) ns = kMillerMax;
        v[ns + 1] = 0.0;
        v[ns] = 1.0;
        for (int n = ns; n > 0; --n) {
            v[n - 1] = (2 * n + 1) / x * v[n] - v[n + 1];
            if (fabs(v[n - 1]) > 1e100)
                for (int m = n - 1; m <= ns + 1; ++m) v[m] *= 1e-100;
        }
        double s = 0;
        for (int n = 0; n <= ns + 1; ++n) s += (2.0 * n + 1.0) * v[n] * v[n];
        double inv = 1.0 / sqrt(s);
        for (int n = 0; n <= L; ++n) h[n].x = v[n] * inv;
    }
}

template <typename C>
__global__ void k_translation(int L, int nth, int nph, double edge, const double* __restrict__ x, const int* __restrict__ dxyz,
                              const double2* __restrict__ hn, C* __restrict__ T) {
    int64_t K = (int64_t)nth * nph;
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= K * kNumOffsets) return;
    int o = (int)(idx / K);
    int64_t p = idx % K;
    int i = (int)(p / nph), j = (int)(p % nph);
    double X[3] = {(double)dxyz[3 * o], (double)dxyz[3 * o + 1], (double)dxyz[3 * o + 2]};
    double r = sqrt(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
    double sp, cp;
    sincospi(2.0 * j / nph, &sp, &cp);
    double st = sqrt(1.0 - x[i] * x[i]);
    double t = (st * cp * X[0] + st * sp * X[1] + x[i] * X[2]) / r;
    const double2* h = hn + (size_t)o * (L + 1);
    double re = 0, im = 0;
    double pm1 = 1.0, p0 = t;
    // n = 0: i^0 (1) h_0 P_0
    re += h[0].x; im += h[0].y;
    for (int n = 1; n <= L; ++n) {
        double Pn = (n == 1) ? t : p0;
        if (n >= 2) {
            Pn = ((2 * n - 1) * t * p0 - (n - 1) * pm1) / n;
            pm1 = p0; p0 = Pn;
        }
        double a = (2 * n + 1) * Pn;
        // i^n h_n
        double hr = h[n].x, hi = h[n].y, cr, ci;
        switch (n & 3) {
            case 0: cr = hr; ci = hi; break;
            case 1: cr = -hi; ci = hr; break;
            case 2: cr = -hr; ci = -hi; break;
            default: cr = hi; ci = -hr; break;
        }
        re += a * cr; im += a * ci;
    }
    (void)edge;
    // row of the offset in the 7^3 cube (the 27 near rows stay zero)
    const int row = (dxyz[3 * o] + 3) + 7 * (dxyz[3 * o + 1] + 3) + 49 * (dxyz[3 * o + 2] + 3);
    T[(int64_t)row * K + p] = cmake<C>(re, im);
}

// ---------------------------------------------------------------- sampled translation operators
// Sec. 3.2.3 ("Translation Operators"): operators that would not fit are sampled and
// interpolated.  T_X(khat) = sum_n i^n (2n+1) h_n(k|X|) P_n(cos psi) depends on khat only through
// the angle psi between khat and X, and is an even, 2 pi-periodic cosine polynomial of degree L
// in psi.  One thread per (class c, entry i): T at psi_i = (i - kOpOrder) pi / S into row d2[c]
// (|X/edge|^2 of the class) of the level's table.  Entries with psi_i < 0 or > pi are the
// reflections the interpolation stencil reads next to psi = 0 and pi; cos(psi_i) yields them.
// hn: [ncls][L+1] spherical Hankel functions of the classes' k|X|.
template <typename C>
__global__ void k_op_samples(int L, int S, int ncls, int T1n, const int* __restrict__ d2, const double2* __restrict__ hn,
                             C* __restrict__ T1) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)ncls * T1n) return;
    const int c = (int)(idx / T1n), i = (int)(idx % T1n);
    const double t = cospi((double)(i - kOpOrder) / S);
    const double2* h = hn + (size_t)c * (L + 1);
    double re = h[0].x, im = h[0].y, pm1 = 1.0, p0 = t;
    for (int n = 1; n <= L; ++n) {
        double Pn = t;
        if (n >= 2) {
            Pn = ((2 * n - 1) * t * p0 - (n - 1) * pm1) / n;
            pm1 = p0;
            p0 = Pn;
        }
        const double a = (2 * n + 1) * Pn, hr = h[n].x, hi = h[n].y;
        switch (n & 3) {                            // i^n h_n
            case 0: re += a * hr; im += a * hi; break;
            case 1: re -= a * hi; im += a * hr; break;
            case 2: re -= a * hr; im -= a * hi; break;
            default: re += a * hi; im -= a * hr; break;
        }
    }
    T1[(int64_t)d2[c] * T1n + i] = cmake<C>(re, im);
}

// ---------------------------------------------------------------- interpolation matrices
// Pbar_m^m = sqrt((2m+1)/2 prod_{k<=m} (2k-1)/(2k)) (1-x^2)^{m/2}, then the column recurrence in n.
__device__ double pbar_mm(int m, double x) {
    double c = 0.5 * (2 * m + 1);
    for (int kk = 1; kk <= m; ++kk) c *= (2.0 * kk - 1.0) / (2.0 * kk);
    double s2 = fmax(1.0 - x * x, 0.0);
    return sqrt(c) * pow(s2, 0.5 * m);
}

template <typename R>
__global__ void k_interp(int Lc, const double* __restrict__ xc, const double* __restrict__ wc, int nthp,
                         const double* __restrict__ xp, const double* __restrict__ wp, R* __restrict__ At, R* __restrict__ Bt) {
    const int nthc = Lc + 1;
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t tot = (int64_t)(Lc + 1) * nthc * nthp;
    if (idx >= tot) return;
    int ip = (int)(idx % nthp);
    int i = (int)((idx / nthp) % nthc);
    int m = (int)(idx / ((int64_t)nthp * nthc));
    double a = xc[i], b = xp[ip];
    double pa = pbar_mm(m, a), pb = pbar_mm(m, b);
    double s = pa * pb;
    if (m + 1 <= Lc) {
        double qa = a * sqrt(2.0 * m + 3.0) * pa, qb = b * sqrt(2.0 * m + 3.0) * pb;
        s += qa * qb;
        for (int n = m + 2; n <= Lc; ++n) {
            double an = sqrt((4.0 * n * n - 1.0) / ((double)n * n - (double)m * m));
            double bn = sqrt(((n - 1.0) * (n - 1.0) - (double)m * m) / (4.0 * (n - 1.0) * (n - 1.0) - 1.0));
            double ra = an * (a * qa - bn * pa), rb = an * (b * qb - bn * pb);
            pa = qa; qa = ra; pb = qb; qb = rb;
            s += ra * rb;
        }
    }
    double A = s * wc[i];                       // A_m[i'][i]
    At[((int64_t)m * nthc + i) * nthp + ip] = (R)A;
    Bt[((int64_t)m * nthp + ip) * nthc + i] = (R)(A * wp[ip] / wc[i]);
}

// shift tables of a parent level: Sz[sz][i'] and Sxy[q][p']
template <typename C>
__global__ void k_shifts(int nth, int nph, double k, double edge, const double* __restrict__ x, C* __restrict__ Sz, C* __restrict__ Sxy) {
    int64_t K = (int64_t)nth * nph;
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const double q4 = 0.25 * edge;
    if (idx < 2 * nth) {
        int sz = (int)(idx / nth), i = (int)(idx % nth);
        double dz = (2 * sz - 1) * q4;
        double s, c;
        sincos(-k * x[i] * dz, &s, &c);
        Sz[idx] = cmake<C>(c, s);
    }
    if (idx < 4 * K) {
        int q = (int)(idx / K);
        int64_t p = idx % K;
        int i = (int)(p / nph), j = (int)(p % nph);
        double dx = (2 * (q & 1) - 1) * q4, dy = (2 * ((q >> 1) & 1) - 1) * q4;
        double sp, cp;
        sincospi(2.0 * j / nph, &sp, &cp);
        double st = sqrt(1.0 - x[i] * x[i]);
        double s, c;
        sincos(-k * st * (cp * dx + sp * dy), &s, &c);
        Sxy[idx] = cmake<C>(c, s);
    }
}

// Dense maps of a level pair (tensor-core precisions, fine levels): the forward phi transform
// of the child grid, the theta maps of every mode and the inverse phi transform of the parent
// grid composed into one real matrix each way,
//   Mp[(i,j)][(i',j')] = (1/n_c) sum_{|m| <= Lc} At[|m|][i][i'] cos(2 pi m (j'/n_p - j/n_c))   (M2M, [Kc][Kp])
//   Mq[(i',j')][(i,j)] = (1/n_p) sum_{|m| <= Lc} Bt[|m|][i'][i] cos(2 pi m (j'/n_p - j/n_c))   (L2L, [Kp][Kc])
// the same operators as the FFT path (whose mode m and -m terms are complex conjugates).  The
// phases are reduced with integer residues m j mod n; FP64 sums.
__global__ void k_dense_maps(int Lc, int nthc, int nphc, int nthp, int nphp, const float* __restrict__ At,
                             const float* __restrict__ Bt, float* __restrict__ Mp, float* __restrict__ Mq) {
    const int64_t Kc = (int64_t)nthc * nphc, Kp = (int64_t)nthp * nphp;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= Kc * Kp) return;
    const int64_t kc = idx / Kp, sp = idx - kc * Kp;
    const int i = (int)(kc / nphc), j = (int)(kc % nphc);
    const int ip = (int)(sp / nphp), jp = (int)(sp % nphp);
    double sa = 0, sb = 0;
    for (int m = -Lc; m <= Lc; ++m) {
        const int am = m < 0 ? -m : m;
        int rp = (int)(((int64_t)m * jp) % nphp), rc = (int)(((int64_t)m * j) % nphc);
        if (rp < 0) rp += nphp;
        if (rc < 0) rc += nphc;
        const double c = cospi(2.0 * ((double)rp / nphp - (double)rc / nphc));
        sa += (double)At[((int64_t)am * nthc + i) * nthp + ip] * c;
        sb += (double)Bt[((int64_t)am * nthp + ip) * nthc + i] * c;
    }
    Mp[kc * Kp + sp] = (float)(sa / nphc);
    Mq[sp * Kc + kc] = (float)(sb / nphp);
}

// Parity split of the theta maps (the GEMM form of the unfused level pairs evaluates the
// even and odd parts at half the size each).  One thread per (m, i, i') over the half ranges
// i < ceil(nth_c/2), i' < ceil(nth_p/2): the sums over n of Pbar_n^m(x_i) Pbar_n^m(x'_i') split
// by the parity of n + m, times w_i (M2M map, input i) or w'_i' (L2L map, input i').  A row
// for the middle input node of an odd grid (x = 0: only even terms) is halved, since the GEMM
// forms its input as in[i] + in[n-1-i], twice the middle value; odd entries at a middle node
// are zero.
template <typename R>
__global__ void k_interp_par(int Lc, const double* __restrict__ xc, const double* __restrict__ wc, int nthp,
                             const double* __restrict__ xp, const double* __restrict__ wp, R* __restrict__ AtE,
                             R* __restrict__ AtD, R* __restrict__ BtE, R* __restrict__ BtD) {
    const int nthc = Lc + 1, hc = (nthc + 1) / 2, hp = (nthp + 1) / 2;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)(Lc + 1) * hc * hp) return;
    const int ip = (int)(idx % hp);
    const int i = (int)((idx / hp) % hc);
    const int m = (int)(idx / ((int64_t)hp * hc));
    const double a = xc[i], b = xp[ip];
    double pa = pbar_mm(m, a), pb = pbar_mm(m, b);
    double se = pa * pb, so = 0;                 // n = m: n + m even
    if (m + 1 <= Lc) {
        double qa = a * sqrt(2.0 * m + 3.0) * pa, qb = b * sqrt(2.0 * m + 3.0) * pb;
        so += qa * qb;
        for (int n = m + 2; n <= Lc; ++n) {
            double an = sqrt((4.0 * n * n - 1.0) / ((double)n * n - (double)m * m));
            double bn = sqrt(((n - 1.0) * (n - 1.0) - (double)m * m) / (4.0 * (n - 1.0) * (n - 1.0) - 1.0));
            double ra = an * (a * qa - bn * pa), rb = an * (b * qb - bn * pb);
            pa = qa; qa = ra; pb = qb; qb = rb;
            if (((n + m) & 1) == 0) se += ra * rb;
            else so += ra * rb;
        }
    }
    const bool midc = (nthc & 1) && i == hc - 1, midp = (nthp & 1) && ip == hp - 1;
    const double sd = (midc || midp) ? 0.0 : so;
    AtE[((int64_t)m * hc + i) * hp + ip] = (R)(se * wc[i] * (midc ? 0.5 : 1.0));
    AtD[((int64_t)m * hc + i) * hp + ip] = (R)(sd * wc[i]);
    BtE[((int64_t)m * hp + ip) * hc + i] = (R)(se * wp[ip] * (midp ? 0.5 : 1.0));
    BtD[((int64_t)m * hp + ip) * hc + i] = (R)(sd * wp[ip]);
}

// the children's shifts by octant o: So[o][i'][j'] = Sz[o >> 2][i'] Sxy[o & 3][i'][j']
template <typename C>
__global__ void k_soct(int nth, int nph, const C* __restrict__ Sz, const C* __restrict__ Sxy, C* __restrict__ So) {
    const int64_t K = (int64_t)nth * nph;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= 8 * K) return;
    const int o = (int)(idx / K);
    const int64_t sp = idx - o * K;
    So[idx] = cmul(Sz[(o >> 2) * nth + sp / nph], Sxy[(o & 3) * K + sp]);
}

static inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

template <typename R>
static void build_far_levels_t(Plan& p) {
    using C = typename Cx<R>::T;
    cudaStream_t s = p.stream;
    int off343[343], dxyz[3 * kNumOffsets];
    offsets_table(off343, dxyz);
    p.off343 = p.mem.make<int>(343);
    MLFMA_CUDA(cudaMemcpyAsync(p.off343, off343, sizeof(off343), cudaMemcpyHostToDevice, s));
    int* d_dxyz = p.mem.make<int>(3 * kNumOffsets);
    MLFMA_CUDA(cudaMemcpyAsync(d_dxyz, dxyz, sizeof(dxyz), cudaMemcpyHostToDevice, s));
    // sampled operators: one representative offset per squared length |X/edge|^2 that far
    // offsets take (every d2 >= 4 that is a sum of three squares of at most 3)
    int rep[3 * kOpRows], cls_d2[kOpRows], ncls = 0;
    for (int d2 = 4; d2 < kOpRows; ++d2)
        for (int o = 0; o < kNumOffsets; ++o) {
            const int* d = dxyz + 3 * o;
            if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] != d2) continue;
            rep[3 * ncls] = d[0]; rep[3 * ncls + 1] = d[1]; rep[3 * ncls + 2] = d[2];
            cls_d2[ncls++] = d2;
            break;
        }
    int* d_rep = nullptr;
    int* d_cls = nullptr;
    if (p.op_s > 0) {
        d_rep = p.mem.make<int>(3 * kOpRows);
        d_cls = p.mem.make<int>(kOpRows);
        MLFMA_CUDA(cudaMemcpyAsync(d_rep, rep, sizeof(rep), cudaMemcpyHostToDevice, s));
        MLFMA_CUDA(cudaMemcpyAsync(d_cls, cls_d2, sizeof(cls_d2), cudaMemcpyHostToDevice, s));
    }

    // top: highest level with a non-empty V list
    p.top = 0;
    for (int l = 2; l <= p.nlev; ++l)
        if (p.lev[l].nv > 0) { p.top = l; break; }
    if (!p.top) return;
    int Lmax = 0;
    for (int l = p.top; l <= p.nlev; ++l) {
        FarLevel& F = p.far[l];
        F.L = truncation_L(p.lev[l].edge, p.k, p.digits, p.margin);
        F.nth = F.L + 1;
        F.nph = smooth_even(2 * F.L + 2);
        F.fft = make_fft_plan(F.nph);
        F.K = (int64_t)F.nth * F.nph;
        Lmax = std::max(Lmax, F.L);
    }
    double2* hn = p.mem.make<double2>((size_t)kNumOffsets * (Lmax + 1));
    double* work = p.mem.make<double>((size_t)kNumOffsets * (kMillerMax + 2));
    for (int l = p.top; l <= p.nlev; ++l) {
        FarLevel& F = p.far[l];
        F.x = p.mem.make<double>(F.nth);
        F.wgl = p.mem.make<double>(F.nth);
        k_gauss_legendre<<<nblk(F.nth, 64), 64, 0, s>>>(F.nth, F.x, F.wgl);
        MLFMA_LAUNCH_CHECK();
        F.dirs = p.mem.make<R>(4 * F.K);
        k_dirs<R><<<nblk(F.K, 256), 256, 0, s>>>(F.x, F.wgl, F.nth, F.nph, (R*)F.dirs);
        MLFMA_LAUNCH_CHECK();
        F.tw = p.mem.make<C>(F.nph);
        k_twiddle<C><<<nblk(F.nph, 256), 256, 0, s>>>(F.nph, (C*)F.tw);
        MLFMA_LAUNCH_CHECK();
        if (p.op_s > 0 && p.k * p.lev[l].edge >= 2.0 * M_PI * (1.0 - 1e-9)) {
            // boxes of a wavelength or more: sampled operators, interpolated in M2L
            const int S = p.op_s * F.L;
            F.T1n = S + 2 * kOpOrder + 1;
            F.T1inv_h = S / M_PI;
            k_hankel<<<nblk(ncls, 32), 32, 0, s>>>(ncls, F.L, p.k, p.lev[l].edge, d_rep, hn, work);
            MLFMA_LAUNCH_CHECK();
            F.T1 = p.mem.make<C>((size_t)kOpRows * F.T1n);
            MLFMA_CUDA(cudaMemsetAsync(F.T1, 0, (size_t)kOpRows * F.T1n * sizeof(C), s));
            k_op_samples<C><<<nblk((int64_t)ncls * F.T1n, 128), 128, 0, s>>>(F.L, S, ncls, F.T1n, d_cls, hn, (C*)F.T1);
            MLFMA_LAUNCH_CHECK();
            memset(&F.tmT, 0, sizeof(F.tmT));
        } else {
            k_hankel<<<nblk(kNumOffsets, 32), 32, 0, s>>>(kNumOffsets, F.L, p.k, p.lev[l].edge, d_dxyz, hn, work);
            MLFMA_LAUNCH_CHECK();
            F.T = p.mem.make<C>((size_t)343 * F.K);
            MLFMA_CUDA(cudaMemsetAsync(F.T, 0, (size_t)343 * F.K * sizeof(C), s));
            k_translation<C><<<nblk(F.K * kNumOffsets, 128), 128, 0, s>>>(F.L, F.nth, F.nph, p.lev[l].edge, F.x, d_dxyz,
                                                                          hn, (C*)F.T);
            MLFMA_LAUNCH_CHECK();
            encode_translation_map(F, sizeof(C));
        }
        F.F = p.mem.make<C>((size_t)p.lev[l].nbox * F.K);
        F.G = p.mem.make<C>((size_t)p.lev[l].nbox * F.K);
    }
    for (int l = p.top; l < p.nlev; ++l) {
        FarLevel& P = p.far[l];
        FarLevel& Ch = p.far[l + 1];
        int64_t nA = (int64_t)(Ch.L + 1) * Ch.nth * P.nth;
        P.At = p.mem.make<R>(nA);
        P.Bt = p.mem.make<R>(nA);
        k_interp<R><<<nblk(nA, 128), 128, 0, s>>>(Ch.L, Ch.x, Ch.wgl, P.nth, P.x, P.wgl, (R*)P.At, (R*)P.Bt);
        MLFMA_LAUNCH_CHECK();
        const int64_t nH = (int64_t)(Ch.L + 1) * ((Ch.nth + 1) / 2) * ((P.nth + 1) / 2);
        P.AtE = p.mem.make<R>(nH);
        P.AtD = p.mem.make<R>(nH);
        P.BtE = p.mem.make<R>(nH);
        P.BtD = p.mem.make<R>(nH);
        k_interp_par<R><<<nblk(nH, 128), 128, 0, s>>>(Ch.L, Ch.x, Ch.wgl, P.nth, P.x, P.wgl, (R*)P.AtE, (R*)P.AtD,
                                                       (R*)P.BtE, (R*)P.BtD);
        MLFMA_LAUNCH_CHECK();
        if (p.prec == MLFMA_PREC_FP32_TF32X3 || p.prec == MLFMA_PREC_FP32_BF16X3) {
            // the maps split once into the tensor-core operand blocks (At: nth_c -> nth_p, Bt: nth_p -> nth_c)
            P.AtTc = p.mem.get(theta_tc_map_bytes(p, Ch.L + 1, Ch.nth, P.nth));
            P.BtTc = p.mem.get(theta_tc_map_bytes(p, Ch.L + 1, P.nth, Ch.nth));
            presplit_theta_tc(p, Ch.L + 1, Ch.nth, P.nth, (const float*)P.At, P.AtTc, s);
            presplit_theta_tc(p, Ch.L + 1, P.nth, Ch.nth, (const float*)P.Bt, P.BtTc, s);
        }
        P.Sz = p.mem.make<C>(2 * P.nth);
        P.Sxy = p.mem.make<C>(4 * P.K);
        k_shifts<C><<<nblk(4 * P.K, 256), 256, 0, s>>>(P.nth, P.nph, p.k, p.lev[l].edge, P.x, (C*)P.Sz, (C*)P.Sxy);
        MLFMA_LAUNCH_CHECK();
        if ((p.prec == MLFMA_PREC_FP32_TF32X3 || p.prec == MLFMA_PREC_FP32_BF16X3) && Ch.K <= p.dense_kc &&
            dense_tc_fits(p, (int)Ch.K, (int)P.K)) {
            // fine pair: the whole interpolation and anterpolation as dense tensor-core maps
            P.dense = 1;
            const int64_t nKK = Ch.K * P.K;
            float* Mp = p.mem.make<float>(nKK);
            float* Mq = p.mem.make<float>(nKK);
            k_dense_maps<<<nblk(nKK, 128), 128, 0, s>>>(Ch.L, Ch.nth, Ch.nph, P.nth, P.nph, (const float*)P.At,
                                                          (const float*)P.Bt, Mp, Mq);
            MLFMA_LAUNCH_CHECK();
            P.DmTc = p.mem.get(dense_tc_map_bytes(p, true, (int)Ch.K, (int)P.K));
            P.DlTc = p.mem.get(dense_tc_map_bytes(p, false, (int)P.K, (int)Ch.K));
            presplit_dense_tc(p, true, (int)Ch.K, (int)P.K, Mp, P.DmTc, s);
            presplit_dense_tc(p, false, (int)P.K, (int)Ch.K, Mq, P.DlTc, s);
            P.Soct = p.mem.make<C>(8 * P.K);
            k_soct<C><<<nblk(8 * P.K, 256), 256, 0, s>>>(P.nth, P.nph, (const C*)P.Sz, (const C*)P.Sxy, (C*)P.Soct);
            MLFMA_LAUNCH_CHECK();
            MLFMA_CUDA(cudaStreamSynchronize(s));      // the unsplit maps are temporaries
            p.mem.drop(Mq);
            p.mem.drop(Mp);
        }
    }
    // spectral scratch shared by all level pairs: X [nbox_c][2Lc+1][nth_c], Y [nbox_c][2Lc+1][nth_p]
    size_t xs = 0, ys = 0;
    for (int l = p.top; l < p.nlev; ++l) {
        const FarLevel& P = p.far[l];
        const FarLevel& Ch = p.far[l + 1];
        size_t nb = (size_t)p.lev[l + 1].nbox;
        xs = std::max(xs, nb * (2 * Ch.L + 1) * Ch.nth);
        ys = std::max(ys, nb * (2 * Ch.L + 1) * P.nth);
    }
    if (xs) {
        void* X = p.mem.make<C>(xs);
        void* Y = p.mem.make<C>(ys);
        for (int l = p.top; l < p.nlev; ++l) { p.far[l].X = X; p.far[l].Y = Y; }
    }
    MLFMA_CUDA(cudaStreamSynchronize(s));
}

void build_far_levels(Plan& p) {
    if (p.prec == MLFMA_PREC_FP64) build_far_levels_t<double>(p);
    else build_far_levels_t<float>(p);
}

}  // namespace mlfma
