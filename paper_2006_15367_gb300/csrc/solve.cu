// Restarted GMRES around the matvec.  Sec. 1 places the potential evaluation inside an
// iterative integral-equation solver, where it is the most expensive kernel; this file is
// that outer loop: (sigma I + A) x = b for one right-hand side, A the Helmholtz potential
// matrix the plan applies and sigma a complex diagonal term (a Nystrom self term or a
// regularisation; the plain potential matrix has no diagonal).  The Krylov method is
// GMRES(m) (Saad and Schultz, SIAM J. Sci. Stat. Comput. 7, 1986) with classical
// Gram-Schmidt applied twice per step (CGS2, Giraud et al., Numer. Math. 101, 2005), so
// each orthogonalisation pass is one multi-dot kernel and one update kernel over the
// device-resident basis.  The (m+1) x m Hessenberg matrix, its Givens rotations and the
// triangular solve for the update live on the host (m <= 256 numbers per column).
#include "common.cuh"

#include <cmath>
#include <complex>
#include <vector>

namespace mlfma {

using cplx = std::complex<double>;

constexpr int kDotThreads = 256;

// part[j][blockIdx.x] = sum over this block's elements p of conj(V_j[p]) w[p], j = blockIdx.y.
// Each thread accumulates its strided elements in the plan's real type; the block combines
// the threads in double in a fixed tree order, so the result does not depend on timing.
template <typename C>
__global__ void __launch_bounds__(kDotThreads) k_dots(const C* __restrict__ V, int64_t ldv, const C* __restrict__ w,
                                                     int64_t n, double2* __restrict__ part) {
    using R = decltype(C().x);
    const C* v = V + blockIdx.y * ldv;
    R sr = 0, si = 0;
    for (int64_t p = blockIdx.x * (int64_t)kDotThreads + threadIdx.x; p < n; p += (int64_t)gridDim.x * kDotThreads) {
        const C a = v[p], b = w[p];
        sr += a.x * b.x + a.y * b.y;
        si += a.x * b.y - a.y * b.x;
    }
    __shared__ double2 red[kDotThreads];
    red[threadIdx.x] = make_double2((double)sr, (double)si);
    __syncthreads();
    for (int s = kDotThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            red[threadIdx.x].x += red[threadIdx.x + s].x;
            red[threadIdx.x].y += red[threadIdx.x + s].y;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = red[0];
}

// out[j] = sum over b of part[j][b] in a fixed order (one block per j)
__global__ void __launch_bounds__(kDotThreads) k_dots_reduce(const double2* __restrict__ part, int nblk,
                                                            double2* __restrict__ out) {
    const double2* pj = part + (int64_t)blockIdx.x * nblk;
    double sr = 0, si = 0;
    for (int b = threadIdx.x; b < nblk; b += kDotThreads) {
        sr += pj[b].x;
        si += pj[b].y;
    }
    __shared__ double2 red[kDotThreads];
    red[threadIdx.x] = make_double2(sr, si);
    __syncthreads();
    for (int s = kDotThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            red[threadIdx.x].x += red[threadIdx.x + s].x;
            red[threadIdx.x].y += red[threadIdx.x + s].y;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// w[p] += sign sum_{j < nv} h[j] V_j[p]  (h complex double on the device, nv <= 257)
template <typename C>
__global__ void k_combine(C* __restrict__ w, const C* __restrict__ V, int64_t ldv, int nv, const double2* __restrict__ h,
                          double sign, int64_t n) {
    using R = decltype(C().x);
    __shared__ C hs[257];
    for (int j = threadIdx.x; j < nv; j += blockDim.x) hs[j] = cmake<C>((R)(sign * h[j].x), (R)(sign * h[j].y));
    __syncthreads();
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        C acc = w[p];
        for (int j = 0; j < nv; ++j) cfma(acc, hs[j], V[j * ldv + p]);
        w[p] = acc;
    }
}

// out[p] = y[p] + sigma x[p]  (the diagonal term added to the plan's A x)
template <typename C>
__global__ void k_add_diag(C* __restrict__ out, const C* __restrict__ y, const C* __restrict__ x, double sr, double si,
                           int64_t n) {
    using R = decltype(C().x);
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    C a = y[p];
    cfma(a, cmake<C>((R)sr, (R)si), x[p]);
    out[p] = a;
}

// r[p] = b[p] - y[p]  (the residual, y = sigma x + A x)
template <typename C>
__global__ void k_residual(C* __restrict__ r, const C* __restrict__ b, const C* __restrict__ y, int64_t n) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    r[p] = cmake<C>(b[p].x - y[p].x, b[p].y - y[p].y);
}

// v[p] = w[p] / sqrt(nrm2.x), zero when the norm is zero (breakdown: the host stops there)
template <typename C>
__global__ void k_normalize(C* __restrict__ v, const C* __restrict__ w, const double2* __restrict__ nrm2, int64_t n) {
    using R = decltype(C().x);
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double q = nrm2->x;
    const R s = q > 0 ? (R)(1.0 / sqrt(q)) : (R)0;
    v[p] = cmake<C>(w[p].x * s, w[p].y * s);
}

namespace {

template <typename C>
struct Gmres {
    Plan& P;
    int64_t n;
    double sr, si;
    int nblk;
    C* V = nullptr;          // [m+1][n] basis
    C* w = nullptr;          // [n]
    double2* part = nullptr; // [m+1][nblk]
    double2* dh = nullptr;   // [3][m+2]: pass-1 and pass-2 coefficients, squared norm
    double2* dy = nullptr;   // [m] update coefficients
    int m;

    // partial-sum blocks of a dot product: two per SM of a 152-SM GB300, fewer for short vectors
    static int blocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(304, (n + 255) / 256)); }

    // h[0..nv-1] = V_j^H w on the device
    void dots(const C* basis, int nv, const C* vec, double2* h) {
        k_dots<C><<<dim3(nblk, nv), kDotThreads, 0, P.stream>>>(basis, n, vec, n, part);
        MLFMA_LAUNCH_CHECK();
        k_dots_reduce<<<nv, kDotThreads, 0, P.stream>>>(part, nblk, h);
        MLFMA_LAUNCH_CHECK();
    }
    void combine(C* dst, int nv, const double2* h, double sign) {
        k_combine<C><<<nblk, 256, 0, P.stream>>>(dst, V, n, nv, h, sign, n);
        MLFMA_LAUNCH_CHECK();
    }
    // dst = sigma v + A v
    void matvec(const C* v, C* dst) {
        apply_device(P, v);
        k_add_diag<C><<<(unsigned)((n + 255) / 256), 256, 0, P.stream>>>(dst, (const C*)P.phiout, v, sr, si, n);
        MLFMA_LAUNCH_CHECK();
    }
    // ||v||, its square left on the device at dh[2 (m + 2)]
    double norm(const C* v) {
        dots(v, 1, v, dh + 2 * (m + 2));
        double2 h;
        MLFMA_CUDA(cudaMemcpyAsync(&h, dh + 2 * (m + 2), sizeof(h), cudaMemcpyDeviceToHost, P.stream));
        MLFMA_CUDA(cudaStreamSynchronize(P.stream));
        return std::sqrt(std::max(h.x, 0.0));
    }
};

}  // namespace

template <typename C>
static void gmres_impl(Plan& P, const C* b, C* x, double sr, double si, double tol, int m, int max_iter,
                       mlfma_solve_info* info) {
    Gmres<C> G{P, P.ntot, sr, si};
    G.m = m;
    G.nblk = Gmres<C>::blocks(G.n);
    const int64_t n = G.n;
    const unsigned eb = (unsigned)((n + 255) / 256);
    G.V = (C*)P.mem.get((size_t)(m + 1) * n * sizeof(C));
    G.w = (C*)P.mem.get((size_t)n * sizeof(C));
    G.part = (double2*)P.mem.get((size_t)(m + 1) * G.nblk * sizeof(double2));
    G.dh = (double2*)P.mem.get((size_t)3 * (m + 2) * sizeof(double2));
    G.dy = (double2*)P.mem.get((size_t)m * sizeof(double2));
    auto release = [&] {
        cudaStreamSynchronize(P.stream);
        P.mem.drop(G.V);
        P.mem.drop(G.w);
        P.mem.drop(G.part);
        P.mem.drop(G.dh);
        P.mem.drop(G.dy);
    };
    try {
        info->iterations = info->restarts = info->matvecs = info->converged = 0;
        info->rel_residual = 0;
        const double bnorm = G.norm(b);
        if (bnorm == 0) {
            MLFMA_CUDA(cudaMemsetAsync(x, 0, (size_t)n * sizeof(C), P.stream));
            info->converged = 1;
            release();
            return;
        }
        std::vector<cplx> H((size_t)(m + 1) * m), g(m + 1), sn(m), y(m);
        std::vector<double> cs(m);
        std::vector<double2> hh(2 * (m + 2) + 1);
        auto Hat = [&](int r, int c) -> cplx& { return H[(size_t)r * m + c]; };
        for (;;) {
            // true residual r = b - (sigma I + A) x into V_0
            G.matvec(x, G.w);
            ++info->matvecs;
            k_residual<C><<<eb, 256, 0, P.stream>>>(G.V, b, G.w, n);
            MLFMA_LAUNCH_CHECK();
            const double beta = G.norm(G.V);
            info->rel_residual = beta / bnorm;
            if (beta <= tol * bnorm) {
                info->converged = 1;
                break;
            }
            if (info->iterations >= max_iter) break;
            if (info->iterations > 0) ++info->restarts;
            k_normalize<C><<<eb, 256, 0, P.stream>>>(G.V, G.V, G.dh + 2 * (m + 2), n);
            MLFMA_LAUNCH_CHECK();
            std::fill(g.begin(), g.end(), cplx(0));
            g[0] = beta;
            int k = 0;                                  // columns of this cycle
            for (int i = 0; i < m && info->iterations < max_iter; ++i) {
                C* vi = G.V + (int64_t)i * n;
                G.matvec(vi, G.w);
                ++info->matvecs;
                // two classical Gram-Schmidt passes, then the norm and the next basis vector
                G.dots(G.V, i + 1, G.w, G.dh);
                G.combine(G.w, i + 1, G.dh, -1.0);
                G.dots(G.V, i + 1, G.w, G.dh + (m + 2));
                G.combine(G.w, i + 1, G.dh + (m + 2), -1.0);
                G.dots(G.w, 1, G.w, G.dh + 2 * (m + 2));
                k_normalize<C><<<eb, 256, 0, P.stream>>>(vi + n, G.w, G.dh + 2 * (m + 2), n);
                MLFMA_LAUNCH_CHECK();
                MLFMA_CUDA(cudaMemcpyAsync(hh.data(), G.dh, (size_t)(2 * (m + 2) + 1) * sizeof(double2),
                                           cudaMemcpyDeviceToHost, P.stream));
                MLFMA_CUDA(cudaStreamSynchronize(P.stream));
                for (int j = 0; j <= i; ++j) Hat(j, i) = cplx(hh[j].x + hh[m + 2 + j].x, hh[j].y + hh[m + 2 + j].y);
                const double hn = std::sqrt(std::max(hh[2 * (m + 2)].x, 0.0));
                Hat(i + 1, i) = hn;
                // earlier rotations, then the one that zeroes H[i+1][i]
                for (int j = 0; j < i; ++j) {
                    const cplx a = Hat(j, i), c = Hat(j + 1, i);
                    Hat(j, i) = cs[j] * a + sn[j] * c;
                    Hat(j + 1, i) = -std::conj(sn[j]) * a + cs[j] * c;
                }
                const cplx a = Hat(i, i);
                const double r = std::hypot(std::abs(a), hn);
                if (r == 0) {
                    cs[i] = 1;
                    sn[i] = 0;
                } else if (std::abs(a) == 0) {
                    cs[i] = 0;
                    sn[i] = 1;
                } else {
                    cs[i] = std::abs(a) / r;
                    sn[i] = (a / std::abs(a)) * hn / r;
                }
                Hat(i, i) = cs[i] * a + sn[i] * hn;
                Hat(i + 1, i) = 0;
                g[i + 1] = -std::conj(sn[i]) * g[i];
                g[i] = cs[i] * g[i];
                ++info->iterations;
                k = i + 1;
                if (std::abs(g[i + 1]) <= tol * bnorm || hn == 0) break;
            }
            // x += V y with R y = g (R the rotated Hessenberg, upper triangular k x k)
            for (int i = k - 1; i >= 0; --i) {
                cplx s = g[i];
                for (int j = i + 1; j < k; ++j) s -= Hat(i, j) * y[j];
                y[i] = Hat(i, i) != cplx(0) ? s / Hat(i, i) : cplx(0);
            }
            std::vector<double2> yd(k);
            for (int i = 0; i < k; ++i) yd[i] = make_double2(y[i].real(), y[i].imag());
            MLFMA_CUDA(cudaMemcpyAsync(G.dy, yd.data(), (size_t)k * sizeof(double2), cudaMemcpyHostToDevice, P.stream));
            G.combine(x, k, G.dy, 1.0);
            MLFMA_CUDA(cudaStreamSynchronize(P.stream));   // yd leaves scope
        }
    } catch (...) {
        release();
        throw;
    }
    release();
}

void gmres_solve(Plan& P, const void* b, void* x, double sr, double si, double tol, int restart, int max_iter,
                 mlfma_solve_info* info) {
    if (P.prec == MLFMA_PREC_FP64)
        gmres_impl<double2>(P, (const double2*)b, (double2*)x, sr, si, tol, restart, max_iter, info);
    else
        gmres_impl<float2>(P, (const float2*)b, (float2*)x, sr, si, tol, restart, max_iter, info);
}

}  // namespace mlfma
