/*
 * FP64 direct evaluation of the Helmholtz sum: the exact result the MLFMA approximates.
 *
 * TEST INFRASTRUCTURE (CPU oracle).  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this library; the product path never does.
 *
 * Definition (Sec. 2, Eq. (1) with the kernel read as e^{+ikR}/R, no 1/(4 pi)):
 *   phi_i     = sum_{j != i, R_ij > 0} q_j e^{ik R_ij} / R_ij
 *   grad phi_i = sum_{j != i, R_ij > 0} q_j e^{ik R_ij} (ik R_ij - 1) / R_ij^3 (r_i - r_j)
 * Coincident points (R = 0) contribute nothing.  Each target's sum is
 * accumulated with Neumaier's compensated summation, one target per thread.
 * Complex values are interleaved (re, im) doubles.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { double s, c; } neumaier;

static inline void nadd(neumaier* a, double v) {
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* phi_out[t] = phi at point targets[t]; pts [n][3], q [nrhs][n] complex, phi_out [nrhs][nt] complex. */
void oracle_direct(const double* pts, const double* q, int64_t n, int nrhs, double k,
                   const int64_t* targets, int64_t nt, double* phi_out, int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int64_t t = 0; t < nt; ++t) {
        const int64_t i = targets[t];
        const double xi = pts[3 * i], yi = pts[3 * i + 1], zi = pts[3 * i + 2];
        for (int r = 0; r < nrhs; ++r) {
            const double* qr = q + (size_t)2 * (size_t)n * (size_t)r;
            neumaier re = {0, 0}, im = {0, 0};
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                double dx = xi - pts[3 * j], dy = yi - pts[3 * j + 1], dz = zi - pts[3 * j + 2];
                double R = sqrt(dx * dx + dy * dy + dz * dz);
                if (R == 0.0) continue;
                double c = cos(k * R) / R, s = sin(k * R) / R;
                double qre = qr[2 * j], qim = qr[2 * j + 1];
                nadd(&re, qre * c - qim * s);
                nadd(&im, qre * s + qim * c);
            }
            phi_out[2 * ((size_t)r * nt + t)] = re.s + re.c;
            phi_out[2 * ((size_t)r * nt + t) + 1] = im.s + im.c;
        }
    }
}

/* grad_out [nrhs][nt][3] complex: gradient of phi with respect to the target position. */
void oracle_direct_grad(const double* pts, const double* q, int64_t n, int nrhs, double k,
                        const int64_t* targets, int64_t nt, double* grad_out, int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int64_t t = 0; t < nt; ++t) {
        const int64_t i = targets[t];
        const double xi = pts[3 * i], yi = pts[3 * i + 1], zi = pts[3 * i + 2];
        for (int r = 0; r < nrhs; ++r) {
            const double* qr = q + (size_t)2 * (size_t)n * (size_t)r;
            neumaier acc[6] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}};
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                double d[3] = {xi - pts[3 * j], yi - pts[3 * j + 1], zi - pts[3 * j + 2]};
                double R = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                if (R == 0.0) continue;
                /* e^{ikR} (ikR - 1) / R^3 = (cos + i sin)(-1 + i kR) / R^3 */
                double c = cos(k * R), s = sin(k * R), R3 = R * R * R;
                double gre = (-c - s * k * R) / R3;
                double gim = (c * k * R - s) / R3;
                double qre = qr[2 * j], qim = qr[2 * j + 1];
                double pre = qre * gre - qim * gim, pim = qre * gim + qim * gre;
                for (int a = 0; a < 3; ++a) {
                    nadd(&acc[2 * a], pre * d[a]);
                    nadd(&acc[2 * a + 1], pim * d[a]);
                }
            }
            for (int a = 0; a < 3; ++a) {
                size_t o = 2 * (((size_t)r * nt + t) * 3 + a);
                grad_out[o] = acc[2 * a].s + acc[2 * a].c;
                grad_out[o + 1] = acc[2 * a + 1].s + acc[2 * a + 1].c;
            }
        }
    }
}
