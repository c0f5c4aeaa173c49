/*
 * mlfma.h -- C ABI of the GB300 (sm_103a) MLFMA matvec library.
 *
 * The library evaluates, for points r_1..r_n and complex charges q,
 *
 *     phi_i = sum_{j != i, |r_i - r_j| > 0}  q_j e^{ik|r_i - r_j|} / |r_i - r_j|
 *
 * (the Helmholtz potential of Sec. 2, Eq. (1); read here with the kernel
 * e^{+ikR}/R and without the 1/(4 pi) factor -- the paper's e^{-jkR}/(4 pi R) is its
 * complex conjugate over 4 pi) with the multilevel fast multipole algorithm: an
 * octree with Morton-Z keys (Sec. 3.1), near-field direct sums at the leaves and
 * the five far-field stages C2M, M2M, M2L, L2L, L2O (Sec. 2, Sec. 3.2.1-3.2.5),
 * with global interpolation/anterpolation between levels and diagonal
 * translation over the far-field (V) lists (Alg. 1, Alg. 2).
 *
 * Conventions shared by every entry point:
 *   - Complex numbers are interleaved (re, im): complex128 for MLFMA_PREC_FP64,
 *     complex64 for every other precision.
 *   - Vectors with several right-hand sides are [nrhs][n], contiguous, in the
 *     caller's point order (the plan permutes internally).
 *   - Pointers may address device memory or host memory (pageable or pinned);
 *     the library detects which.  Device pointers: the call only enqueues work
 *     on the plan stream and returns.  Host pointers: the call stages the data
 *     through plan-owned device buffers and synchronises the plan stream before
 *     returning, so the output is ready.
 *   - The caller owns every buffer it passes; the plan copies the points at
 *     creation and never keeps a caller pointer.
 *   - Errors are returned as mlfma_status; nothing aborts or traps.  A
 *     thread-local message is available from mlfma_last_error().
 *   - Every device wait of a kernel (a copy or a tensor-core MMA to complete) is
 *     bounded; a kernel whose wait runs out raises the plan's error flag and returns.
 *     Calls that synchronise the plan stream (applies with host pointers,
 *     mlfma_apply_vjp, mlfma_solve_gmres, mlfma_plan_info, mlfma_plan_export,
 *     mlfma_plan_timings) report a raised flag as MLFMA_ERR_TIMEOUT once and clear it;
 *     an asynchronous apply's timeout is reported by the next such call.
 *   - A plan is not thread-safe: calls on one plan must not overlap.
 */
#ifndef MLFMA_H
#define MLFMA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mlfma_plan mlfma_plan;   /* opaque; owns all device state of one tree */

typedef enum {
    MLFMA_OK = 0,
    MLFMA_ERR_INVALID_ARG = 1,    /* bad size, null pointer, non-finite input, k <= 0 ... */
    MLFMA_ERR_OUT_OF_MEMORY = 2,  /* a device allocation failed; nothing leaked */
    MLFMA_ERR_CUDA = 3,           /* a CUDA runtime call failed (message has the CUDA error) */
    MLFMA_ERR_TIMEOUT = 4,        /* a bounded device wait ran out */
    MLFMA_ERR_UNSUPPORTED = 5     /* valid request outside what this library implements */
} mlfma_status;

typedef enum {
    MLFMA_PREC_FP64 = 0,          /* complex128 data, FP64 arithmetic on every stage */
    MLFMA_PREC_FP32 = 1,          /* complex64 data, FP32 arithmetic; operators built in FP64 */
    MLFMA_PREC_FP32_BF16X3 = 2,   /* as FP32_TF32X3 with BF16 operand parts (hi = x rounded to BF16,
                                     lo = x - hi rounded to BF16; kind::f16 MMAs at twice the TF32 rate):
                                     products good to about 2^-16 relative, enough for 4 digits */
    MLFMA_PREC_FP32_TF32X3 = 3    /* as FP32, but the interpolation (Sec. 3.2.2) and anterpolation
                                     (Sec. 3.2.4) run on the tensor cores as split-TF32 GEMMs (x = hi + lo,
                                     products hi*hi + hi*lo + lo*hi accumulated in FP32): the theta maps
                                     between the phi transforms of the level pairs too large to fuse, or
                                     whole dense maps on the fine pairs (mlfma_options.dense_samples).
                                     FP32-level accuracy */
} mlfma_precision;

/* Options of mlfma_plan_create.  Initialise with mlfma_options_init(). */
typedef struct mlfma_options {
    size_t struct_size;           /* sizeof(mlfma_options), for forward compatibility */
    mlfma_precision precision;    /* default MLFMA_PREC_FP32 */
    double leaf_edge;             /* leaf box edge; <= 0 selects the default: a quarter
                                     wavelength (pi/(2k)) for digits <= 4, half a
                                     wavelength (pi/k) for digits >= 5 */
    int max_depth;                /* deepest tree level, root = 1; default 12 */
    int digit_margin;             /* d0 = digits + digit_margin in the truncation rule; default -1 =
                                     automatic: 1 for FP64 plans, 0 for FP32 plans (in FP32 the roundoff
                                     amplified by |T| at quarter-wavelength boxes grows with L and
                                     dominates the error) */
    void* stream;                 /* cudaStream_t for all work; NULL = the legacy default stream */
    /* Optional device allocator (e.g. a framework's caching allocator).  NULL = cudaMalloc/cudaFree.
       It must return 256-byte aligned device memory (the kernels stage operators by TMA and move
       samples in 16-byte vectors); a misaligned block fails the call with MLFMA_ERR_INVALID_ARG. */
    void* (*alloc)(size_t bytes, void* stream, void* ctx);
    void (*free)(void* ptr, void* stream, void* ctx);
    void* alloc_ctx;
    int disable_graphs;           /* 0 (default): the apply sweep is captured once per (nrhs, kind) as a
                                     CUDA graph and replayed; 1: launch the kernels directly every time */
    int autotune;                 /* 0 (default): the interpolation kernels use the shared-memory tile
                                     budgets 20 / 32 / 40 KB (row tiles, per-parent tiles, fused level
                                     pairs); 1: plan creation times four candidate budget sets on this
                                     plan's own geometry (a few applies each, on a zero vector) and
                                     keeps the fastest; mlfma_plan_info reports the choice */
    int recompute_signatures;     /* reverse mode (mlfma_apply_vjp).  0 (default): a differentiable
                                     forward pass keeps grad phi of its charges (3 n complex values per
                                     right-hand side, from mlfma_apply_grad) for the backward pass;
                                     1: it keeps nothing (plain mlfma_apply) and mlfma_apply_vjp
                                     recomputes grad phi with one more gradient sweep.  The library
                                     reports the choice in mlfma_info; wrappers follow it */
    int test_fail_waits;          /* test hook, 0 (default) in normal use.  1: every bounded device
                                     wait of the apply (the M2L operator-slice copy, the tensor-core
                                     MMA completion) gives up at its first poll; the kernel then waits
                                     for its own copies in flight with the normal limit, raises the
                                     plan's error flag and returns, so MLFMA_ERR_TIMEOUT can be
                                     exercised without a stalled GPU */
    int dense_samples;            /* tensor-core precisions (TF32X3, BF16X3), opt-in: a level pair whose
                                     child sampling grid has at most this many samples runs its
                                     interpolation (M2M) and anterpolation (L2L) each as one dense real
                                     map on the tensor cores, the phi transforms, theta maps and shifts
                                     folded into it (Sec. 3.2.2, 3.2.4), in persistent kernels that keep
                                     a slice of the map in shared memory.  0 (default) or -1: never (the
                                     FFT path with tensor-core theta maps runs everywhere).  Ignored by
                                     FP32 and FP64 plans */
    int sampled_operators;        /* sampled translation operators (Sec. 3.2.3, "Translation Operators":
                                     where the operators do not fit, they are sampled and interpolated).
                                     0 (default): every far level keeps its full table T[316][K].
                                     s in [3, 32]: a level whose boxes are at least one wavelength wide
                                     (k edge >= 2 pi) keeps instead, per squared offset length |X/edge|^2,
                                     T as a function of the angle psi between khat and X, tabulated at
                                     psi_i = i pi / (s L), i = -10 .. s L + 10 (the padding holds the
                                     reflections at psi = 0 and pi); M2L interpolates each (offset,
                                     sample) entry with 10-point Lagrange weights as it stages an
                                     operator slice in shared memory.  Finer levels keep full tables
                                     (small, and their large |T| would magnify the interpolation
                                     error).  Error of the interpolated operators relative to max |T|:
                                     about 1e-5 (s = 4), 2e-7 (s = 6), 1e-8 (s = 8), 1e-11 (s = 16).
                                     max |T| exceeds the sums M2L forms by a factor that grows with L
                                     at small boxes: at 3 digits s = 6 keeps the potentials within
                                     1e-5 of the full tables' (s = 4: 1e-4); 6 digits (L = 26 at
                                     one-wavelength boxes, factor ~10^4) need s >= 16 */
} mlfma_options;

/* Summary of a plan (levels are numbered from the root, level 1). */
#define MLFMA_MAX_LEVELS 22
typedef struct mlfma_info {
    int64_t n;                    /* number of points */
    int nlev;                     /* deepest level */
    int top;                      /* highest level with far-field (M2L) work; 0 if none */
    int precision;
    double k, leaf_edge, root_edge;
    double root_corner[3];        /* x0: lower corner of the root cube */
    int64_t nbox[MLFMA_MAX_LEVELS + 1];     /* boxes per level */
    int64_t nleaf[MLFMA_MAX_LEVELS + 1];    /* leaves per level */
    int L[MLFMA_MAX_LEVELS + 1];            /* truncation per far-field level (0 elsewhere) */
    int64_t K[MLFMA_MAX_LEVELS + 1];        /* samples per box: (L+1)(2L+2) */
    int64_t nv[MLFMA_MAX_LEVELS + 1];       /* far-field (V) pairs per level */
    int64_t near_pairs;                      /* point pairs summed directly */
    int64_t device_bytes;                    /* device memory held by the plan */
    double setup_ms;                         /* wall time of mlfma_plan_create */
    int n_geom;                              /* geometries (1 unless created by mlfma_plan_create_batched;
                                                per-level fields are then those of geometry 0) */
    int tile_bytes[3];                       /* shared-memory budgets of the interpolation tiles in use:
                                                row tiles, per-parent tiles, fused level pairs */
    int recompute_signatures;                /* the plan's mlfma_options.recompute_signatures */
    int dense[MLFMA_MAX_LEVELS + 1];         /* 1 where the level pair (l, l + 1) runs as dense tensor-core
                                                maps (mlfma_options.dense_samples) */
    int sampled_operators;                   /* the plan's mlfma_options.sampled_operators */
    int sampled[MLFMA_MAX_LEVELS + 1];       /* 1 where the level's M2L interpolates sampled operators */
} mlfma_info;

/* Tree and list arrays that mlfma_plan_export can copy out (for verification). */
typedef enum {
    MLFMA_EXPORT_PERM = 0,        /* int32 [n]: sorted position -> caller index */
    MLFMA_EXPORT_KEYS = 1,        /* uint64 [n]: sorted Morton keys */
    MLFMA_EXPORT_BOX_KEY = 2,     /* uint64 [nbox(level)] */
    MLFMA_EXPORT_BOX_BEGIN = 3,   /* int32 [nbox(level)] first sorted point */
    MLFMA_EXPORT_BOX_END = 4,     /* int32 [nbox(level)] */
    MLFMA_EXPORT_BOX_PARENT = 5,  /* int32 [nbox(level)] */
    MLFMA_EXPORT_BOX_LEAF = 6,    /* uint8 [nbox(level)] */
    MLFMA_EXPORT_V_OFFSETS = 7,   /* int32 [nbox(level)+1] CSR offsets of the V lists */
    MLFMA_EXPORT_V_SOURCES = 8,   /* int32 [nv(level)] source boxes (same level), ascending */
    MLFMA_EXPORT_NEAR_OFFSETS = 9,/* int32 [nleaf_total+1] CSR offsets, leaves ordered by (level, key) */
    MLFMA_EXPORT_NEAR_SOURCES = 10,/* int32 [2*nnear] (source level, source box) pairs */
    MLFMA_EXPORT_F = 11,          /* complex [nbox(level)][K(level)]: last apply's multipole signatures */
    MLFMA_EXPORT_G = 12,          /* complex [nbox(level)][K(level)]: last apply's local signatures */
    MLFMA_EXPORT_NEAR_PHI = 13,   /* complex [n] sorted order: last apply's near-field part (last rhs) */
    MLFMA_EXPORT_TRANSLATION = 14,/* complex [316][K(level)]: translation operators of a level
                                     (MLFMA_ERR_UNSUPPORTED at a level with sampled operators) */
    MLFMA_EXPORT_OPERATOR_SAMPLES = 15 /* complex [28][s L + 21]: a sampled level's table, row |X/edge|^2
                                     (rows that no far offset has are zero), entry i + 10 = T at
                                     psi_i = i pi / (s L) (MLFMA_ERR_UNSUPPORTED at other levels) */
} mlfma_export_item;

/* Stages timed by mlfma_plan_profile / mlfma_plan_timings. */
typedef enum {
    MLFMA_STAGE_PERMUTE = 0,      /* caller order <-> Morton order */
    MLFMA_STAGE_P2P = 1,          /* near-field direct sums */
    MLFMA_STAGE_C2M = 2,
    MLFMA_STAGE_M2M = 3,          /* interpolate, shift, aggregate (all kernels of one level) */
    MLFMA_STAGE_M2L = 4,
    MLFMA_STAGE_L2L = 5,          /* shift, anterpolate, add */
    MLFMA_STAGE_L2O = 6,
    MLFMA_STAGE_COUNT = 7
} mlfma_stage;

typedef struct mlfma_timings {
    double ms[MLFMA_STAGE_COUNT];             /* summed CUDA-event time per stage */
    int64_t launches[MLFMA_STAGE_COUNT];      /* kernel launches per stage */
    double m2l_ms[MLFMA_MAX_LEVELS + 1];      /* M2L time per level */
    int64_t applies;                          /* right-hand sides applied while profiling */
} mlfma_timings;

/* Fills *opt with the defaults. */
void mlfma_options_init(mlfma_options* opt);

/*
 * Builds the octree, interaction lists, sampling grids, interpolation matrices
 * and translation operators of one point set.  Sec. 3.1 (tree, level count,
 * Morton keys), Sec. 2 (near/far rule), Sec. 3.2.3 (precomputed translation
 * operators).
 *   points   [n][3] FP64 xyz, device or host; copied.
 *   n        >= 1.
 *   k        wavenumber 2 pi / lambda, finite and > 0.
 *   digits   requested accuracy 1..12; sets the truncation per level.
 *   leaf_max 0 = level-uniform tree (leaf edge = options.leaf_edge, Sec. 3.1);
 *            > 0 = adaptive tree: split while a box holds more than leaf_max points,
 *            far field only on levels whose edge is >= the leaf edge.
 *   opt      NULL = defaults.
 *   out      receives the plan (NULL on error).
 * Errors: INVALID_ARG (n < 1, k, digits, leaf_max < 0, null pointers, non-finite
 * coordinates), UNSUPPORTED (uniform tree deeper than max_depth; more than 2^32
 * far-field samples on one level), OUT_OF_MEMORY, CUDA.  Synchronises the plan stream.
 */
mlfma_status mlfma_plan_create(const double* points, int64_t n, double k, int digits, int leaf_max,
                               const mlfma_options* opt, mlfma_plan** out);

/*
 * One plan for many independent geometries (each its own tree, lists and operators,
 * same k, digits and options); an apply runs all of them, concurrently on internal
 * streams, inside one captured CUDA graph.  Points of geometry g are
 * points[offsets[g] .. offsets[g+1]); vectors are [nrhs][offsets[n_geom]] in that order
 * and geometries never interact.
 *   offsets  host [n_geom + 1], offsets[0] = 0, strictly increasing.
 * Errors: as mlfma_plan_create; INVALID_ARG for bad offsets.  mlfma_plan_export and
 * mlfma_apply_near_noalloc reject batched plans.
 */
mlfma_status mlfma_plan_create_batched(const double* points, const int64_t* offsets, int n_geom, double k, int digits,
                                       int leaf_max, const mlfma_options* opt, mlfma_plan** out);

/*
 * phi = A q: the matvec above for nrhs right-hand sides (Sec. 2, five stages +
 * near field).  q [nrhs][n] complex, phi [nrhs][n] complex (overwritten).
 * Errors: INVALID_ARG (null plan/pointers, nrhs < 1), CUDA.
 */
mlfma_status mlfma_apply(mlfma_plan* plan, const void* q, void* phi, int nrhs);

/*
 * g = A^H r.  A is complex symmetric, so A^H r = conj(A conj(r)); the
 * conjugations are folded into the permutation kernels.  Same layout and
 * errors as mlfma_apply.
 */
mlfma_status mlfma_apply_adjoint(mlfma_plan* plan, const void* r, void* g, int nrhs);

/*
 * phi = A q and grad_i = grad_{r_i} phi_i, the gradient of each potential with
 * respect to its own target position (needed for derivatives of a loss with
 * respect to the points).  Near field: q_j e^{ikR} (ikR - 1) / R^3 (r_i - r_j)
 * per pair; far field: the L2O sum with the extra factor ik khat_p (Sec. 3.2.5).
 *   q     [nrhs][n] complex, device
 *   phi   [nrhs][n] complex, device, or NULL if only the gradient is wanted
 *   grad  [nrhs][n][3] complex, device (x, y, z components interleaved per point)
 * Errors: INVALID_ARG (null plan/q/grad, host pointers, nrhs < 1), CUDA.
 */
mlfma_status mlfma_apply_grad(mlfma_plan* plan, const void* q, void* phi, void* grad, int nrhs);

/*
 * Reverse mode of phi = A(r) q (Sec. 2, Eq. (1)): given the upstream gradient g of a real
 * loss L with respect to phi, the gradients of L with respect to the charges and the
 * positions.  Complex gradients follow PyTorch's convention, g = dL/dRe(phi) + i dL/dIm(phi).
 * A is complex symmetric, so with psi = A conj(g):
 *     grad_q   = dL/dRe(q) + i dL/dIm(q) = A^H g = conj(psi)
 *     grad_r_i = dL/dr_i = sum over right-hand sides of Re[conj(g_i) grad phi_i + q_i grad psi_i]
 * where grad phi_i and grad psi_i are gradients with respect to the target position r_i: the
 * first term is r_i's role as a target of phi_i, the second its role as a source of every other
 * phi_j (the kernel is symmetric, so those derivatives sum to the target gradient of psi).  One
 * gradient sweep computes psi and grad psi (the conjugations are folded into the permutation
 * kernels) and one kernel forms grad_r; with gphi = NULL a second gradient sweep recomputes
 * grad phi first.
 *   q       [nrhs][n] complex, device: the forward charges
 *   g       [nrhs][n] complex, device: upstream gradient
 *   gphi    [nrhs][n][3] complex, device, from mlfma_apply_grad on q; NULL = recompute
 *   grad_q  [nrhs][n] complex, device, or NULL (not wanted)
 *   grad_r  [n][3] FP64, device, or NULL (not wanted); summed over the right-hand sides
 * Scratch: plan-owned buffers (grown on first use, kept).  Synchronises the plan stream.
 * Errors: INVALID_ARG (null plan/q/g, host pointers, nrhs < 1, both outputs NULL), CUDA,
 * OUT_OF_MEMORY, TIMEOUT.
 */
mlfma_status mlfma_apply_vjp(mlfma_plan* plan, const void* q, const void* g, const void* gphi, void* grad_q,
                             double* grad_r, int nrhs);

/* Fills *info.  INVALID_ARG on null pointers. */
mlfma_status mlfma_plan_info(const mlfma_plan* plan, mlfma_info* info);

/*
 * Copies one tree/list/signature array to dst (device or host), for
 * verification.  level is ignored for per-point items.  bytes must be at
 * least the item's size (returned in *needed when dst is NULL).
 * Errors: INVALID_ARG (unknown item, level outside 1..nlev, too small), CUDA.
 * Synchronises the plan stream.
 */
mlfma_status mlfma_plan_export(const mlfma_plan* plan, int item, int level, void* dst, size_t bytes,
                               size_t* needed);

/*
 * Exact FP64 direct sum on the GPU at selected targets (the quantity the MLFMA
 * approximates, Sec. 2 Eq. (1)), for accuracy measurement.
 *   points [n][3] FP64 device, q [n] complex128 device, targets [nt] int64 device
 *   (caller indices), phi [nt] complex128 device.  Enqueued on ``stream``.
 * Errors: INVALID_ARG, CUDA.
 */
mlfma_status mlfma_direct_fp64(const double* points, int64_t n, const void* q, double k,
                               const int64_t* targets, int64_t nt, void* phi, void* stream);

/*
 * Starts (enable = 1) or stops (0) recording CUDA events around every stage of
 * the apply on the plan stream.  Recording adds two event records per stage
 * launch group and nothing else.  INVALID_ARG on a null plan.
 */
mlfma_status mlfma_plan_profile(mlfma_plan* plan, int enable);

/*
 * Synchronises the plan stream and returns the per-stage times recorded since
 * the last reset; reset = 1 clears them.  INVALID_ARG on null pointers, CUDA.
 */
mlfma_status mlfma_plan_timings(mlfma_plan* plan, mlfma_timings* out, int reset);

/*
 * Near-field part of phi = A q (the direct sums over each leaf's near lists, one
 * right-hand side) without allocating any device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate once they
 * are running (a fixed memory budget, or code that must not stall on an
 * allocation); they create the plan during set-up and call this afterwards.
 *   q, phi  [n] complex (precision of the plan), DEVICE pointers only; phi is
 *           overwritten, in the caller's point order.
 * Scratch: a file-scope 16 MiB device array (every GPU that loads the library
 * holds it until exit), so 2 n complex values must fit: n <= 1,048,576 for FP32
 * plans, n <= 524,288 for FP64 plans.  All calls share that array and it keeps
 * the last call's contents; calls that overlap on the GPU (several streams or
 * threads at once) race on it.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current; make
 * that first call before any stream capture.  Enqueued on the plan stream.
 * Errors: INVALID_ARG (null pointers, host pointers, n beyond the maximum), CUDA.
 */
mlfma_status mlfma_apply_near_noalloc(mlfma_plan* plan, const void* q, void* phi);

/* Outcome of mlfma_solve_gmres. */
typedef struct {
    int iterations;               /* Krylov steps taken (one matvec each) */
    int restarts;                 /* cycles begun after the first */
    int matvecs;                  /* applies of the plan, including one per cycle for the true residual */
    int converged;                /* 1 when the true relative residual reached tol */
    double rel_residual;          /* ||b - (sigma x + A x)||_2 / ||b||_2 at exit, from a fresh matvec */
} mlfma_solve_info;

/*
 * Iterative solve around the matvec (Sec. 1: the potential evaluation is the kernel of
 * an iterative integral-equation solver): restarted GMRES(restart) for
 *     (sigma I + A) x = b,
 * A the matrix the plan applies (no diagonal: pairs i = j contribute nothing) and
 * sigma = sigma_re + i sigma_im a diagonal term.  Orthogonalisation is classical
 * Gram-Schmidt applied twice per step on the device; the Hessenberg least-squares
 * problem (Givens rotations) is solved on the host, one small device-to-host copy
 * per step.  Each cycle starts from the true residual of a fresh matvec, and the
 * returned rel_residual is recomputed that way at exit.
 *   b  [n] complex (precision of the plan), DEVICE, caller order; not modified.
 *   x  [n] complex, DEVICE: the initial guess on entry, the iterate on exit.
 *   tol in (0, 1): stop when ||b - (sigma x + A x)|| <= tol ||b|| (the MLFMA's own
 *       error, about 10^-digits, bounds what tol can be met).
 *   restart in [1, 256]; max_iter >= 1 (Krylov steps over all cycles).
 * Scratch: (restart + 2) n complex values from the plan's allocator, released before
 * return.  Blocks until the solve ends.  Not converging is not an error (info->converged
 * = 0).  b = 0 gives x = 0.  Errors: INVALID_ARG (null or host pointers, parameters out
 * of range, non-finite sigma), OUT_OF_MEMORY, CUDA, TIMEOUT (as mlfma_apply).
 */
mlfma_status mlfma_solve_gmres(mlfma_plan* plan, const void* b, void* x, double sigma_re, double sigma_im,
                               double tol, int restart, int max_iter, mlfma_solve_info* info);

/* Releases all device memory of the plan after synchronising its stream.  NULL-safe. */
void mlfma_destroy(mlfma_plan* plan);

/* Message of the last error on this thread ("" if none). */
const char* mlfma_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MLFMA_H */
