// Internal declarations of the MLFMA library (plan layout, helpers, kernels' launchers).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <cmath>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/mlfma.h"

namespace mlfma {

constexpr int kMaxLev = MLFMA_MAX_LEVELS;   // levels 1..22 (21 key bits per axis)
constexpr int kBits = 21;
constexpr int kNumOffsets = 316;            // [-3,3]^3 minus [-1,1]^3: far offsets of one level
constexpr int kSmallLeaf = 64;              // P2P: leaves up to this size take one warp
constexpr int kP2PTile = 128;               // P2P: targets per CTA for larger leaves
constexpr int kMaxNR = 4;                   // right-hand sides per pass of the sweep

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
struct Failure {
    mlfma_status status;
};
[[noreturn]] void fail(mlfma_status st, const char* fmt, ...);

#define MLFMA_CUDA(call)                                                                     \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            ::mlfma::fail(e_ == cudaErrorMemoryAllocation ? MLFMA_ERR_OUT_OF_MEMORY          \
                                                          : MLFMA_ERR_CUDA,                  \
                          "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,  \
                          __LINE__);                                                         \
    } while (0)

#define MLFMA_LAUNCH_CHECK() MLFMA_CUDA(cudaGetLastError())

// ---------------------------------------------------------------- complex helpers
template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

template <typename C> __host__ __device__ __forceinline__ C cmake(decltype(C::x) a, decltype(C::x) b) {
    C c; c.x = a; c.y = b; return c;
}
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return cmake<C>(a.x + b.x, a.y + b.y); }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
    return cmake<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { return cmake<C>(a.x, -a.y); }
// acc += a * b
template <typename C> __host__ __device__ __forceinline__ void cfma(C& acc, C a, C b) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename C> __host__ __device__ __forceinline__ void cfma_conj(C& acc, C a, C b) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}
// acc += s * b (s real)
template <typename C, typename R> __host__ __device__ __forceinline__ void crfma(C& acc, R s, C b) {
    acc.x = fma(s, b.x, acc.x); acc.y = fma(s, b.y, acc.y);
}

// ---------------------------------------------------------------- device allocation
struct Allocator {
    void* (*alloc)(size_t, void*, void*) = nullptr;
    void (*free)(void*, void*, void*) = nullptr;
    void* ctx = nullptr;
    cudaStream_t stream = nullptr;
    std::vector<std::pair<void*, size_t>> live;
    size_t bytes = 0;
    void* get(size_t n);
    void drop(void* ptr);          // releases one allocation made by get (no-op for nullptr)
    template <typename T> T* make(size_t count) { return static_cast<T*>(get(count * sizeof(T))); }
    void release_all();
};

// ---------------------------------------------------------------- plan layout
struct TreeLevel {                 // one octree level (root = 1)
    int l = 0;
    double edge = 0;
    int64_t nbox = 0;
    uint64_t* key = nullptr;       // [nbox] ascending level keys
    int* begin = nullptr;          // [nbox] first sorted point
    int* end = nullptr;            // [nbox]
    int* parent = nullptr;         // [nbox] box at level l-1 (-1 at root)
    int* child_begin = nullptr;    // [nbox] first child at level l+1
    int* child_end = nullptr;      // [nbox]
    uint8_t* leaf = nullptr;       // [nbox]
    int* ijk = nullptr;            // [nbox][3]
    double* center = nullptr;      // [nbox][3]
    int* coll = nullptr;           // [nbox][27] colleagues (-1 absent), slot = (dx+1)+3(dy+1)+9(dz+1)
    int* v_off = nullptr;          // [nbox+1]
    int* v_src = nullptr;          // [nv]
    int64_t nv = 0;
    int64_t nleaf = 0;
    // leaves of this level split by size for C2M / L2O: small ones take one warp, larger
    // ones a CTA per sample chunk (C2M) or per tile of kP2PTile points (L2O)
    int* small_leaves = nullptr;   // [n_small_leaves] box indices
    int64_t n_small_leaves = 0;
    int* big_leaves = nullptr;     // [n_big_leaves] box indices
    int64_t n_big_leaves = 0;
    int2* big_tiles = nullptr;     // [n_big_tiles] (box, first point offset)
    int64_t n_big_tiles = 0;
    // forest plans: boxes of this level without a parent (a geometry's first level in the
    // forest), as (first box, count) ranges; L2L into this level zeroes their spectral rows
    int2* orphans = nullptr;
    int n_orphan_ranges = 0;
    int64_t n_orphans = 0;
    // M2L work of the children of each box (this level acting as parent level):
    // per box, the candidate sources with at least one far child, packed
    // (src * K) << 32 | far-children mask << 8 | code, code = colleague slot (0..26) * 8 + source octant
    int* m2l_off = nullptr;        // [nbox+1]
    unsigned long long* m2l_src = nullptr;   // [m2l_n]
    int64_t m2l_n = 0;
};

// x / d for 0 <= x < 2^31 by multiply-high and shift (round-up multiplier, Granlund and
// Montgomery 1994): q = (umulhi(x, m) + x) >> l with l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1
struct FastDiv {
    unsigned m = 1;
    int l = 0;
    static FastDiv make(unsigned d) {
        FastDiv f;
        while ((1ull << f.l) < d) ++f.l;
        f.m = (unsigned)(((1ull << 32) * ((1ull << f.l) - d)) / d + 1);
        return f;
    }
    __host__ __device__ __forceinline__ unsigned div(unsigned x) const {
#ifdef __CUDA_ARCH__
        return (__umulhi(x, m) + x) >> l;
#else
        return (unsigned)((((unsigned long long)x * m) >> 32) + x) >> l;
#endif
    }
};

struct FftPlan {                   // mixed-radix factorisation of an FFT length (radices 2, 3, 4, 5, 7)
    int n = 0;
    int ns = 0;
    int r[16] = {0};
    // per Stockham stage st: Ns = r[0] ... r[st-1], nb = n / r[st] butterflies per row,
    // tstep = n / (Ns r[st]) twiddle stride
    int Ns[16] = {0}, nb[16] = {0}, tstep[16] = {0};
    FastDiv dNs[16], dnb[16];
    FastDiv dn;                    // divides by n
};
FftPlan make_fft_plan(int n);
int smooth_even(int m);

constexpr int kTBoxRows = 172;     // rows of one TMA box of T (two boxes cover the 343 rows)
// sampled operators: Lagrange points per interpolated entry, and table rows (|X/edge|^2 = 0..27)
constexpr int kOpOrder = 10;
constexpr int kOpRows = 28;

struct FarLevel {                  // sampling grid, operators and signatures of one far-field level
    int L = 0, nth = 0, nph = 0;
    FftPlan fft;                   // plan for length nph
    int64_t K = 0;
    double* x = nullptr;           // [nth] Gauss-Legendre nodes (cos theta), ascending, FP64
    double* wgl = nullptr;         // [nth] weights, FP64
    void* dirs = nullptr;          // [K][4] real: khat_p (x, y, z) and quadrature weight w_p
    void* tw = nullptr;            // [nph] complex: e^{-2 pi i j / nph}
    void* T = nullptr;             // [343][K] complex translation operators by offset raster index
                                   // (dx+3) + 7 (dy+3) + 49 (dz+3); the 27 near rows are zero
    CUtensorMap tmT;               // TMA descriptor of T (boxes of 32 samples x kTBoxRows rows)
    // sampled operators (instead of T, at levels with k edge >= 2 pi when the plan asks for them):
    // T1[d2][i + kOpOrder] = T at angle psi_i = i pi / S between khat and X, |X/edge|^2 = d2,
    // i = -kOpOrder .. S + kOpOrder, S = s L; T1n = S + 2 kOpOrder + 1 entries per row
    void* T1 = nullptr;
    int T1n = 0;
    double T1inv_h = 0;            // S / pi
    void* F = nullptr;             // [nbox][K] complex multipole signatures
    void* G = nullptr;             // [nbox][K] complex local signatures
    // interpolation from level l+1 (child) to this level (parent); set when l+1 is far-field
    void* At = nullptr;            // [Lc+1][nth_c][nth_p] real: At[m][i][i'] = A_m[i'][i]
    void* Bt = nullptr;            // [Lc+1][nth_p][nth_c] real: Bt[m][i'][i] = A_m[i'][i] w'_i' / w_i
    // the same maps split by parity (Gauss-Legendre nodes come in pairs x, -x, and
    // Pbar_n^m(-x) = (-1)^(n+m) Pbar_n^m(x), so each map is centrosymmetric): for input index
    // i < ceil(nin/2) and output index o < ceil(nout/2), E = the terms n + m even, D = n + m odd,
    // times the map's weights; E's middle input row (odd nin) is halved, D's middle row and
    // column are zero.  Layout [Lc+1][ceil(nin/2)][ceil(nout/2)] real.
    void* AtE = nullptr;           // M2M (nin = nth_c, nout = nth_p)
    void* AtD = nullptr;
    void* BtE = nullptr;           // L2L (nin = nth_p, nout = nth_c)
    void* BtD = nullptr;
    void* AtTc = nullptr;          // tensor-core precisions: At and Bt split into hi + lo parts, in the
    void* BtTc = nullptr;          // blocks the MMA reads (one per mode, output tile and K chunk)
    // tensor-core precisions, fine level pairs: the whole interpolation (anterpolation) of the
    // pair as one real Kp x Kc (Kc x Kp) matrix, split into the MMA's operand blocks, and the
    // children's shifts by octant
    int dense = 0;
    void* DmTc = nullptr;          // M2M: Pm (child samples -> parent samples)
    void* DlTc = nullptr;          // L2L: Qm (parent samples -> child samples)
    void* Soct = nullptr;          // [8][K] complex: Sz[o >> 2][i'] Sxy[o & 3][i'][j']
    void* Sz = nullptr;            // [2][nth] complex: e^{-ik cos(theta_i') dz}, dz = -+ edge/4
    void* Sxy = nullptr;           // [4][K] complex: e^{-ik sin(theta)(cos(phi) dx + sin(phi) dy)}
    void* X = nullptr;             // [nbox(l+1)][2Lc+1][nth_c] complex scratch (spectral, child grid)
    void* Y = nullptr;             // [nbox(l+1)][2Lc+1][nth_p] complex scratch (spectral, parent rows)
};

struct Plan {
    int64_t n = 0;
    double k = 0;
    int digits = 0, leaf_max = 0, max_depth = 12, margin = 1;
    mlfma_precision prec = MLFMA_PREC_FP32;
    int* dev_err = nullptr;        // raised by kernels whose bounded waits ran out
    long long wait_first = 1ll << 22;   // polls of a kernel's first try of a bounded wait (0: test hook)
    int recompute = 0;             // mlfma_options.recompute_signatures
    int op_s = 0;                  // mlfma_options.sampled_operators (oversampling s; 0 = full tables)
    void* vjp_buf = nullptr;       // [nrhs_vjp][n][3] complex: grad psi kept while grad phi is recomputed
    int nrhs_vjp = 0;
    int far_nr = 1;                // right-hand sides the far-level signatures F, G have room for
    bool graphs_stale = false;     // buffers captured by earlier graphs were replaced
    double leaf_edge = 0, a1 = 0, D0 = 0;
    double x0[3] = {0, 0, 0}, scale = 0;
    int nlev = 0, top = 0;
    int* off343 = nullptr;         // [343] (dx+3)+7(dy+3)+49(dz+3) -> far-offset index 0..315, -1 if near
    cudaStream_t stream = nullptr;
    Allocator mem;
    // per point (sorted order)
    double* pos = nullptr;         // [n][3] sorted positions, FP64
    uint64_t* keys = nullptr;      // [n] sorted keys
    int* perm = nullptr;           // [n] sorted -> caller index
    int* leaf_of_pt = nullptr;     // [n] index into the leaf table
    // leaf table (all leaves, ordered by (level, key))
    int64_t nleaf_total = 0;
    int* leaf_level = nullptr;     // [nleaf_total]
    int* leaf_box = nullptr;       // [nleaf_total]
    std::vector<int64_t> leaf_first;  // host: first leaf-table index of each level
    // near field: per leaf, source boxes (level, box) summed directly
    int* near_off = nullptr;       // [nleaf_total+1]
    int* near_lev = nullptr;       // [nnear]
    int* near_box = nullptr;       // [nnear]
    int64_t nnear = 0, near_pairs = 0;
    // P2P work split: leaves with at most kSmallLeaf points (one warp each) and
    // tiles of kP2PTile targets of the larger leaves (one CTA each)
    int* p2p_small = nullptr;      // [n_small] leaf-table indices: first the n_small32 leaves with at
    int64_t n_small = 0;           // most 32 points, then those with 33 .. kSmallLeaf
    int64_t n_small32 = 0;
    int2* p2p_tiles = nullptr;     // [n_tiles] (leaf-table index, first target offset)
    int64_t n_tiles = 0;
    // symmetric near field of the large leaves (one right-hand side, no gradient): each pair of
    // mutually near large leaves (A, B), A < B in the leaf table, and each large leaf with itself
    // (pairs j > i) is evaluated once by k_p2p_sym, whose work items (A, target offset in A, B,
    // scratch offset) write both directions' partial sums to sym_buf; k_p2p_sym_reduce adds them
    // to the potentials in a fixed order.  The tiled kernel then takes the large leaves' remaining
    // near boxes (asym_*).
    int64_t n_sym_items = 0;
    int4* sym_items = nullptr;     // [n_sym_items]
    void* sym_buf = nullptr;       // complex [sum over items of kP2PTile + |B|]
    int* asym_off = nullptr;       // [nleaf_total+1] CSR over the leaf table (large leaves only)
    int* asym_lev = nullptr;
    int* asym_box = nullptr;
    int* sym_red_off = nullptr;    // [nleaf_total+1] per large leaf: its blocks in sym_buf
    int2* sym_red = nullptr;       // (item scratch offset, target offset of the item in this leaf, or -1: B side)
    TreeLevel lev[kMaxLev + 1];
    FarLevel far[kMaxLev + 1];
    // apply buffers
    void* qs = nullptr;            // [nrhs_cap][n] complex, sorted order
    void* phis = nullptr;          // [nrhs_cap][n] complex, sorted order
    void* near_dump = nullptr;     // [n] complex near-field part of the last apply
    void* grads = nullptr;         // [nrhs_grad][n][3] complex, sorted order
    int nrhs_grad = 0;
    int nrhs_cap = 0;
    void* host_stage = nullptr;    // device staging for host pointers: [2][nrhs_stage][n] complex
    int nrhs_stage = 0;
    double setup_ms = 0;
    // caller-order staging of one apply: the captured graph reads q from qin and writes
    // phiout / gout, so one graph serves every call with the same nrhs
    void* qin = nullptr;           // [nrhs_io][ntot] complex
    void* phiout = nullptr;        // [nrhs_io][ntot] complex
    void* gout = nullptr;          // [nrhs_io][ntot][3] complex
    int nrhs_io = 0;
    int64_t ntot = 0;              // points of the plan (sum over geometries for batched plans)
    // CUDA graphs of the apply sweep, keyed by nrhs * 4 + adjoint * 2 + grad
    bool use_graphs = true;
    // shared-memory budgets (bytes) of the interpolation tiles: row-tile FFT kernels, per-parent
    // kernels, fused level pairs; defaults from sweeps on a 2^20-point sphere, or chosen by the
    // plan-time autotuner
    int tile_fft = 20 * 1024, tile_parent = 32 * 1024, tile_fused = 40 * 1024;
    // tensor-core precisions: level pairs whose child grid has at most this many samples run
    // as dense maps (0: never, the default)
    int dense_kc = 0;
    cudaStream_t gstream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // near field beside the far field: P2P runs on nstream from ev_nfork while the far field's
    // upward and downward passes run on the plan stream, which waits for ev_near before L2O
    // (single and forest plans; null: one stream)
    cudaStream_t nstream = nullptr;
    cudaEvent_t ev_nfork = nullptr, ev_near = nullptr;
    // M2L beside the upward pass: a level's M2L runs on mstream once its F is complete (ev_mfork,
    // recorded after the level's C2M and M2M), while the plan stream goes on up the tree; the
    // downward pass waits for ev_mdone, recorded after the last (top) level's M2L
    cudaStream_t mstream = nullptr;
    cudaEvent_t ev_mfork = nullptr, ev_mdone = nullptr;
    // inside the near field of plans with large leaves: the small leaves' kernels run on sstream
    // beside the large leaves' tiled and symmetric kernels (disjoint targets), joined by ev_sdone
    cudaStream_t sstream = nullptr;
    cudaEvent_t ev_sfork = nullptr, ev_sdone = nullptr;
    std::map<int64_t, cudaGraphExec_t> graphs;
    // batched plans: independent geometries; level-uniform ones are merged into this plan as a
    // forest (the sub-plans then only hold the shared operators), others run concurrently on
    // sub_streams
    bool forest = false;
    std::vector<Plan*> subs;
    std::vector<int64_t> sub_off;  // [n_geom + 1] offsets into the caller's point order
    std::vector<cudaStream_t> sub_streams;
    std::vector<cudaEvent_t> sub_events;
    // stage profiling (CUDA events on the plan stream)
    bool profiling = false;
    struct EventRec {
        int stage, level, launches;
        cudaEvent_t a, b;
    };
    std::vector<EventRec> recs;
    std::vector<cudaEvent_t> pool;
    mlfma_timings acc{};
};

// Records CUDA events around a group of launches of one stage while profiling is on.
struct StageTimer {
    Plan& p;
    int idx = -1;
    StageTimer(Plan& plan, int stage, int level, int launches, bool on = true);
    ~StageTimer();
};
void collect_timings(Plan& p);

size_t csize(const Plan& p);       // bytes per complex number
const char* prec_name(mlfma_precision p);

// ---------------------------------------------------------------- steps (host launchers)
// tree.cu
void build_tree(Plan& p, const double* pts_dev);
void build_lists(Plan& p);
// setup.cu
int truncation_L(double edge, double k, int digits, int margin);
void encode_translation_map(FarLevel& F, size_t csz);
void build_far_levels(Plan& p);
void build_m2l_lists(Plan& p);
void build_p2p_work(Plan& p);
void prepare_kernels(Plan& p);
// forest.cu
bool forest_possible(const std::vector<Plan*>& subs);
void build_forest(Plan& P);
// theta_tc.cu: split-TF32 tensor-core theta maps (complex64 data)
void prepare_theta_tc();
void launch_theta_map_tc(const Plan& p, int64_t nbox, int Lc, int nin, int nout, const void* Mtc, const float2* in,
                         float2* out, cudaStream_t s);
size_t theta_tc_map_bytes(const Plan& p, int nmaps, int nin, int nout);
// dense_tc.cu: fine level pairs as dense tensor-core maps (persistent kernels)
void prepare_dense_tc();
bool dense_tc_fits(const Plan& p, int Kc, int Kp);
size_t dense_tc_map_bytes(const Plan& p, bool m2m, int K, int Nout);
void presplit_dense_tc(const Plan& p, bool m2m, int K, int Nout, const float* M, void* out, cudaStream_t s);
void launch_dense_m2m_tc(const Plan& p, int64_t nbox_c, int Kc, int Kp, const void* Mtc, const int* par,
                         const uint64_t* ckey, const float2* soct, const float2* Fc, float2* Fp, cudaStream_t s);
void launch_dense_l2l_tc(const Plan& p, int64_t nbox_c, int Kp, int Kc, const void* Mtc, const int* par,
                         const uint64_t* ckey, const float2* soct, const float2* Gp, float2* Gc, cudaStream_t s);
void presplit_theta_tc(const Plan& p, int nmaps, int nin, int nout, const float* M, void* out, cudaStream_t s);
// far.cu / near.cu
// one right-hand side in sorted order; grads_r (nullable): [n][3] complex gradient of phi
// nr right-hand sides per pass (1, or kMaxNR without gradients): q and phi r n apart
void apply_pipeline(Plan& p, const void* qs_r, void* phis_r, void* grads_r, int nr);
void far_apply(Plan& p, const void* qs, void* phis, void* grads, int nr, cudaEvent_t near_done = nullptr);
// one apply of a top-level plan on a device vector in caller order; the result stays in P.phiout
void apply_device(Plan& P, const void* q);
// restarted GMRES on (sigma I + A) x = b with the plan's matvec (solve.cu)
void gmres_solve(Plan& P, const void* b, void* x, double sr, double si, double tol, int restart, int max_iter,
                 mlfma_solve_info* info);
// ld: row stride of the caller-order vectors (default n)
void permute_out3(Plan& p, const void* gs, void* g, int nrhs, int64_t ld = -1);
// grad_r[i][a] = sum_r Re[conj(g[r][i]) gphi[r][i][a] + q[r][i] gpsi[r][i][a]] (caller order, FP64 out)
void position_grad(const Plan& p, int64_t n, int nrhs, const void* q, const void* g, const void* gphi, const void* gpsi,
                   double* grad_r, cudaStream_t s);
void permute_in(Plan& p, const void* q, void* qs, int nrhs, bool conj, int64_t ld = -1);
void permute_out(Plan& p, const void* phis, void* phi, int nrhs, bool conj, int64_t ld = -1);
void direct_fp64(const double* pts, int64_t n, const void* q, double k, const int64_t* tg, int64_t nt,
                 void* phi, cudaStream_t s);

// device-wide exclusive scan of int32 (returns total); tmp must hold scan_tmp_ints(n) ints
int64_t scan_tmp_ints(int64_t n);
int scan_exclusive(const int* in, int* out, int64_t n, int* tmp, cudaStream_t s);

// near field only (P2P over the near lists), one right-hand side, sorted order; timed = false
// records no stage events even while the plan is profiling
void near_only(Plan& p, const void* qs, void* phis, bool timed = true);

}  // namespace mlfma

// the opaque handle of the C ABI
struct mlfma_plan {
    mlfma::Plan p;
};
