// Interpolation (Sec. 3.2.2) and anterpolation (Sec. 3.2.4) of the fine level pairs as dense
// maps on the 5th-generation tensor cores (precisions MLFMA_PREC_FP32_TF32X3 / _BF16X3).
//
// Per child box c of parent P, octant o (shift S_o = Sz[o >> 2] Sxy[o & 3] on the parent grid):
//   M2M:  F_P[s'] = sum_c S_o[s'] sum_s Pm[s'][s] F_c[s]              Pm: Kp x Kc real
//   L2L:  G_c[s] += sum_s' Qm[s][s'] conj(S_o[s']) G_P[s']             Qm: Kc x Kp real
// Pm (Qm) is the composition of the forward phi transform, the theta maps of every mode and
// the inverse phi transform that the FFT path applies one after another (the matrices are built
// at plan creation).  Each is a GEMM with the child boxes as M (A rows 2b = Re, 2b + 1 = Im of
// box b, 64 boxes per tile) and the output samples as N, split x = hi + lo and accumulated in
// FP32 as hi*hi + hi*lo + lo*hi (see tc_common.cuh for the two split forms).
//
// Kernel structure (persistent, one CTA per SM, 288 threads in three roles):
//   - the CTA owns one N slice of the map (NS output samples): both split parts stay resident in
//     shared memory, loaded once by one bulk copy; the CTA walks the box tiles t = first, first +
//     stride, ...;
//   - warps 4-7 (producers) load the tile's A rows (M2M: F_c; L2L: conj(S_o) G_P of each child's
//     parent), split them and store them into a ring of two stages of 64 (BF16) or 32 (TF32) K
//     values, one register-prefetched chunk ahead;
//   - one thread of warp 8 issues tcgen05.mma (M = 128, N = the slice) from the stages and the
//     resident map into one of two tensor-memory accumulators, and commits each stage back to
//     the producers and each finished tile to the epilogue;
//   - warps 0-3 (epilogue) read the accumulator rows (tcgen05.ld, lanes 32 w ..) while the next
//     tile accumulates in the other buffer.  M2M: rows pass through a small shared buffer, and
//     each parent whose first child lies in the tile's first 56 rows (all its <= 8 children are
//     then among the 64) is summed with its children's shifts and written; no atomics.  L2L:
//     lane pairs exchange halves so that each lane adds 8 consecutive complex samples to G.
// Every mbarrier wait is bounded; a wait that runs out raises the plan's error flag and a
// shared abort flag that ends the other roles' waits, the CTA waits (normal limit) for its
// copy and MMAs in flight, releases its tensor memory and returns.
#include <algorithm>

#include "common.cuh"
#include "tc_common.cuh"

namespace mlfma {

namespace {

using tc::SplitBF16;
using tc::SplitTF32;
using tc::smem_u32;

constexpr int kDM = 128;                     // MMA M: 64 child boxes x (Re, Im)
constexpr int kDBoxes = 64;
constexpr int kDAnchor = 56;                 // M2M tile t: parents whose first child is box 56 t .. 56 t + 55
constexpr int kDRowBytes = 128;              // A stage: bytes per row (4 MMA K-steps)
constexpr uint32_t kDAPart = kDM * kDRowBytes;   // one split part of an A stage (16 KB)
constexpr int kDStages = 2;
constexpr int kDThreads = 288;               // warps 0-3 epilogue, 4-7 producers, 8 MMA
constexpr int kDZPitch = 20;                 // M2M epilogue buffer: floats per accumulator row (16 used)
constexpr int kDMaxChunks = 16;              // 16-column chunks of a slice (NS <= 256)
constexpr int kDL2LChunks = 6;               // L2L: NS <= 96, so a lane's G values fit in registers
constexpr size_t kDSmemMax = 232448 - 3072;  // dynamic shared memory (the static part stays below 3 KB)

enum { kDenseM2M = 0, kDenseL2L = 1 };

struct DenseShape {
    int K, Kpad, Nout, NS, nslices;
    size_t bslice;                           // bytes of one pre-split slice (hi + lo)
    size_t smem;                             // dynamic shared memory of the kernel
};

template <typename Op>
DenseShape dense_shape(int K, int Nout, bool m2m) {
    DenseShape d{};
    const int ES = (int)sizeof(typename Op::T);
    d.K = K;
    d.Kpad = (K + 15) & ~15;
    d.Nout = Nout;
    const size_t fixed = (size_t)kDStages * 2 * kDAPart + (m2m ? (size_t)kDM * kDZPitch * sizeof(float) : 0);
    const size_t row = (size_t)d.Kpad * ES * 2;                      // one map row, hi + lo
    int rmax = (int)((kDSmemMax - fixed) / row) / 16 * 16;
    rmax = std::min(rmax, m2m ? 16 * kDMaxChunks : 16 * kDL2LChunks);
    if (rmax < 16) return d;                                         // NS = 0: does not fit
    d.nslices = (Nout + rmax - 1) / rmax;
    d.NS = ((Nout + d.nslices - 1) / d.nslices + 15) & ~15;
    d.bslice = (size_t)d.NS * row;
    d.smem = fixed + d.bslice;
    return d;
}

// Pre-split slices of a map M [K][Nout] (row k, column n): slice t holds B[n][k] = M[k][t NS + n]
// as two parts [hi, lo], each NS rows x Kpad in the canonical K-major core layout (zero outside
// K x Nout).  One thread per element.
template <typename Op>
__global__ void k_presplit_dense(int K, int Kpad, int Nout, int NS, int nslices, const float* __restrict__ M,
                                 unsigned char* __restrict__ out) {
    using T = typename Op::T;
    const int64_t per = (int64_t)NS * Kpad;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nslices * per) return;
    const int t = (int)(idx / per);
    const int e = (int)(idx - t * per);
    const int n = e / Kpad, k = e - n * Kpad;
    const int gn = t * NS + n;
    const float v = (gn < Nout && k < K) ? M[(int64_t)k * Nout + gn] : 0.f;
    T h, lo;
    Op::split(v, h, lo);
    unsigned char* base = out + (int64_t)t * 2 * per * (int64_t)sizeof(T);
    const uint32_t off = tc::core_off_kr<T>(n, k, Kpad);
    tc::st_part(base, off, h);
    tc::st_part(base + per * (int64_t)sizeof(T), off, lo);
}

struct DenseArgs {
    int nbox;                                // child boxes
    int K, Kpad, Nout, NS, nslices;
    int ntiles;                              // box tiles
    const unsigned char* Bm;                 // pre-split slices
    const float2* in;                        // M2M: F_c [nbox][K]; L2L: G_P [nbox_p][K]
    float2* out;                             // M2M: F_P [nbox_p][Nout]; L2L: G_c [nbox][Nout] (added to)
    const int* par;                          // parent of each child box (-1: none)
    const uint64_t* ckey;                    // child keys (octant = key & 7)
    const float2* soct;                      // [8][Kp] shifts S_o
    int* err;
    long long wait_first;
};

// the 8 K values of group kg of box row b, the two split parts stored as 16-byte core rows
template <typename Op> struct GroupStore;

template <> struct GroupStore<SplitBF16> {
    // 8 BF16 values = one core row (16 bytes)
    __device__ static void store(unsigned char* part_hi, unsigned char* part_lo, int row, int k, const float (&x)[8]) {
        uint4 h, l;
        SplitBF16::split2(x[0], x[1], h.x, l.x);
        SplitBF16::split2(x[2], x[3], h.y, l.y);
        SplitBF16::split2(x[4], x[5], h.z, l.z);
        SplitBF16::split2(x[6], x[7], h.w, l.w);
        const uint32_t off = tc::core_off_kr<__nv_bfloat16>(row, k, kDRowBytes / 2);
        *reinterpret_cast<uint4*>(part_hi + off) = h;
        *reinterpret_cast<uint4*>(part_lo + off) = l;
    }
};

template <> struct GroupStore<SplitTF32> {
    // 8 TF32 values = two core rows
    __device__ static void store(unsigned char* part_hi, unsigned char* part_lo, int row, int k, const float (&x)[8]) {
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
            uint2 ha, la, hb, lb;
            SplitTF32::split2(x[4 * h2], x[4 * h2 + 1], ha, la);
            SplitTF32::split2(x[4 * h2 + 2], x[4 * h2 + 3], hb, lb);
            const uint32_t off = tc::core_off_kr<float>(row, k + 4 * h2, kDRowBytes / 4);
            *reinterpret_cast<uint4*>(part_hi + off) = make_uint4(ha.x, ha.y, hb.x, hb.y);
            *reinterpret_cast<uint4*>(part_lo + off) = make_uint4(la.x, la.y, lb.x, lb.y);
        }
    }
};

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 128;\n" ::: "memory"); }

template <typename Op, int MODE>
__global__ void __launch_bounds__(kDThreads, 1) k_dense_tc(const DenseArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t s_bar[1 + 2 * kDStages + 4];
    __shared__ uint32_t s_taddr;
    __shared__ volatile int s_abort;
    __shared__ int s_ok;                     // epilogue: outcome of the accumulator wait of this tile
    __shared__ int s_par[kDBoxes];           // epilogue (M2M): parent of each row's box
    __shared__ unsigned char s_oct[kDBoxes];
    __shared__ int s_prev, s_np, s_plist[kDBoxes];
    __shared__ unsigned char s_nch[kDBoxes];         // children of each listed parent
    __shared__ float2 s_sh[8][16];                   // M2M: shifts S_o of the current 16 columns
    using T = typename Op::T;
    constexpr int ES = (int)sizeof(T);
    constexpr int KC = kDRowBytes / ES;      // K values per A stage
    constexpr int GPB = KC / 8;              // 8-value groups per box and stage
    constexpr int GPT = kDBoxes * GPB / 128; // groups per producer thread and stage
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nsl = a.nslices;
    const int slice = blockIdx.x % nsl;
    const int tstride = gridDim.x / nsl;
    const int tfirst = blockIdx.x / nsl;
    const int n0 = slice * a.NS;
    const int N = min(a.NS, a.Nout - n0);
    const int Np = (N + 15) & ~15;
    const uint32_t accoff = a.NS <= 128 ? 128u : 256u;               // column of accumulator 1
    const uint32_t ncols = 2 * accoff;
    const uint32_t bpart = (uint32_t)a.NS * a.Kpad * ES;              // one part of the resident slice
    const uint32_t sB = smem_u32(smem);
    unsigned char* pA = smem + 2 * bpart;
    const uint32_t sA = sB + 2 * bpart;
    float* zbuf = reinterpret_cast<float*>(pA + kDStages * 2 * kDAPart);
    const uint32_t bar0 = smem_u32(&s_bar[0]);                       // B slice landed
    auto bar_full = [&](int s) { return bar0 + 8u * (1 + s); };       // A stage s filled (128 producers)
    auto bar_empty = [&](int s) { return bar0 + 8u * (1 + kDStages + s); };   // A stage s read (commit)
    auto bar_accf = [&](int q) { return bar0 + 8u * (1 + 2 * kDStages + q); };   // accumulator q done (commit)
    auto bar_acce = [&](int q) { return bar0 + 8u * (3 + 2 * kDStages + q); };   // accumulator q read (128)
    const int K = a.K;
    const int nchunks = (K + KC - 1) / KC;
    const int ntiles = a.ntiles;
    const int tile_boxes = MODE == kDenseM2M ? kDAnchor : kDBoxes;

    if (warp == 8) tc::tmem_alloc(smem_u32(&s_taddr), ncols);
    if (threadIdx.x == 0) {
        tc::mbar_init(bar0, 1);
        for (int s = 0; s < kDStages; ++s) {
            tc::mbar_init(bar_full(s), 128);
            tc::mbar_init(bar_empty(s), 1);
        }
        for (int q = 0; q < 2; ++q) {
            tc::mbar_init(bar_accf(q), 1);
            tc::mbar_init(bar_acce(q), 128);
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_taddr;
    const long long limit = a.wait_first;
    // bounded wait that also gives up once another role has aborted; a wait that runs out aborts
    auto wait = [&](uint32_t b, uint32_t parity) -> bool {
        for (long long i = 0; i < limit; ++i) {
            uint32_t done;
            asm volatile(
                "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}\n"
                : "=r"(done)
                : "r"(b), "r"(parity)
                : "memory");
            if (done) return true;
            if ((i & 31) == 31 && s_abort) return false;
        }
        s_abort = 1;
        atomicExch(a.err, 1);
        return false;
    };

    if (warp == 8) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            tc::bulk_load(sB, a.Bm + (size_t)slice * 2 * bpart, 2 * bpart, bar0);
            bool ok = wait(bar0, 0);
            bool landed = ok;
            const uint32_t idesc = Op::idesc(kDM, Np);
            const uint32_t sboB = (uint32_t)(a.Kpad / (16 / ES)) * 128u;
            uint32_t last_bar = 0, last_par = 0;
            int g = 0, it = 0;
            if (ok) tc::fence_after_sync();
            for (int t = tfirst; ok && t < ntiles; t += tstride, ++it) {
                const int q = it & 1, v = it >> 1;
                if (v >= 1 && !wait(bar_acce(q), (v - 1) & 1)) { ok = false; break; }
                tc::fence_after_sync();
                const uint32_t d = tmem + (uint32_t)q * accoff;
                for (int ch = 0; ch < nchunks; ++ch, ++g) {
                    const int s = g % kDStages, u = g / kDStages;
                    if (!wait(bar_full(s), u & 1)) { ok = false; break; }
                    tc::fence_after_sync();
                    const uint32_t aS = sA + (uint32_t)s * 2 * kDAPart;
                    const int ksteps = min(4, (K - ch * KC + Op::KSTEP - 1) / Op::KSTEP);
#pragma unroll
                    for (int s4 = 0; s4 < 4; ++s4) {
                        if (s4 < ksteps) {
                            const uint32_t ka = (uint32_t)s4 * 256, kb = (uint32_t)(ch * 4 + s4) * 256;
                            const uint64_t ah = tc::smem_desc(aS + ka, 1024u), al = tc::smem_desc(aS + kDAPart + ka, 1024u);
                            const uint64_t bh = tc::smem_desc(sB + kb, sboB), bl = tc::smem_desc(sB + bpart + kb, sboB);
                            Op::mma(d, ah, bh, idesc, ch > 0 || s4 > 0);
                            Op::mma(d, ah, bl, idesc, 1);
                            Op::mma(d, al, bh, idesc, 1);
                        }
                    }
                    tc::mma_commit(bar_empty(s));
                    last_bar = bar_empty(s);
                    last_par = u & 1;
                }
                if (!ok) break;
                tc::mma_commit(bar_accf(q));
                last_bar = bar_accf(q);
                last_par = v & 1;
            }
            // copies and MMAs in flight land before the CTA releases its memory (normal limit)
            if (!landed) tc::mbar_wait(bar0, 0);
            if (last_bar) tc::mbar_wait(last_bar, last_par);
        }
        __syncwarp();
    } else if (warp >= 4) {
        // ---------------------------------------------------------------- producers
        const int pt = threadIdx.x - 128;
        float x[GPT][16];                    // one chunk's groups: Re and Im of 8 K values each
        // group i of this thread: box row b, 8-value group kg; lane pairs take the two groups of
        // a pair (kg even, odd) of one box, so a core's 8 rows (4 boxes x Re, Im) fill one store
        auto grp = [&](int i, int& b, int& kg) {
            const int gidx = pt + 128 * i, pair = gidx >> 1;
            b = pair & (kDBoxes - 1);
            kg = 2 * (pair >> 6) + (gidx & 1);
        };
        // per group: the source row (M2M: F_c of the box; L2L: G_P of its parent) and the shift row
        // (L2L), fixed for a whole tile.  The next tile's parents and octants are loaded a tile
        // ahead into registers, so no chunk waits on a dependent lookup.
        const float2* src[GPT];
        const float2* sh[GPT];
        int nxt_p[GPT], nxt_o[GPT];
        auto fetch = [&](int t) {                        // raw lookups of tile t (M2M: box validity only)
#pragma unroll
            for (int i = 0; i < GPT; ++i) {
                int b, kg;
                grp(i, b, kg);
                const int c = t * tile_boxes + b;
                const bool in = t < ntiles && c < a.nbox;
                if (MODE == kDenseM2M) {
                    nxt_p[i] = in ? c : -1;
                    nxt_o[i] = 0;
                } else {
                    nxt_p[i] = in ? a.par[c] : -1;
                    nxt_o[i] = in ? (int)(a.ckey[c] & 7) : 0;
                }
            }
        };
        auto adopt = [&]() {                             // the fetched tile becomes the current one
#pragma unroll
            for (int i = 0; i < GPT; ++i) {
                src[i] = nxt_p[i] >= 0 ? a.in + (int64_t)nxt_p[i] * K : nullptr;
                sh[i] = MODE == kDenseL2L && nxt_p[i] >= 0 ? a.soct + (int64_t)nxt_o[i] * K : nullptr;
            }
        };
        auto load = [&](int ch) {
#pragma unroll
            for (int i = 0; i < GPT; ++i) {
                int b, kg;
                grp(i, b, kg);
                const int k0 = ch * KC + 8 * kg;
                if (src[i] && k0 + 8 <= K) {
                    const float4* s4 = reinterpret_cast<const float4*>(src[i] + k0);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float4 v = s4[j];
                        x[i][2 * j] = v.x; x[i][8 + 2 * j] = v.y; x[i][2 * j + 1] = v.z; x[i][9 + 2 * j] = v.w;
                    }
                    if (MODE == kDenseL2L) {
                        const float4* h4 = reinterpret_cast<const float4*>(sh[i] + k0);
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const float4 w = h4[j];
                            const float gr0 = x[i][2 * j], gi0 = x[i][8 + 2 * j], gr1 = x[i][2 * j + 1], gi1 = x[i][9 + 2 * j];
                            x[i][2 * j] = w.x * gr0 + w.y * gi0;          // conj(S) G
                            x[i][8 + 2 * j] = w.x * gi0 - w.y * gr0;
                            x[i][2 * j + 1] = w.z * gr1 + w.w * gi1;
                            x[i][9 + 2 * j] = w.z * gi1 - w.w * gr1;
                        }
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        float re = 0.f, im = 0.f;
                        if (src[i] && k0 + j < K) {
                            const float2 v = src[i][k0 + j];
                            re = v.x; im = v.y;
                            if (MODE == kDenseL2L) {
                                const float2 w = sh[i][k0 + j];
                                re = w.x * v.x + w.y * v.y;
                                im = w.x * v.y - w.y * v.x;
                            }
                        }
                        x[i][j] = re;
                        x[i][8 + j] = im;
                    }
                }
            }
        };
        bool ok = true;
        int g = 0;
        int t = tfirst, ch = 0;
        fetch(t);
        adopt();
        fetch(t + tstride);
        if (t < ntiles) load(ch);
        while (ok && t < ntiles) {
            const int s = g % kDStages, u = g / kDStages;
            if (u >= 1 && !wait(bar_empty(s), (u - 1) & 1)) { ok = false; break; }
            unsigned char* hi = pA + (size_t)s * 2 * kDAPart;
            unsigned char* lo = hi + kDAPart;
#pragma unroll
            for (int i = 0; i < GPT; ++i) {
                int b, kg;
                grp(i, b, kg);
                float re[8], im[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) { re[j] = x[i][j]; im[j] = x[i][8 + j]; }
                // odd lanes store the Im row first: a store instruction covers rows 0..7 of a core
                if (kg & 1) {
                    GroupStore<Op>::store(hi, lo, 2 * b + 1, 8 * kg, im);
                    GroupStore<Op>::store(hi, lo, 2 * b, 8 * kg, re);
                } else {
                    GroupStore<Op>::store(hi, lo, 2 * b, 8 * kg, re);
                    GroupStore<Op>::store(hi, lo, 2 * b + 1, 8 * kg, im);
                }
            }
            tc::fence_proxy_async();
            tc::mbar_arrive(bar_full(s));
            ++g;
            if (++ch == nchunks) {
                ch = 0;
                t += tstride;
                adopt();
                fetch(t + tstride);
            }
            if (t < ntiles) load(ch);                    // next chunk in flight while this one is consumed
        }
    } else {
        // ---------------------------------------------------------------- epilogue (TMEM lanes 32 warp ..)
        const int et = threadIdx.x;                      // accumulator row
        const int b = et >> 1, odd = et & 1;
        // M2M: the shifts S_o[n0 + 16 qq + c] (o = et / 16, c = et % 16) of every column chunk qq,
        // loaded once (the slice is fixed for the CTA); staged per chunk for the parent sums
        float2 shr[kDMaxChunks];
        if constexpr (MODE == kDenseM2M) {
            const int o = et >> 4, c = et & 15;
#pragma unroll
            for (int qq = 0; qq < kDMaxChunks; ++qq) {
                const int col = 16 * qq + c;
                shr[qq] = col < N ? a.soct[(int64_t)o * a.Nout + n0 + col] : make_float2(0.f, 0.f);
            }
        }
        int it = 0;
        for (int t = tfirst; t < ntiles; t += tstride, ++it) {
            const int q = it & 1, v = it >> 1;
            const int c0 = t * tile_boxes;
            bool row_ok = false;
            float4 gpre[kDL2LChunks][4];                 // L2L: the G values this lane adds to
            if constexpr (MODE == kDenseL2L) {
                row_ok = c0 + b < a.nbox && a.par[c0 + b] >= 0;
                const float2* go = a.out + (int64_t)(c0 + b) * a.Nout + n0;
                // loaded before the accumulator is ready (this CTA alone writes these samples)
#pragma unroll
                for (int qq = 0; qq < kDL2LChunks; ++qq) {
                    const int cs = 16 * qq + 8 * odd;
                    if (row_ok && cs + 8 <= N) {
#pragma unroll
                        for (int j = 0; j < 4; ++j) gpre[qq][j] = reinterpret_cast<const float4*>(go + cs)[j];
                    }
                }
            } else {
                if (et < kDBoxes) {
                    const int c = c0 + et;
                    s_par[et] = c < a.nbox ? a.par[c] : -1;
                    s_oct[et] = c < a.nbox ? (unsigned char)(a.ckey[c] & 7) : 0;
                } else if (et == kDBoxes) {
                    s_prev = c0 > 0 && c0 - 1 < a.nbox ? a.par[c0 - 1] : -1;
                }
            }
            if (et == 0) s_ok = wait(bar_accf(q), v & 1) ? 1 : 0;
            epi_sync();
            if (!s_ok) break;                            // uniform: every epilogue thread read the same flag
            tc::fence_after_sync();
            const uint32_t tl = tmem + (uint32_t)q * accoff + ((uint32_t)(32 * warp) << 16);
            if constexpr (MODE == kDenseM2M) {
                if (warp == 0) {
                    // parents summed here: first child in rows 0 .. 55, compacted in row order, with
                    // their numbers of children
                    auto first = [&](int r) {
                        if (r >= kDAnchor || s_par[r] < 0) return false;
                        return (r == 0 ? s_prev : s_par[r - 1]) != s_par[r];
                    };
                    auto nchild = [&](int r) {
                        int u = 1;
                        while (u < 8 && r + u < kDBoxes && s_par[r + u] == s_par[r]) ++u;
                        return u;
                    };
                    const bool f0 = first(lane), f1 = first(lane + 32);
                    const unsigned m0 = __ballot_sync(0xffffffffu, f0), m1 = __ballot_sync(0xffffffffu, f1);
                    const unsigned below = (1u << lane) - 1u;
                    if (f0) {
                        const int j = __popc(m0 & below);
                        s_plist[j] = lane;
                        s_nch[j] = (unsigned char)nchild(lane);
                    }
                    if (f1) {
                        const int j = __popc(m0) + __popc(m1 & below);
                        s_plist[j] = lane + 32;
                        s_nch[j] = (unsigned char)nchild(lane + 32);
                    }
                    if (lane == 0) s_np = __popc(m0) + __popc(m1);
                }
                epi_sync();                              // the parent list is complete
                const int np = s_np;
#pragma unroll
                for (int qq = 0; qq < kDMaxChunks; ++qq) {
                    if (16 * qq >= Np) break;
                    uint32_t r[16];
                    tc::tmem_ld16(tl + (uint32_t)(16 * qq), r);
                    float4* zr = reinterpret_cast<float4*>(zbuf + et * kDZPitch);
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        zr[j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                            __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
                    s_sh[et >> 4][et & 15] = shr[qq];
                    epi_sync();
                    for (int idx = et; idx < np * 16; idx += 128) {
                        const int j = idx >> 4, cc = idx & 15, col = 16 * qq + cc;
                        if (col >= N) continue;
                        const int r0 = s_plist[j], nch = s_nch[j];
                        float zre[8], zim[8];
                        float2 sv[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) {            // every load before the sums
                            if (u < nch) {
                                zre[u] = zbuf[(2 * (r0 + u)) * kDZPitch + cc];
                                zim[u] = zbuf[(2 * (r0 + u) + 1) * kDZPitch + cc];
                                sv[u] = s_sh[s_oct[r0 + u]][cc];
                            }
                        }
                        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            if (u < nch) {
                                acc.x = fmaf(sv[u].x, zre[u], acc.x);
                                acc.x = fmaf(-sv[u].y, zim[u], acc.x);
                                acc.y = fmaf(sv[u].x, zim[u], acc.y);
                                acc.y = fmaf(sv[u].y, zre[u], acc.y);
                            }
                        }
                        a.out[(int64_t)s_par[r0] * a.Nout + n0 + col] = acc;
                    }
                    epi_sync();                          // the buffers are free for the next columns
                }
            } else {
#pragma unroll
                for (int qq = 0; qq < kDL2LChunks; ++qq) {
                    if (16 * qq >= Np) break;
                    uint32_t r[16];
                    tc::tmem_ld16(tl + (uint32_t)(16 * qq), r);
                    // even lane (Re row): columns 0..7 with the Im parts of its partner; odd lane
                    // (Im row): columns 8..15 with the Re parts of its partner
                    float xr[8], xi[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float send = __uint_as_float(odd ? r[j] : r[8 + j]);
                        const float got = __shfl_xor_sync(0xffffffffu, send, 1);
                        xr[j] = odd ? got : __uint_as_float(r[j]);
                        xi[j] = odd ? __uint_as_float(r[8 + j]) : got;
                    }
                    const int cs = 16 * qq + 8 * odd;
                    if (row_ok && cs < N) {
                        float2* o = a.out + (int64_t)(c0 + b) * a.Nout + n0 + cs;
                        if (cs + 8 <= N) {
                            float4* o4 = reinterpret_cast<float4*>(o);
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                float4 w = gpre[qq][j];
                                w.x += xr[2 * j]; w.y += xi[2 * j]; w.z += xr[2 * j + 1]; w.w += xi[2 * j + 1];
                                o4[j] = w;
                            }
                        } else {
                            for (int j = 0; j < 8 && cs + j < N; ++j) {
                                float2 w = o[j];
                                w.x += xr[j]; w.y += xi[j];
                                o[j] = w;
                            }
                        }
                    }
                }
            }
            tc::fence_before_sync();
            tc::mbar_arrive(bar_acce(q));
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 8) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, ncols);
    }
}

template <typename Op>
DenseShape shape_of(bool m2m, int K, int Nout) {
    return dense_shape<Op>(K, Nout, m2m);
}

template <typename Op>
void launch_dense(const Plan& p, bool m2m, int64_t nbox_c, int K, int Nout, const void* Bm, const int* par,
                  const uint64_t* ckey, const float2* soct, const float2* in, float2* out, cudaStream_t s) {
    const DenseShape d = dense_shape<Op>(K, Nout, m2m);
    if (d.NS == 0) fail(MLFMA_ERR_UNSUPPORTED, "dense map of %d x %d does not fit in shared memory", K, Nout);
    DenseArgs a{};
    a.nbox = (int)nbox_c;
    a.K = K;
    a.Kpad = d.Kpad;
    a.Nout = Nout;
    a.NS = d.NS;
    a.nslices = d.nslices;
    a.ntiles = (int)((nbox_c + (m2m ? kDAnchor : kDBoxes) - 1) / (m2m ? kDAnchor : kDBoxes));
    a.Bm = (const unsigned char*)Bm;
    a.in = in;
    a.out = out;
    a.par = par;
    a.ckey = ckey;
    a.soct = soct;
    a.err = p.dev_err;
    a.wait_first = std::min<long long>(p.wait_first, tc::kWaitLimit);
    int dev = 0, nsm = 0;
    MLFMA_CUDA(cudaGetDevice(&dev));
    MLFMA_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int per_slice = std::max(1, std::min(nsm / d.nslices, a.ntiles));
    const dim3 grid((unsigned)(per_slice * d.nslices));
    if (m2m)
        k_dense_tc<Op, kDenseM2M><<<grid, kDThreads, d.smem, s>>>(a);
    else
        k_dense_tc<Op, kDenseL2L><<<grid, kDThreads, d.smem, s>>>(a);
    MLFMA_LAUNCH_CHECK();
}

template <typename K>
static void allow_dense_smem(K kernel) {
    MLFMA_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDSmemMax));
}

}  // namespace

void prepare_dense_tc() {
    allow_dense_smem(k_dense_tc<SplitTF32, kDenseM2M>);
    allow_dense_smem(k_dense_tc<SplitBF16, kDenseM2M>);
    allow_dense_smem(k_dense_tc<SplitTF32, kDenseL2L>);
    allow_dense_smem(k_dense_tc<SplitBF16, kDenseL2L>);
}

bool dense_tc_fits(const Plan& p, int Kc, int Kp) {
    const bool bf = p.prec == MLFMA_PREC_FP32_BF16X3;
    const DenseShape m = bf ? dense_shape<SplitBF16>(Kc, Kp, true) : dense_shape<SplitTF32>(Kc, Kp, true);
    const DenseShape l = bf ? dense_shape<SplitBF16>(Kp, Kc, false) : dense_shape<SplitTF32>(Kp, Kc, false);
    return m.NS > 0 && l.NS > 0;
}

// bytes of the pre-split slices of a map M [K][Nout] (m2m: the M2M kernel's shared-memory budget)
size_t dense_tc_map_bytes(const Plan& p, bool m2m, int K, int Nout) {
    const bool bf = p.prec == MLFMA_PREC_FP32_BF16X3;
    const DenseShape d = bf ? dense_shape<SplitBF16>(K, Nout, m2m) : dense_shape<SplitTF32>(K, Nout, m2m);
    return (size_t)d.nslices * d.bslice;
}

void presplit_dense_tc(const Plan& p, bool m2m, int K, int Nout, const float* M, void* out, cudaStream_t s) {
    const bool bf = p.prec == MLFMA_PREC_FP32_BF16X3;
    const DenseShape d = bf ? dense_shape<SplitBF16>(K, Nout, m2m) : dense_shape<SplitTF32>(K, Nout, m2m);
    const int64_t tot = (int64_t)d.nslices * d.NS * d.Kpad;
    const unsigned nb = (unsigned)((tot + 255) / 256);
    if (bf)
        k_presplit_dense<SplitBF16><<<nb, 256, 0, s>>>(K, d.Kpad, Nout, d.NS, d.nslices, M, (unsigned char*)out);
    else
        k_presplit_dense<SplitTF32><<<nb, 256, 0, s>>>(K, d.Kpad, Nout, d.NS, d.nslices, M, (unsigned char*)out);
    MLFMA_LAUNCH_CHECK();
}

void launch_dense_m2m_tc(const Plan& p, int64_t nbox_c, int Kc, int Kp, const void* Mtc, const int* par,
                         const uint64_t* ckey, const float2* soct, const float2* Fc, float2* Fp, cudaStream_t s) {
    if (nbox_c <= 0) return;
    if (p.prec == MLFMA_PREC_FP32_BF16X3)
        launch_dense<SplitBF16>(p, true, nbox_c, Kc, Kp, Mtc, par, ckey, soct, Fc, Fp, s);
    else
        launch_dense<SplitTF32>(p, true, nbox_c, Kc, Kp, Mtc, par, ckey, soct, Fc, Fp, s);
}

void launch_dense_l2l_tc(const Plan& p, int64_t nbox_c, int Kp, int Kc, const void* Mtc, const int* par,
                         const uint64_t* ckey, const float2* soct, const float2* Gp, float2* Gc, cudaStream_t s) {
    if (nbox_c <= 0) return;
    if (p.prec == MLFMA_PREC_FP32_BF16X3)
        launch_dense<SplitBF16>(p, false, nbox_c, Kp, Kc, Mtc, par, ckey, soct, Gp, Gc, s);
    else
        launch_dense<SplitTF32>(p, false, nbox_c, Kp, Kc, Mtc, par, ckey, soct, Gp, Gc, s);
}

}  // namespace mlfma
