// Theta maps of the interpolation (Sec. 3.2.2) and anterpolation (Sec. 3.2.4) on the
// 5th-generation tensor cores, split-TF32 (MLFMA_PREC_FP32_TF32X3) or split-BF16
// (MLFMA_PREC_FP32_BF16X3) form:
//
//   out[mi][c][o] = sum_i M[|m|][i][o] in[mi][c][i],   m = mi - Lc
//
// a real matrix applied to complex vectors, one GEMM per Fourier mode.  A CTA takes 64
// boxes of one mode: the A operand has 128 rows (row 2b = Re in[c0+b][.], row 2b+1 = Im),
// the B operand is the mode's map with N <= 256 output rows as K-major rows.  Both are
// split into two parts, x = hi + lo, and the product is accumulated in FP32 in tensor
// memory as hi*hi + hi*lo + lo*hi:
//   TF32: hi = x truncated to TF32, lo = x - hi (exact); the dropped lo*lo term is below
//         2^-22 relative, so the result carries FP32-level accuracy (kind::tf32, K = 8 per MMA);
//   BF16: hi = x rounded to BF16, lo = (x - hi) rounded to BF16; hi + lo keeps 16 significant
//         bits, the products are good to about 2^-16 relative (kind::f16 with BF16 operands,
//         K = 16 per MMA, twice the tensor rate of TF32).
// The maps are constants of the plan: they are split once at plan creation into blocks laid
// out exactly as the MMA reads them from shared memory (one block per mode, output tile and K
// chunk), so each chunk of B is one bulk copy (cp.async.bulk, completion on an mbarrier).  The
// A chunk (spectral samples written by the previous kernel) is loaded into registers one chunk
// ahead, split and stored by all 256 threads.  Two stages of shared memory alternate: while the
// tensor cores run the MMAs of chunk c, the threads stage chunk c + 1 and the bulk copy of its B
// block is in flight.  The K dimension is staged in chunks of 128 bytes per row (32 TF32 or 64
// BF16 values, four MMA K-steps); one thread issues tcgen05.mma (M = 128) and tcgen05.commit
// signals the stage's mbarrier; the accumulator is read back with tcgen05.ld and written
// through shared memory as whole output rows.  Every wait has an iteration limit after which the
// kernel raises the plan's error flag, waits (normal limit) for its copies and MMAs in flight,
// releases its tensor memory and returns.
#include <algorithm>

#include "common.cuh"
#include "tc_common.cuh"

namespace mlfma {

namespace {

constexpr int kTcBoxes = 64;                 // boxes per CTA (A rows 2b, 2b + 1)
constexpr int kTcM = 128;                    // MMA M
constexpr int kTcRowBytes = 128;             // bytes of one operand row per staged K chunk (4 MMA K-steps)
constexpr int kTcMaxN = 256;                 // output rows per CTA (MMA N <= 256)
constexpr int kTcThreads = 256;
constexpr uint32_t kABytes = kTcM * kTcRowBytes;          // one part of the A chunk (16 KB)
constexpr uint32_t kBBytesMax = kTcMaxN * kTcRowBytes;    // one part of the widest B chunk (32 KB)
// two stages of (A hi, A lo, B hi, B lo): 192 KB at the widest B
constexpr size_t kTcSmemMax = 2 * (2 * (size_t)kABytes + 2 * (size_t)kBBytesMax);
using tc::mbar_init;
using tc::mbar_wait;
using tc::SplitBF16;
using tc::SplitTF32;
using tc::smem_u32;
using tc::st_part;
using tc::tmem_ld16;
constexpr long long kWaitLimit = tc::kWaitLimit;

// K elements of one staged chunk row (kTcRowBytes)
template <typename Op> struct Chunk {
    static constexpr int KC = kTcRowBytes / (int)sizeof(typename Op::T);
};

template <typename Op>
__device__ __forceinline__ uint32_t core_off(int row, int k) {
    return tc::core_off_kr<typename Op::T>(row, k, Chunk<Op>::KC);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) { return tc::smem_desc(addr, 1024u); }

// bulk copy of one pre-split B block (both parts) into shared memory, completing on bar
__device__ __forceinline__ void bulk_b(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    tc::bulk_load(dst, src, bytes, bar);
}

// Pre-split map blocks: for mode m, output tile t (kTcMaxN rows) and K chunk ch, a block of two
// parts [hi, lo], each Npmax rows x kTcRowBytes in the canonical K-major core layout, holding
// B[n][k] = M[m][k0 + k][n0 + n] (zero outside nin x nout).  One thread per element.
template <typename Op>
__global__ void k_presplit_map(int nmaps, int nin, int nout, int Npmax, int ntiles, int nchunks,
                               const float* __restrict__ M, unsigned char* __restrict__ out) {
    constexpr int KC = Chunk<Op>::KC;
    using T = typename Op::T;
    const int64_t per_block = (int64_t)Npmax * KC;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nmaps * ntiles * nchunks * per_block) return;
    const int64_t blk = idx / per_block;
    const int e = (int)(idx - blk * per_block);
    const int n = e / KC, k = e % KC;
    const int ch = (int)(blk % nchunks);
    const int t = (int)((blk / nchunks) % ntiles);
    const int m = (int)(blk / ((int64_t)nchunks * ntiles));
    const int gn = t * kTcMaxN + n, gk = ch * KC + k;
    const int N = min(kTcMaxN, nout - t * kTcMaxN);
    const float v = (n < N && gk < nin) ? M[((int64_t)m * nin + gk) * nout + gn] : 0.f;
    T h, lo;
    Op::split(v, h, lo);
    unsigned char* base = out + blk * 2 * (int64_t)Npmax * kTcRowBytes;
    st_part(base, core_off<Op>(n, k), h);
    st_part(base + (int64_t)Npmax * kTcRowBytes, core_off<Op>(n, k), lo);
}

// Npmax: the MMA N of the widest output tile (sizes the B stages and the map blocks)
template <typename Op>
__global__ void __launch_bounds__(kTcThreads, 1) k_theta_map_tc(int nbox, int Lc, int nin, int nout, int Npmax, int ntiles,
                                                                int nchunks, const unsigned char* __restrict__ Mtc,
                                                                const float2* __restrict__ in, float2* __restrict__ out,
                                                                int* __restrict__ err, long long wait_first) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t s_bar[4];       // [0, 1]: B block of stage s landed; [2, 3]: MMAs of stage s done
    __shared__ uint32_t s_taddr;
    constexpr int KC = Chunk<Op>::KC;
    using T = typename Op::T;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mi = blockIdx.z, m = abs(mi - Lc);
    const int c0 = blockIdx.x * kTcBoxes;
    const int tile = blockIdx.y;
    const int n0 = tile * kTcMaxN;
    const int N = min(kTcMaxN, nout - n0);
    const int Np = (N + 15) & ~15;                                      // MMA N: multiple of 16 for M = 128
    const uint32_t ncols = Np <= 32 ? 32u : Np <= 64 ? 64u : Np <= 128 ? 128u : 256u;
    const uint32_t bbytes = (uint32_t)Npmax * kTcRowBytes;            // one part of a B block
    const uint32_t stage_bytes = 2 * kABytes + 2 * bbytes;
    // stage q at smem_raw + q stage_bytes: A hi, A lo, B hi, B lo
    const uint32_t s_base = smem_u32(smem_raw);
    const uint32_t bar0 = smem_u32(&s_bar[0]);
    auto pS = [&](int q) { return smem_raw + q * stage_bytes; };
    auto sS = [&](int q) { return s_base + q * stage_bytes; };
    auto bar_b = [&](int q) { return bar0 + 8u * q; };
    auto bar_m = [&](int q) { return bar0 + 16u + 8u * q; };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_taddr)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int q = 0; q < 4; ++q) mbar_init(bar0 + 8u * q);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = s_taddr;

    const int64_t blk0 = ((int64_t)m * ntiles + tile) * nchunks;    // first map block of this CTA
    const unsigned char* Mblk = Mtc + blk0 * 2 * (int64_t)bbytes;
    const float2* inm = in + (int64_t)mi * nbox * nin;
    const uint32_t idesc = Op::idesc(kTcM, Np);
    // A: a warp stores 4 boxes x 8 columns (each part's 32 stores cover the banks at most twice);
    // its reads are 4 runs of 8 contiguous samples
    constexpr int kAPer = kTcBoxes * KC / kTcThreads;
    float2 va[kAPer];
    auto load_a = [&](int k0) {
#pragma unroll
        for (int it = 0; it < kAPer; ++it) {
            const int idx = threadIdx.x + it * kTcThreads;
            const int w = idx >> 5, l = idx & 31;
            const int b = (w & 15) * 4 + (l >> 3), k = (w >> 4) * 8 + (l & 7);
            va[it] = (c0 + b < nbox && k0 + k < nin) ? inm[(int64_t)(c0 + b) * nin + k0 + k] : make_float2(0.f, 0.f);
        }
    };
    auto store_a = [&](unsigned char* aS) {
#pragma unroll
        for (int it = 0; it < kAPer; ++it) {
            const int idx = threadIdx.x + it * kTcThreads;
            const int w = idx >> 5, l = idx & 31;
            const int b = (w & 15) * 4 + (l >> 3), k = (w >> 4) * 8 + (l & 7);
            T h, lo;
            Op::split(va[it].x, h, lo);
            st_part(aS, core_off<Op>(2 * b, k), h);
            st_part(aS + kABytes, core_off<Op>(2 * b, k), lo);
            Op::split(va[it].y, h, lo);
            st_part(aS, core_off<Op>(2 * b + 1, k), h);
            st_part(aS + kABytes, core_off<Op>(2 * b + 1, k), lo);
        }
    };

    int last_bulk = -1, last_commit = -1;                             // chunks issued (thread 0's view)
    bool ok = true;
    if (threadIdx.x == 0) {
        bulk_b(sS(0) + 2 * kABytes, Mblk, 2 * bbytes, bar_b(0));
        last_bulk = 0;
    }
    load_a(0);
    for (int ch = 0; ch < nchunks; ++ch) {
        const int st = ch & 1;
        // the stage was read by the MMAs of chunk ch - 2: wait for them before overwriting A
        if (ch >= 2 && !mbar_wait(bar_m(st), ((ch - 2) >> 1) & 1, wait_first)) ok = false;
        if (ok) store_a(pS(st));
        if (ch + 1 < nchunks) load_a((ch + 1) * KC);                  // in flight while the MMAs run
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        if (!__syncthreads_and(ok)) break;
        if (threadIdx.x == 0) {
            bool t_ok = mbar_wait(bar_b(st), (ch >> 1) & 1, wait_first);
            if (t_ok) {
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t a0 = sS(st), b0 = sS(st) + 2 * kABytes;
                // K-steps of this chunk holding samples (the last chunk's zero tail is skipped)
                const int ksteps = min(4, (nin - ch * KC + Op::KSTEP - 1) / Op::KSTEP);
#pragma unroll
                for (int s4 = 0; s4 < 4; ++s4) {
                    if (s4 < ksteps) {
                        const uint32_t ko = (uint32_t)s4 * 256;         // one MMA K-step: two 16-byte cores along K
                        Op::mma(tmem, smem_desc(a0 + ko), smem_desc(b0 + ko), idesc, ch > 0 || s4 > 0);
                        Op::mma(tmem, smem_desc(a0 + ko), smem_desc(b0 + bbytes + ko), idesc, 1);
                        Op::mma(tmem, smem_desc(a0 + kABytes + ko), smem_desc(b0 + ko), idesc, 1);
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                                 bar_m(st))
                             : "memory");
                last_commit = ch;
                // B of chunk ch + 1 goes to the other stage once the MMAs of chunk ch - 1 are done
                if (ch + 1 < nchunks) {
                    const int s1 = (ch + 1) & 1;
                    if (ch >= 1) t_ok = mbar_wait(bar_m(s1), ((ch - 1) >> 1) & 1, wait_first);
                    if (t_ok) {
                        bulk_b(sS(s1) + 2 * kABytes, Mblk + (int64_t)(ch + 1) * 2 * bbytes, 2 * bbytes, bar_b(s1));
                        last_bulk = ch + 1;
                    }
                }
            }
            if (!t_ok) ok = false;
        }
        // thread 0's outcome reaches every thread at the next barrier
    }
    ok = __syncthreads_and(ok);
    if (ok && threadIdx.x == 0 && !mbar_wait(bar_m((nchunks - 1) & 1), ((nchunks - 1) >> 1) & 1, wait_first)) ok = false;
    ok = __syncthreads_and(ok);
    if (!ok) {
        if (threadIdx.x == 0) {
            atomicExch(err, 1);
            // normal limit: the copies and MMAs in flight land before the shared memory is released
            if (last_bulk >= 0) mbar_wait(bar_b(last_bulk & 1), (last_bulk >> 1) & 1);
            if (last_commit >= 0) mbar_wait(bar_m(last_commit & 1), (last_commit >> 1) & 1);
        }
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        // accumulator rows 2b (Re) and 2b + 1 (Im) -> tile[b][n] (complex), then whole rows out
        float2* tileS = reinterpret_cast<float2*>(smem_raw);           // [64][Np + 1], stages are free now
        const int pitch = Np + 1;
        if (warp < 4) {
            const int row = 32 * warp + lane, b = row >> 1;
            const uint32_t tl = tmem + ((uint32_t)(32 * warp) << 16);
            for (int col0 = 0; col0 < Np; col0 += 16) {
                uint32_t r[16];
                tmem_ld16(tl + (uint32_t)col0, r);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float v = __uint_as_float(r[j]);
                    const float w = __shfl_xor_sync(0xffffffffu, v, 1);  // the other part of the same box
                    if (!(row & 1)) tileS[b * pitch + col0 + j] = make_float2(v, w);
                }
            }
        }
        __syncthreads();
        const int nb = min(kTcBoxes, nbox - c0);
        for (int idx = threadIdx.x; idx < nb * N; idx += kTcThreads) {
            const int b = idx / N, n = idx - b * N;
            out[((int64_t)mi * nbox + c0 + b) * nout + n0 + n] = tileS[b * pitch + n];
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols) : "memory");
}

struct TcShape {
    int Npmax, ntiles, nchunks;
};

template <typename Op>
TcShape tc_shape(int nin, int nout) {
    TcShape t;
    t.Npmax = ((std::min(nout, kTcMaxN) + 15) / 16) * 16;
    t.ntiles = (nout + kTcMaxN - 1) / kTcMaxN;
    t.nchunks = (nin + Chunk<Op>::KC - 1) / Chunk<Op>::KC;
    return t;
}

}  // namespace

void prepare_theta_tc() {
    MLFMA_CUDA(cudaFuncSetAttribute(k_theta_map_tc<SplitTF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kTcSmemMax));
    MLFMA_CUDA(cudaFuncSetAttribute(k_theta_map_tc<SplitBF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kTcSmemMax));
}

// bytes of the pre-split blocks of nmaps maps of nin x nout
size_t theta_tc_map_bytes(const Plan& p, int nmaps, int nin, int nout) {
    const TcShape t = p.prec == MLFMA_PREC_FP32_BF16X3 ? tc_shape<SplitBF16>(nin, nout) : tc_shape<SplitTF32>(nin, nout);
    return (size_t)nmaps * t.ntiles * t.nchunks * 2 * (size_t)t.Npmax * kTcRowBytes;
}

void presplit_theta_tc(const Plan& p, int nmaps, int nin, int nout, const float* M, void* out, cudaStream_t s) {
    const bool bf = p.prec == MLFMA_PREC_FP32_BF16X3;
    const TcShape t = bf ? tc_shape<SplitBF16>(nin, nout) : tc_shape<SplitTF32>(nin, nout);
    const int KC = bf ? Chunk<SplitBF16>::KC : Chunk<SplitTF32>::KC;
    const int64_t tot = (int64_t)nmaps * t.ntiles * t.nchunks * t.Npmax * KC;
    const unsigned nb = (unsigned)((tot + 255) / 256);
    if (bf)
        k_presplit_map<SplitBF16><<<nb, 256, 0, s>>>(nmaps, nin, nout, t.Npmax, t.ntiles, t.nchunks, M, (unsigned char*)out);
    else
        k_presplit_map<SplitTF32><<<nb, 256, 0, s>>>(nmaps, nin, nout, t.Npmax, t.ntiles, t.nchunks, M, (unsigned char*)out);
    MLFMA_LAUNCH_CHECK();
}

void launch_theta_map_tc(const Plan& p, int64_t nbox, int Lc, int nin, int nout, const void* Mtc, const float2* in,
                         float2* out, cudaStream_t s) {
    const int nm = 2 * Lc + 1;
    const bool bf = p.prec == MLFMA_PREC_FP32_BF16X3;
    const TcShape t = bf ? tc_shape<SplitBF16>(nin, nout) : tc_shape<SplitTF32>(nin, nout);
    const dim3 grid((unsigned)((nbox + kTcBoxes - 1) / kTcBoxes), (unsigned)t.ntiles, (unsigned)nm);
    // two stages; the output tile [64][Np + 1] complex reuses them
    const size_t stages = 2 * (2 * (size_t)kABytes + 2 * (size_t)t.Npmax * kTcRowBytes);
    const size_t smem = std::max(stages, (size_t)kTcBoxes * (t.Npmax + 1) * sizeof(float2));
    const long long wf = std::min<long long>(p.wait_first, kWaitLimit);
    const unsigned char* M = (const unsigned char*)Mtc;
    if (bf)
        k_theta_map_tc<SplitBF16><<<grid, kTcThreads, smem, s>>>((int)nbox, Lc, nin, nout, t.Npmax, t.ntiles, t.nchunks, M,
                                                                 in, out, p.dev_err, wf);
    else
        k_theta_map_tc<SplitTF32><<<grid, kTcThreads, smem, s>>>((int)nbox, Lc, nin, nout, t.Npmax, t.ntiles, t.nchunks, M,
                                                                 in, out, p.dev_err, wf);
    MLFMA_LAUNCH_CHECK();
}

}  // namespace mlfma
