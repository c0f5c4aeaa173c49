// Theta maps of the interpolation (Sec. 3.2.2) and anterpolation (Sec. 3.2.4) on the
// 5th-generation tensor cores, split-TF32 (MLFMA_PREC_FP32_TF32X3) or split-BF16
// (MLFMA_PREC_FP32_BF16X3) form:
//
//   out[mi][c][o] = sum_i M[|m|][i][o] in[mi][c][i],   m = mi - Lc
//
// a real matrix applied to complex vectors, one GEMM per Fourier mode.  A CTA takes 64
// boxes of one mode: the A operand has 128 rows (row 2b = Re in[c0+b][.], row 2b+1 = Im),
// the B operand is the mode's map with N <= 256 output rows as K-major rows.  Both are
// split into two parts while staged in shared memory, x = hi + lo, and the product is
// accumulated in FP32 in tensor memory as hi*hi + hi*lo + lo*hi:
//   TF32: hi = x truncated to TF32, lo = x - hi (exact); the dropped lo*lo term is below
//         2^-22 relative, so the result carries FP32-level accuracy (kind::tf32, K = 8 per MMA);
//   BF16: hi = x rounded to BF16, lo = (x - hi) rounded to BF16; hi + lo keeps 16 significant
//         bits, the products are good to about 2^-16 relative (kind::f16 with BF16 operands,
//         K = 16 per MMA, twice the tensor rate of TF32).
// The K dimension is staged in chunks of 128 bytes per row (32 TF32 or 64 BF16 values); one
// thread issues tcgen05.mma (M = 128) and tcgen05.commit signals an mbarrier; the
// accumulator is read back with tcgen05.ld.  Every wait has an iteration limit after which
// the kernel raises the plan's error flag, releases its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"

namespace mlfma {

namespace {

constexpr int kTcBoxes = 64;                 // boxes per CTA (A rows 2b, 2b + 1)
constexpr int kTcM = 128;                    // MMA M
constexpr int kTcRowBytes = 128;             // bytes of one operand row per staged K chunk (4 MMA K-steps)
constexpr int kTcMaxN = 256;                 // output rows per CTA (MMA N <= 256)
constexpr int kTcThreads = 128;
constexpr uint32_t kABytes = kTcM * kTcRowBytes;          // one part of the A chunk (16 KB)
constexpr uint32_t kBBytesMax = kTcMaxN * kTcRowBytes;    // one part of the widest B chunk (32 KB)
constexpr size_t kTcSmemMax = 2 * (size_t)kABytes + 2 * (size_t)kBBytesMax;   // 96 KB
constexpr long long kWaitLimit = 1ll << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// The two operand forms: element type in shared memory, K elements per chunk, the split of an
// FP32 value into hi + lo, the instruction descriptor (D = F32, A and B of the same type, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24) and the MMA kind.
struct SplitTF32 {
    using T = float;
    static constexpr int KC = kTcRowBytes / 4;       // 32
    __device__ static void split(float x, T& hi, T& lo) {
        hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
        lo = x - hi;
    }
    __device__ static uint32_t idesc(int M, int N) {
        return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
    }
    __device__ static void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    }
};

struct SplitBF16 {
    using T = __nv_bfloat16;
    static constexpr int KC = kTcRowBytes / 2;       // 64
    __device__ static void split(float x, T& hi, T& lo) {
        hi = __float2bfloat16_rn(x);
        lo = __float2bfloat16_rn(x - __bfloat162float(hi));
    }
    __device__ static uint32_t idesc(int M, int N) {
        return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
    }
    __device__ static void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    }
};

// Canonical K-major layout without swizzle: core matrices of 8 rows x 16 bytes (EPC = 16 /
// sizeof(T) elements), core (row / 8, k / EPC) at byte ((row / 8) (KC / EPC) + k / EPC) 128, row
// r % 8 at 16 (r % 8).  Leading-dimension offset (next core along K) 128 B, stride offset (next
// 8 rows) KC / EPC * 128 = 1024 B for both forms.
template <typename Op>
__device__ __forceinline__ uint32_t core_off(int row, int k) {
    constexpr int ES = (int)sizeof(typename Op::T), EPC = 16 / ES;
    return (uint32_t)(((row >> 3) * (Op::KC / EPC) + k / EPC) * 128 + (row & 7) * 16 + (k % EPC) * ES);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);                    // start address
    d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;                       // leading-dimension byte offset
    d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 32;                      // stride-dimension byte offset
    d |= (uint64_t)1 << 46;                                             // descriptor version of tcgen05
    return d;                                                           // base offset 0, no swizzle
}

template <typename T> __device__ __forceinline__ void st_part(unsigned char* base, uint32_t off, T v) {
    *reinterpret_cast<T*>(base + off) = v;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, long long limit = kWaitLimit) {
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

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// Npmax: the MMA N of the widest tile of the launch (sizes the B region of shared memory)
template <typename Op>
__global__ void __launch_bounds__(kTcThreads, 1) k_theta_map_tc(int nbox, int Lc, int nin, int nout, int Npmax,
                                                                const float* __restrict__ Mt, const float2* __restrict__ in,
                                                                float2* __restrict__ out, int* __restrict__ err,
                                                                long long wait_first) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t s_taddr;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mi = blockIdx.z, m = abs(mi - Lc);
    const int c0 = blockIdx.x * kTcBoxes;
    const int n0 = blockIdx.y * kTcMaxN;
    const int N = min(kTcMaxN, nout - n0);
    const int Np = (N + 15) & ~15;                                      // MMA N: multiple of 16 for M = 128
    const uint32_t ncols = Np <= 32 ? 32u : Np <= 64 ? 64u : Np <= 128 ? 128u : 256u;
    constexpr int KC = Op::KC;
    using T = typename Op::T;
    const uint32_t bbytes = (uint32_t)Npmax * kTcRowBytes;            // one part of the B chunk
    // plain stores (no compiler barrier between them, so the global loads of the staging
    // loops overlap); the async-proxy fence before the MMAs orders them
    unsigned char* pA[2] = {smem_raw, smem_raw + kABytes};
    unsigned char* pB[2] = {smem_raw + 2 * kABytes, smem_raw + 2 * kABytes + bbytes};
    const uint32_t sA[2] = {smem_u32(pA[0]), smem_u32(pA[1])};
    const uint32_t sB[2] = {smem_u32(pB[0]), smem_u32(pB[1])};
    const uint32_t bar = smem_u32(&mbar);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_taddr)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = s_taddr;

    const float* Mm = Mt + (int64_t)m * nin * nout;
    const float2* inm = in + (int64_t)mi * nbox * nin;
    const uint32_t idesc = Op::idesc(kTcM, Np);
    uint32_t phase = 0;
    bool ok = true;
    bool issued = false;                                                // MMAs committed but not yet waited for
    const int nchunks = (nin + KC - 1) / KC;
    for (int ch = 0; ch < nchunks && ok; ++ch) {
        const int k0 = ch * KC;
        // A: a warp stores 4 boxes x 8 columns, so its 32 stores of one part cover the banks
        // (row mod 8, k mod 4) at most twice; reads are 4 runs of 8 contiguous samples.  Each
        // thread issues its kAPer loads before any store.
        {
            constexpr int kAPer = kTcBoxes * KC / kTcThreads;
            float2 va[kAPer];
#pragma unroll
            for (int it = 0; it < kAPer; ++it) {
                const int idx = threadIdx.x + it * kTcThreads;
                const int w = idx >> 5, l = idx & 31;
                const int b = (w & 15) * 4 + (l >> 3), k = (w >> 4) * 8 + (l & 7);
                va[it] = (c0 + b < nbox && k0 + k < nin) ? inm[(int64_t)(c0 + b) * nin + k0 + k] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int it = 0; it < kAPer; ++it) {
                const int idx = threadIdx.x + it * kTcThreads;
                const int w = idx >> 5, l = idx & 31;
                const int b = (w & 15) * 4 + (l >> 3), k = (w >> 4) * 8 + (l & 7);
                T h, lo;
                Op::split(va[it].x, h, lo);
                st_part(pA[0], core_off<Op>(2 * b, k), h);
                st_part(pA[1], core_off<Op>(2 * b, k), lo);
                Op::split(va[it].y, h, lo);
                st_part(pA[0], core_off<Op>(2 * b + 1, k), h);
                st_part(pA[1], core_off<Op>(2 * b + 1, k), lo);
            }
        }
        // B: output row n, column k, B[n][k] = M[|m|][k0 + k][n0 + n]; a warp stores 8 rows x 4
        // columns (all 32 banks once); reads are 4 runs of 8 contiguous entries, issued in
        // batches of kBBatch per thread
        {
            constexpr int kBBatch = 8;
            const int ng = Np >> 3;
            const int tot = Np * KC;                         // a multiple of kTcThreads * kBBatch / 2
            for (int base = 0; base < tot; base += kTcThreads * kBBatch) {
                float vb[kBBatch];
#pragma unroll
                for (int it = 0; it < kBBatch; ++it) {
                    const int idx = base + threadIdx.x + it * kTcThreads;
                    const int w = idx >> 5, l = idx & 31;
                    const int kq = w / ng, nq = w - kq * ng;
                    const int n = nq * 8 + (l >> 2), k = kq * 4 + (l & 3);
                    vb[it] = (idx < tot && n < N && k0 + k < nin) ? Mm[(int64_t)(k0 + k) * nout + n0 + n] : 0.f;
                }
#pragma unroll
                for (int it = 0; it < kBBatch; ++it) {
                    const int idx = base + threadIdx.x + it * kTcThreads;
                    if (idx >= tot) break;
                    const int w = idx >> 5, l = idx & 31;
                    const int kq = w / ng, nq = w - kq * ng;
                    const int n = nq * 8 + (l >> 2), k = kq * 4 + (l & 3);
                    T h, lo;
                    Op::split(vb[it], h, lo);
                    st_part(pB[0], core_off<Op>(n, k), h);
                    st_part(pB[1], core_off<Op>(n, k), lo);
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const uint32_t ko = (uint32_t)s * 256;          // one MMA K-step: two 16-byte cores along K
                Op::mma(tmem, smem_desc(sA[0] + ko), smem_desc(sB[0] + ko), idesc, ch > 0 || s > 0);
                Op::mma(tmem, smem_desc(sA[0] + ko), smem_desc(sB[1] + ko), idesc, 1);
                Op::mma(tmem, smem_desc(sA[1] + ko), smem_desc(sB[0] + ko), idesc, 1);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                         : "memory");
        }
        issued = true;
        // the MMAs read the staged chunk: wait before it is overwritten (and before the epilogue)
        ok = __syncthreads_and(mbar_wait(bar, phase, wait_first));   // one decision for the whole CTA
        issued = !ok;
        phase ^= 1;
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (ok) {
        const int row = 32 * warp + lane, b = row >> 1;
        const uint32_t tl = tmem + ((uint32_t)(32 * warp) << 16);
        for (int col0 = 0; col0 < Np; col0 += 16) {
            uint32_t r[16];
            tmem_ld16(tl + (uint32_t)col0, r);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float v = __uint_as_float(r[j]);
                const float w = __shfl_xor_sync(0xffffffffu, v, 1);      // the other part of the same box
                const int n = col0 + j;
                if (!(row & 1) && c0 + b < nbox && n < N)
                    out[((int64_t)mi * nbox + c0 + b) * nout + n0 + n] = make_float2(v, w);
            }
        }
    } else {
        if (threadIdx.x == 0) atomicExch(err, 1);
        if (issued) mbar_wait(bar, phase ^ 1);        // let the MMAs in flight finish (bounded, normal limit)
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols) : "memory");
}

}  // namespace

void prepare_theta_tc() {
    MLFMA_CUDA(cudaFuncSetAttribute(k_theta_map_tc<SplitTF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kTcSmemMax));
    MLFMA_CUDA(cudaFuncSetAttribute(k_theta_map_tc<SplitBF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kTcSmemMax));
}

void launch_theta_map_tc(const Plan& p, int64_t nbox, int Lc, int nin, int nout, const float* M, const float2* in,
                         float2* out, cudaStream_t s) {
    const int nm = 2 * Lc + 1;
    const dim3 grid((unsigned)((nbox + kTcBoxes - 1) / kTcBoxes), (unsigned)((nout + kTcMaxN - 1) / kTcMaxN), (unsigned)nm);
    const int Npmax = ((std::min(nout, kTcMaxN) + 15) / 16) * 16;
    const size_t smem = 2 * (size_t)kABytes + 2 * (size_t)Npmax * kTcRowBytes;
    const long long wf = std::min<long long>(p.wait_first, kWaitLimit);
    if (p.prec == MLFMA_PREC_FP32_BF16X3)
        k_theta_map_tc<SplitBF16><<<grid, kTcThreads, smem, s>>>((int)nbox, Lc, nin, nout, Npmax, M, in, out, p.dev_err, wf);
    else
        k_theta_map_tc<SplitTF32><<<grid, kTcThreads, smem, s>>>((int)nbox, Lc, nin, nout, Npmax, M, in, out, p.dev_err, wf);
    MLFMA_LAUNCH_CHECK();
}

}  // namespace mlfma
