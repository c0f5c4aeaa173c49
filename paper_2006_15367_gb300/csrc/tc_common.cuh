// Helpers shared by the tensor-core kernels (theta maps and dense level-pair maps): the two
// split operand forms, the canonical no-swizzle K-major shared-memory layout and its matrix
// descriptor, bounded mbarrier waits, bulk copies and tensor-memory loads (inline PTX for
// sm_103a: tcgen05, cp.async.bulk, mbarrier).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace mlfma {
namespace tc {

constexpr long long kWaitLimit = 1ll << 22;  // polls of a bounded wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// The two operand forms: element type in shared memory, the split of an FP32 value into
// hi + lo, the instruction descriptor (D = F32, A and B of the same type, both K-major, N >> 3
// at bit 17, M >> 4 at bit 24), the MMA kind and the K of one MMA (32 bytes of each operand).
struct SplitTF32 {
    using T = float;
    static constexpr int KSTEP = 8;
    __device__ static void split(float x, T& hi, T& lo) {
        hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
        lo = x - hi;
    }
    // hi and lo parts of two consecutive values as 8 bytes each
    __device__ static void split2(float x0, float x1, uint2& hi, uint2& lo) {
        T h0, l0, h1, l1;
        split(x0, h0, l0);
        split(x1, h1, l1);
        hi = make_uint2(__float_as_uint(h0), __float_as_uint(h1));
        lo = make_uint2(__float_as_uint(l0), __float_as_uint(l1));
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
    static constexpr int KSTEP = 16;
    __device__ static void split(float x, T& hi, T& lo) {
        hi = __float2bfloat16_rn(x);
        lo = __float2bfloat16_rn(x - __bfloat162float(hi));
    }
    // hi and lo parts of two consecutive values packed as bf16x2 (first value in the low half)
    __device__ static void split2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
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

// Canonical K-major layout without swizzle for rows of KR elements: core matrices of 8 rows x
// 16 bytes (EPC = 16 / sizeof(T) elements), core (row / 8, k / EPC) at byte ((row / 8) (KR / EPC)
// + k / EPC) 128, row r % 8 at 16 (r % 8).  Leading-dimension offset (next core along K) 128 B,
// stride offset (next 8 rows) KR / EPC * 128 B.  One MMA K-step covers two cores along K (256 B).
template <typename T>
__host__ __device__ __forceinline__ uint32_t core_off_kr(int row, int k, int KR) {
    constexpr int ES = (int)sizeof(T), EPC = 16 / ES;
    return (uint32_t)(((row >> 3) * (KR / EPC) + k / EPC) * 128 + (row & 7) * 16 + (k % EPC) * ES);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);                    // start address
    d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;                       // leading-dimension byte offset
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;                        // stride-dimension byte offset
    d |= (uint64_t)1 << 46;                                             // descriptor version of tcgen05
    return d;                                                           // base offset 0, no swizzle
}

template <typename T> __device__ __forceinline__ void st_part(unsigned char* base, uint32_t off, T v) {
    *reinterpret_cast<T*>(base + off) = v;
}

// true once the phase of the given parity has completed; false after limit polls
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

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count = 1) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

// bulk copy of bytes (16-byte aligned, a multiple of 16) into shared memory, completing on bar
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
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

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

}  // namespace tc
}  // namespace mlfma
