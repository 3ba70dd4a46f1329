// sm_103a primitives for the tensor-core block kernels: mbarriers with bounded
// waits, 2D TMA loads, TMEM allocation, tcgen05 MMA (kind::tf32, one CTA) and
// TMEM loads, and the descriptors they take.  Inline PTX only.
//
// Shared-memory operand layout used throughout (K-major, no swizzle): a tile of
// R rows (the M or N index) by K 32-bit elements is stored as 8-row x 16-byte
// "core matrices"; core matrix (g, kg) -- rows 8g..8g+7, elements 4kg..4kg+3 --
// occupies 128 contiguous bytes (row r at byte 16 (r mod 8)) at byte offset
// (g KG + kg) 128, KG = K / 4.  Its descriptor has leading-dimension byte offset
// (between core matrices adjacent in K) 128 and stride-dimension byte offset
// (between 8-row groups) 128 KG.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------------------
// mbarrier
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// One bounded poll: the thread may be suspended up to about 20 us (the hint) until the
// phase completes, which keeps waiting warps off the issue slots.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(20000u)
        : "memory");
    return ok != 0;
}
// Waits for the phase of the given parity to complete.  Gives up (returns false)
// when *abort becomes nonzero or the global timer passes deadline_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned long long deadline_ns,
                                          volatile int* abort) {
    while (!mbar_try_wait(bar, parity)) {
        if (*abort) return false;
        if (global_ns() > deadline_ns) return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// TMA: one 2D box from global memory into shared memory, completing on an mbarrier
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(map) : "memory");
}

// ---------------------------------------------------------------------------
// tcgen05: tensor memory, MMA, loads
// ---------------------------------------------------------------------------
// Warp-wide.  ncols a power of two >= 32; the TMEM address is written to *dst.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes -> visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle.  The operand is stored
// as 8-row atoms of 8 x 128 bytes (1024 bytes, 1024-aligned), row r of an atom at byte
// 128 r with its 16-byte chunks permuted: logical chunk q at physical chunk q ^ (r & 7)
// (the layout a TMA load with 128-byte swizzle writes).  Atoms along the M/N index are
// 1024 bytes apart; one MMA reads 32 bytes of K from each row, and successive K steps
// inside the 128-byte row advance the start address by 32 bytes.
__device__ __forceinline__ uint64_t desc_kmajor_sw128(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;                      // leading byte offset (unused for this layout): 16 bytes
    d |= (uint64_t)(1024u >> 4) << 32;           // stride byte offset: 1024 between 8-row atoms
    d |= (uint64_t)1 << 46;                      // descriptor version (bits 46-48 = 0b001)
    d |= (uint64_t)2 << 61;                      // 128-byte swizzle
    return d;
}

// Shared-memory matrix descriptor: K-major, no swizzle (layout described above).
__device__ __forceinline__ uint64_t desc_kmajor(uint32_t saddr, uint32_t lbo_bytes, uint32_t sbo_bytes) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo_bytes >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo_bytes >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;                      // descriptor version (bits 46-48 = 0b001)
    return d;                                    // base offset 0, relative LBO, no swizzle
}

// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (TMEM) = A B^T (+ D when accumulate): A M x K and B N x K from shared memory.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         bool accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)accumulate)
        : "memory");
}
// The mbarrier receives one arrival when every MMA this thread issued before has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 TMEM lanes x 16 consecutive 32-bit columns: lane l of the warp gets row (lane base + l).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// TF32 high part as the tensor core reads a 32-bit operand (the low 13 mantissa bits
// ignored), and the remainder x - high rounded to the nearest TF32 value: x = high + low
// to about 2^-22 relative, the rounding of low unbiased.
__device__ __forceinline__ float tf32_low(float x) {
    const float hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
    const uint32_t r = __float_as_uint(x - hi);
    return __uint_as_float((r + 0x1000u) & 0xFFFFE000u);
}

// x = hi + lo with hi = x rounded to the nearest TF32 value (10 explicit mantissa bits)
// and lo = x - hi exact in FP32; the tensor core reads lo to TF32 precision, so
// hi + lo carries about 21 significant bits (the split-operand form of Ootomo and
// Yokota, 2022: products a_hi b_hi + a_hi b_lo + a_lo b_hi).
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
    const uint32_t u = __float_as_uint(x);
    hi = __uint_as_float((u + 0x1000u) & 0xFFFFE000u);
    lo = x - hi;
}

}  // namespace tc
