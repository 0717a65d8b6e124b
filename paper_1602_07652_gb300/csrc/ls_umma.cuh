// ls_umma.cuh -- inline-PTX helpers for the fifth-generation tensor cores (tcgen05),
// bulk copies and mbarriers, shared by the kernels that use them (ls_cr_mma.cu,
// ls_unet.cu).  Device code only.
#pragma once

#include <cuda_runtime.h>

namespace umma {

constexpr unsigned long long kWaitNs = 1000000000ull;   // bound of every wait (1 s)

__device__ __forceinline__ unsigned su32(const void* p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool bar_try(unsigned long long* bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// true once phase `parity` of the barrier has completed; false after kWaitNs.  The
// global timer is slow to read (hundreds of ns), so it is read only once the phase was
// found incomplete, and then once every 32 polls.
__device__ __forceinline__ bool bar_wait(unsigned long long* bar, unsigned parity) {
    if (bar_try(bar, parity)) return true;
    const unsigned long long t0 = gtime();
    for (;;) {
#pragma unroll 1
        for (int i = 0; i < 32; ++i)
            if (bar_try(bar, parity)) return true;
        if (gtime() - t0 > kWaitNs) return false;
    }
}
__device__ __forceinline__ void bar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(su32(bar)), "r"(count) : "memory");
}
// byte offset of 16-byte chunk c (0..7) of row `row` in a 128-byte-swizzled K-major atom
__host__ __device__ __forceinline__ unsigned swz16(int row, int c) {
    return (unsigned)row * 128u + (unsigned)((c ^ (row & 7)) << 4);
}
// Shared-memory matrix descriptor of a K-major operand tile in the 128-byte swizzle
// layout: rows of 128 bytes, 8-row groups 1024 bytes apart (stride byte offset),
// descriptor version 1, swizzle mode 2 (128 bytes).  Advancing the start address by
// 32 bytes moves one MMA K-slice along the row.
__device__ __forceinline__ unsigned long long sdesc(unsigned addr) {
    unsigned long long d = 0;
    d |= (unsigned long long)((addr >> 4) & 0x3FFF);
    d |= (unsigned long long)(16 >> 4) << 16;      // leading byte offset (unused when swizzled)
    d |= (unsigned long long)(1024 >> 4) << 32;    // stride byte offset
    d |= 1ull << 46;                                // version
    d |= 2ull << 61;                                // 128-byte swizzle
    return d;
}
// Instruction descriptors: D FP32; A and B K-major, M x N.  kind::tf32: TF32 operands
// (format 2); kind::f16: BF16 operands (format 1).
__host__ __device__ constexpr unsigned idesc(unsigned fmt, int M, int N) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(unsigned dtmem, unsigned long long a, unsigned long long b, unsigned id,
                                         unsigned acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_bf16(unsigned dtmem, unsigned long long a, unsigned long long b, unsigned id,
                                         unsigned acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}
// the barrier's phase completes once every tcgen05 operation issued so far by this thread has
__device__ __forceinline__ void mma_commit(unsigned long long* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(su32(bar))
                 : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     su32(dst)),
                 "l"(src), "r"(bytes), "r"(su32(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_alloc(unsigned* slot, unsigned ncols) {   // one full warp
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols) {   // one full warp
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// 8 consecutive FP32 columns of this warp's 32 TMEM lanes
__device__ __forceinline__ void tmem_ld8(unsigned taddr, float* v) {
    unsigned r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace umma
