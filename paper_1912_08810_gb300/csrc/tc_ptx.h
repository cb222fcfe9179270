// Thin inline-PTX wrappers for the sm_103a features the mixed kernel uses:
// mbarriers with bounded waits, bulk (TMA) copies global -> shared, and the
// tcgen05 tensor-core instructions (TMEM allocation, MMA, commit, loads, fences).
//
// Shared-memory matrix descriptors follow the canonical K-major layout without
// swizzle: a "core matrix" is 8 rows x 16 bytes stored contiguously (128 B); the
// leading byte offset (LBO) is the distance between core matrices adjacent in K,
// the stride byte offset (SBO) the distance between groups of 8 rows.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sse {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---- mbarrier -------------------------------------------------------------------------

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Plain arrival (release semantics at CTA scope): makes this thread's earlier shared-memory
// writes visible to threads that then observe the phase completing.
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase with the given parity to complete; gives up after `limit_ns`
// nanoseconds of wall time and returns false (the caller records the timeout).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 63u && global_timer_ns() - t0 > limit_ns) return false;
    }
}

// The same bounded wait for threads off the critical path: each try lets the thread sleep
// (up to `sleep_ns`) until the phase completes instead of spinning, so that waiting warps
// leave the issue slots of their scheduler to the warps that work.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, uint32_t parity, uint32_t sleep_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(sleep_ns)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded_sleep(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait_sleep(bar, parity, 1000000u)) return true;
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        if (mbar_try_wait_sleep(bar, parity, 1000000u)) return true;
        if (global_timer_ns() - t0 > limit_ns) return false;
    }
}

// Hint: bring the cache line holding `p` (inside a live allocation) into L2.
__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Fire-and-forget atomic add of two floats to global memory (relaxed, no return value).
__device__ __forceinline__ void red_add_f2(float2 *p, float2 v) {
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(v.x), "f"(v.y) : "memory");
}

// Fire-and-forget atomic add of an FP64 pair (two scalar reductions: PTX has no vector
// form of red.add for f64).
__device__ __forceinline__ void red_add_f64x2(double2 *p, double x, double y) {
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(&p->x), "d"(x) : "memory");
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(&p->y), "d"(y) : "memory");
}

// ---- bulk copies (TMA, non-tensor form) ------------------------------------------------

// 1-D bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from global
// to this CTA's shared memory, completing `bytes` transactions on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst_smem, const void *src_gmem, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---- tcgen05 ----------------------------------------------------------------------------

// Allocate `ncols` TMEM columns (power of two >= 32); one full warp executes this and the
// base address is written to shared memory at `holder`.
__device__ __forceinline__ void tmem_alloc(uint32_t *holder, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(holder)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
    d |= (uint64_t)1 << 46;  // fixed constant 0b001 of the tcgen05 descriptor format
    return d;                // base offset 0, relative LBO mode, swizzle mode 0 (none)
}

// Instruction descriptor for kind::f16 with BF16 A/B, FP32 D, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int m, int n) {
    return (1u << 4)                     // D format: F32
           | (1u << 7)                   // A format: BF16
           | (1u << 10)                  // B format: BF16
           | ((uint32_t)(n >> 3) << 17)  // N / 8
           | ((uint32_t)(m >> 4) << 24); // M / 16
}

// D[tmem] (+)= A[smem] * B[smem]^T  (M x N x 16), issued by one thread.
__device__ __forceinline__ void mma_ss(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on `bar` once every tcgen05 operation this thread issued so far has completed.
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 16 lanes x 4 columns per repetition (lane base a multiple of 16 inside the warp's lane
// quarter): thread t gets, for repetition k, r[2k] from lane (base + t / 4) and r[2k + 1]
// from lane (base + 8 + t / 4), both at column (base + 4k + t % 4).
__device__ __forceinline__ void tmem_ld16x128_x4(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.16x128b.x4.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld16x128_x1(uint32_t taddr, uint32_t (&r)[2]) {
    asm volatile("tcgen05.ld.sync.aligned.16x128b.x1.b32 {%0, %1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld16x128_x2(uint32_t taddr, uint32_t (&r)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.16x128b.x2.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
}
// NK repetitions of the 16-lane shape from column `taddr` on: r[2k] and r[2k + 1] as above.
template <int NK>
__device__ __forceinline__ void tmem_ld16x128_reps(uint32_t taddr, uint32_t (&r)[2 * NK]) {
    using R8 = uint32_t(&)[8];
    using R4 = uint32_t(&)[4];
    using R2 = uint32_t(&)[2];
    if constexpr (NK >= 4) tmem_ld16x128_x4(taddr, reinterpret_cast<R8>(r[0]));
    if constexpr (NK == 5) tmem_ld16x128_x1(taddr + 16, reinterpret_cast<R2>(r[8]));
    if constexpr (NK == 2 || NK == 3) tmem_ld16x128_x2(taddr, reinterpret_cast<R4>(r[0]));
    if constexpr (NK == 3) tmem_ld16x128_x1(taddr + 8, reinterpret_cast<R2>(r[4]));
    if constexpr (NK == 1) tmem_ld16x128_x1(taddr, reinterpret_cast<R2>(r[0]));
}

// 32 lanes x 8 columns of 32-bit values: thread t of the warp gets lane (base + t).  The
// destinations are the caller's registers themselves (no copies before the wait).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

// 4 consecutive columns of the warp's 32 lanes; use the values only after tmem_ld_wait().
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
}

// 16 consecutive columns of the warp's 32 lanes; use the values only after tmem_ld_wait().
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
}

// 32 consecutive columns of the warp's 32 lanes (one register per column); the values may
// be used only after tmem_ld_wait().
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// tcgen05.ld fills its destination registers asynchronously: they hold the loaded values
// only after tcgen05.wait::ld, which the compiler does not know.  Passing each loaded
// register through an empty asm statement after the wait makes the compiler treat it as
// written there, so that no use of it (nor a copy) is scheduled above the wait.
template <int N>
__device__ __forceinline__ void tmem_pin(uint32_t (&r)[N]) {
#pragma unroll
    for (int i = 0; i < N; ++i) asm volatile("" : "+r"(r[i]));
}
template <int N>
__device__ __forceinline__ void tmem_pin(float (&v)[N]) {
#pragma unroll
    for (int i = 0; i < N; ++i) asm volatile("" : "+f"(v[i]));
}

// ---- number formats ---------------------------------------------------------------------

// IEEE-754 binary64 -> binary32 with round-to-nearest-even, in integer arithmetic (the
// GB300 FP64 unit is slow, so conversions stay off it).  Values below the binary32
// normal range flush to signed zero; overflow gives infinity; NaN stays NaN.
__device__ __forceinline__ float f64_to_f32(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const uint32_t sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7FFu);
    if (e == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (((hi & 0xFFFFFu) | lo) ? 0x400000u : 0u));
    const int fe = e - 1023 + 127;
    if (fe >= 255) return __uint_as_float(sign | 0x7F800000u);
    if (fe <= 0) return __uint_as_float(sign);
    const uint32_t m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const uint32_t rest = lo & 0x1FFFFFFFu;
    uint32_t r = ((uint32_t)fe << 23) | m;
    if (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) r += 1u;
    return __uint_as_float(sign | r);
}

// binary32 -> binary64 (exact), in integer arithmetic; subnormal inputs flush to zero.
__device__ __forceinline__ double f32_to_f64(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t sign = b & 0x80000000u;
    const uint32_t e = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
    uint32_t hi, lo;
    if (e == 0) {
        hi = sign;
        lo = 0;
    } else if (e == 0xFF) {
        hi = sign | 0x7FF00000u | (m >> 3);
        lo = m << 29;
    } else {
        hi = sign | ((e + 1023u - 127u) << 20) | (m >> 3);
        lo = m << 29;
    }
    return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}

template <typename CT>
__device__ __forceinline__ float2 load_c32(const CT *p);
template <>
__device__ __forceinline__ float2 load_c32<double2>(const double2 *p) {
    const double2 v = __ldg(p);
    return make_float2(f64_to_f32(v.x), f64_to_f32(v.y));
}
template <>
__device__ __forceinline__ float2 load_c32<float2>(const float2 *p) {
    return __ldg(p);
}

// A complex value in shared memory as FP32 (complex128 values rounded to nearest).
__device__ __forceinline__ float2 load_c32_smem(const double2 *p) {
    const double2 v = *p;
    return make_float2(f64_to_f32(v.x), f64_to_f32(v.y));
}
__device__ __forceinline__ float2 load_c32_smem(const float2 *p) { return *p; }

// (hi, lo) split of x into two bf16 values with x ~= hi + lo (both rounded to nearest).
// Returns the pair packed as one word: hi in the low half, lo in the high half.
__device__ __forceinline__ uint32_t split_bf16(float x) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const float r = x - __bfloat162float(h);
    const __nv_bfloat16 l = __float2bfloat16_rn(r);
    return (uint32_t)__bfloat16_as_ushort(h) | ((uint32_t)__bfloat16_as_ushort(l) << 16);
}

}  // namespace tc
}  // namespace sse
