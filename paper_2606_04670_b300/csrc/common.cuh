// Shared device helpers and the handle layout of liblipfit (sm_103a only).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lipfit.h"

#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ < 1000)
#error "liblipfit is written for sm_103a (Blackwell) only"
#endif

namespace lip {

constexpr int GROUP = 4;          // data points per AoSoA group of the scan layout
constexpr int D_MAX = LIP_D_MAX;
constexpr int TILE_GROUPS_MAX = 64;                     // groups per shared-memory tile
constexpr int PAD_POINTS = GROUP * TILE_GROUPS_MAX;    // capacity is padded to this

// Device-side error bits, OR-ed into the handle's status word.
constexpr unsigned ERRBIT_TIMEOUT = 1u;
constexpr unsigned ERRBIT_NONFINITE = 2u;

// Bounded waits give up after this many nanoseconds of %globaltimer time.
constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;

// ------------------------------------------------------------------ packed FP32

__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 ra, rb, rr;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rr, ra, rb;\n\tmov.b64 {%0, %1}, rr;\n\t}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Three-input min / max (one instruction on sm_100+).  NaN inputs are ignored
// unless all inputs are NaN, which is how padding points drop out of the scan.
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float min2f(float a, float b) {
    float r;
    asm("min.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float max2f(float a, float b) {
    float r;
    asm("max.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// Square roots of two values on the FMA pipe (no special-function unit): the inverse square
// root seeded by Lomont's integer approximation (C. Lomont, "Fast Inverse Square Root",
// 2003: the float with bits 0x5f375a86 - (bits(s) >> 1)), three Newton-Raphson steps
// y <- y (3/2 - (s/2) y^2) in packed f32x2 arithmetic, then s y.  The iteration runs on
// max(s, FLT_MIN), so s = 0 gives exactly 0, a NaN stays NaN, and values below FLT_MIN
// (distances below 1.1e-19) come out within 1.1e-19 of their root.  Relative error a few
// ulps (checked against FP64 in the tests).
__device__ __forceinline__ float2 sqrt_fma2(float2 s) {
    const float2 sc = make_float2(fmaxf(s.x, 1.17549435e-38f), fmaxf(s.y, 1.17549435e-38f));
    float2 y = make_float2(__int_as_float(0x5f375a86 - (__float_as_int(sc.x) >> 1)),
                           __int_as_float(0x5f375a86 - (__float_as_int(sc.y) >> 1)));
    const float2 nh = mul2(sc, make_float2(-0.5f, -0.5f)), th = make_float2(1.5f, 1.5f);
#pragma unroll
    for (int it = 0; it < 3; ++it) y = mul2(y, fma2(nh, mul2(y, y), th));
    return mul2(s, y);
}
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ------------------------------------------------------------ mbarrier + bulk copy

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// 1-D bulk copy global -> shared (TMA), completion signalled on `bar` as tx bytes.
// dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// Wait for phase `parity` of `bar` to complete, giving up after `limit_ns`.  Returns
// false on timeout and records ERRBIT_TIMEOUT in *err.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, unsigned* err,
                                                  unsigned long long limit_ns = WAIT_LIMIT_NS) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 0u && globaltimer() - t0 > limit_ns) {
            if (err) atomicOr(err, ERRBIT_TIMEOUT);
            return false;
        }
    }
}

// -------------------------------------------------------------- orderable keys

__device__ __forceinline__ uint32_t f2ord(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

}  // namespace lip
