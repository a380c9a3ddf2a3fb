// f2.cuh -- packed FP32 pairs (two floats in one 64-bit register) and the
// FP32x2 arithmetic of sm_100-class GPUs: one issue slot per two lanes of work.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace nnqs {

typedef unsigned long long f2;
__device__ __forceinline__ f2 f2_pack(float lo, float hi)
{
    return (f2)__float_as_uint(lo) | ((f2)__float_as_uint(hi) << 32);
}
__device__ __forceinline__ float f2_lo(f2 v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float f2_hi(f2 v) { return __uint_as_float((uint32_t)(v >> 32)); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// one 128-bit shared-memory load as two packed pairs
__device__ __forceinline__ void lds128(const void *p, f2 &a, f2 &b)
{
    const uint32_t addr = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "r"(addr));
}
// the same at a shared-memory address
__device__ __forceinline__ void lds128(uint32_t addr, f2 &a, f2 &b)
{
    asm volatile("ld.shared.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "r"(addr));
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b)
{
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

}  // namespace nnqs
