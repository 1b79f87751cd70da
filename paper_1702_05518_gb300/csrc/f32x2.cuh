// f32x2.cuh -- packed two-lane FP32 arithmetic: two chains' values in one 64-bit register (low
// half: the even chain) and the add/sub/mul/fma .rn.f32x2 instructions, one instruction per pair
// with each lane rounded as the scalar operation would be (lattice3d.cu, which keeps every chain
// of a site in one thread).
#pragma once

#include <cuda_runtime.h>

namespace gmrf {
namespace {

using f2 = unsigned long long;

__device__ __forceinline__ f2 pk(float lo, float hi)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(f2 v, float &lo, float &hi) { asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v)); }
__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b)
{
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
// a * b + c, rounded once per lane
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ f2 splat(float v) { return pk(v, v); }

// Four chain values (two pairs) at p, 16-byte aligned.
__device__ __forceinline__ void ld2x2(const float *p, f2 &a, f2 &b)
{
    const ulonglong2 t = *reinterpret_cast<const ulonglong2 *>(p);
    a = t.x;
    b = t.y;
}
__device__ __forceinline__ void st2x2(float *p, f2 a, f2 b) { *reinterpret_cast<ulonglong2 *>(p) = make_ulonglong2(a, b); }

}  // namespace
}  // namespace gmrf
