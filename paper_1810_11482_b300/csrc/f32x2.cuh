// Paired FP32 arithmetic of sm_100-class GPUs (add.rn.f32x2, fma.rn.f32x2):
// one instruction updates two floats held in a 64-bit register, rounding
// each half exactly as the scalar instruction does, so a kernel may pair
// any two independent scalar evaluations without changing a bit.  (No
// paired multiply here: the code generator was seen to fuse a paired
// multiplication into a following paired subtraction despite the .rn
// modifier, and to fold fma(a, b, -0) with a literal -0 back into such a
// multiplication; a product that must round on its own needs fma with a -0
// that comes from a kernel argument.)
#pragma once

namespace hxc {
namespace k {

typedef unsigned long long f2;  // two floats; the low half comes first in memory

__device__ __forceinline__ f2 pk(float lo, float hi) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float lo_of(f2 v) { return __uint_as_float((unsigned)v); }
__device__ __forceinline__ float hi_of(f2 v) { return __uint_as_float((unsigned)(v >> 32)); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

}  // namespace k
}  // namespace hxc
