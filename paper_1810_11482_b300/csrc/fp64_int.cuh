// IEEE-754 binary64 addition, round to nearest even, on the integer pipe.
//
// B300 executes FP64 at 1/64 of its FP32/INT32 rate, so an FP64-bound
// stencil leaves the integer units idle.  dadd_int computes exactly the
// correctly rounded sum that the FP64 adder returns (the textbook algorithm:
// order the operands by magnitude, align the smaller significand with a
// sticky bit, add or subtract, normalise, round on guard/round/sticky bits),
// so kernels may run any of their additions here and keep every bit of the
// result.  Infinities and NaNs are handed to the FP64 adder.
#pragma once

#include <cstdint>

namespace hxc {
namespace k {

__device__ __forceinline__ double dadd_int(double a, double b) {
    constexpr uint64_t kAbs = 0x7FFFFFFFFFFFFFFFull, kFrac = 0x000FFFFFFFFFFFFFull,
                       kHid = 0x0010000000000000ull, kSign = 0x8000000000000000ull,
                       kInf = 0x7FF0000000000000ull;
    uint64_t ua = (uint64_t)__double_as_longlong(a), ub = (uint64_t)__double_as_longlong(b);
    uint64_t ma = ua & kAbs, mb = ub & kAbs;
    if (ma < mb) {  // |a| >= |b| from here on
        const uint64_t t = ua;
        ua = ub;
        ub = t;
        const uint64_t tm = ma;
        ma = mb;
        mb = tm;
    }
    const int ea = (int)(ma >> 52), eb = (int)(mb >> 52);
    if (ea == 0x7FF) return __dadd_rn(a, b);  // infinity or NaN
    // significands with the hidden bit, 3 extra bits below (guard, round, sticky)
    uint64_t fa = ((ma & kFrac) | (ea ? kHid : 0)) << 3;
    uint64_t fb = ((mb & kFrac) | (eb ? kHid : 0)) << 3;
    const int e1 = ea ? ea : 1, e2 = eb ? eb : 1;  // subnormals share exponent 1
    const int d = e1 - e2;
    if (d >= 60) {
        fb = fb != 0;  // everything is below the sticky position
    } else if (d > 0) {
        const uint64_t lost = fb & ((1ull << d) - 1);
        fb = (fb >> d) | (lost != 0);
    }
    const bool sub = ((ua ^ ub) & kSign) != 0;
    uint64_t f = sub ? fa - fb : fa + fb;
    const uint64_t sign = ua & kSign;
    if (f == 0) return sub ? 0.0 : __longlong_as_double((long long)sign);  // x - x = +0
    int e = e1;
    if (f >> 56) {  // carry out of the addition
        f = (f >> 1) | (f & 1);
        e += 1;
    } else {  // cancellation: bring the leading bit to position 55 (not below e = 1)
        int sh = __clzll((long long)f) - 8;
        if (sh > e - 1) sh = e - 1;
        f <<= sh;
        e -= sh;
    }
    const uint32_t low = (uint32_t)f & 7u;
    f >>= 3;
    if (low > 4u || (low == 4u && (f & 1))) f += 1;  // nearest, ties to even
    // the hidden bit of f (or the carry of the rounding) completes the exponent;
    // e = 1 with no hidden bit encodes a subnormal
    uint64_t r = ((uint64_t)(e - 1) << 52) + f;
    if (r >= kInf) r = kInf;  // overflow rounds to infinity
    return __longlong_as_double((long long)(r | sign));
}

}  // namespace k
}  // namespace hxc
