"""The integer-pipe FP64 adder (csrc/fp64_int.cuh) compiled for the host and
checked bit for bit against the host's IEEE-754 double addition (round to
nearest even) on random bit patterns and on structured cases: equal and
nearby exponents, deep cancellation, subnormals, exact ties, overflow,
signed zeros, infinities and NaNs."""
import os
import subprocess
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1810_11482_b300", "csrc")

DRIVER = r"""
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <cmath>
#define __device__
#define __forceinline__ inline
static inline long long __double_as_longlong(double x) { long long r; memcpy(&r, &x, 8); return r; }
static inline double __longlong_as_double(long long x) { double r; memcpy(&r, &x, 8); return r; }
static inline int __clzll(long long x) { return __builtin_clzll((unsigned long long)x); }
static volatile double g_sink;
static inline double __dadd_rn(double a, double b) { volatile double r = a + b; return r; }
#include "fp64_int.cuh"

static uint64_t s = 0x9E3779B97F4A7C15ull;
static uint64_t rnd() {  /* xorshift64* */
    s ^= s >> 12; s ^= s << 25; s ^= s >> 27; return s * 2685821657736338717ull;
}
static double bits(uint64_t u) { double d; memcpy(&d, &u, 8); return d; }
static uint64_t ubits(double d) { uint64_t u; memcpy(&u, &d, 8); return u; }

static long long bad = 0, total = 0;
static void check(double a, double b) {
    volatile double va = a, vb = b;
    double want = va + vb;
    double got = hxc::k::dadd_int(a, b);
    total++;
    if (std::isnan(want) && std::isnan(got)) return;
    if (ubits(want) != ubits(got)) {
        if (bad < 10) printf("MISMATCH a=%016llx b=%016llx want=%016llx got=%016llx\n",
                             (unsigned long long)ubits(a), (unsigned long long)ubits(b),
                             (unsigned long long)ubits(want), (unsigned long long)ubits(got));
        bad++;
    }
}

int main(int argc, char **argv) {
    long long n = atoll(argv[1]);
    for (long long i = 0; i < n; i++) {
        uint64_t x = rnd(), y = rnd();
        switch (i % 8) {
        case 0: check(bits(x), bits(y)); break;                         /* any patterns */
        case 1: {                                                      /* nearby exponents */
            uint64_t ex = (x >> 52) & 0x7FF, d = y % 70;
            uint64_t ey = ex > d ? ex - d : 0;
            check(bits((x & 0x800FFFFFFFFFFFFFull) | (ex << 52)),
                  bits((y & 0x800FFFFFFFFFFFFFull) | (ey << 52)));
            break; }
        case 2: {                                                      /* cancellation */
            double a = bits((x & 0x3FFFFFFFFFFFFFFFull) | 0x3000000000000000ull);
            uint64_t ua = ubits(a) ^ 0x8000000000000000ull;
            check(a, bits(ua + (int64_t)(y % 64) - 32));
            break; }
        case 3: check(bits(x & 0x801FFFFFFFFFFFFFull), bits(y & 0x801FFFFFFFFFFFFFull)); break; /* subnormal range */
        case 4: {                                                      /* ties: b one half-ulp pattern */
            double a = bits((x & 0x7FEFFFFFFFFFFFFFull) | 0x0010000000000000ull);
            int ea = (int)((ubits(a) >> 52) & 0x7FF);
            int eb = ea - 53; if (eb < 1) eb = 1;
            check(a, bits(((uint64_t)eb << 52) | (y & 0x8000000000000000ull)));
            break; }
        case 5: check(bits((x & 0x000FFFFFFFFFFFFFull) | 0x7FE0000000000000ull),
                      bits((y & 0x000FFFFFFFFFFFFFull) | 0x7FE0000000000000ull)); break; /* overflow */
        case 6: {                                                      /* stencil-like values */
            double a = (double)(x >> 11) * 0x1p-53, b = (double)(y >> 11) * 0x1p-53 * 1e-3;
            check(a, b); check(a, -b); check(-a, b);
            break; }
        default: {                                                     /* specials mixed in */
            const uint64_t sp[] = {0ull, 0x8000000000000000ull, 0x7FF0000000000000ull,
                                   0xFFF0000000000000ull, 0x7FF8000000000001ull, 1ull,
                                   0x8000000000000001ull, 0x0010000000000000ull};
            check(bits(sp[x % 8]), bits(y)); check(bits(x), bits(sp[y % 8]));
            check(bits(sp[x % 8]), bits(sp[y % 8]));
            break; }
        }
    }
    printf("%lld %lld\n", bad, total);
    return bad != 0;
}
"""


def test_dadd_int_matches_ieee_addition():
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.cpp")
        exe = os.path.join(d, "t")
        open(src, "w").write(DRIVER)
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, src,
                               "-o", exe])
        r = subprocess.run([exe, "20000000"], capture_output=True, text=True)
        bad, total = (int(v) for v in r.stdout.strip().splitlines()[-1].split())
        assert bad == 0, r.stdout
        assert total >= 20000000
