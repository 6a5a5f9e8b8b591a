// Step schedule of the 2D FTCS runs (host side).
//
// FTCS is linear: u_{n+1} = (1 - 4r) u_n + r s(u_n), with s the sum of the
// four neighbours, = r ((1 - 4r)/r u_n + s(u_n)).  A run therefore carries
// the field scaled by r^-m after m steps, v = u_n / r^m, and advances it
// with one FMA after the neighbour sum (v' = fma((1 - 4r)/r, v, s(v)), a
// "scaled" step: 3 FP64 operations per point instead of 4); a "closing"
// step takes the scaled field back to true values,
// u_{n+1} = fma(r^(m+1), s(v), ((1 - 4r) r^m) v).
//
// The steps of a run are issued in intervals (between snapshots, or of at
// most 100 steps without them; a captured graph holds one interval).  Each
// interval is cut into groups of at most M + 1 steps: a group's last step
// closes, the others are scaled, so the field is true at every interval end
// (snapshots, graph boundaries, the result).  A step's kind and
// coefficients depend only on its index in its interval, which keeps the
// bits independent of tiling, mode and graph replay.
//
// M bounds the growth of the scaled field: for 0 < r <= 1/4 the scaled
// step's coefficients (1 - 4r)/r and four 1s are non-negative and sum to
// 1/r, so |v| grows by at most 1/r per step; M is the largest m with
// r^-m <= 2^48.  The scaled field of a field with |u| <= 2^975 therefore
// stays finite.  Outside 0 < r <= 1/4, or where M would be 0, every step is
// the canonical one (t = fma(-4, u, s), u' = fma(r, t, u)).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "hxc.h"
#include "kernels.cuh"

namespace hxc {
namespace drv {

// Largest number of scaled steps in a row for diffusion number r (0: none).
inline int ftcs2_max_scaled(double r) {
    if (!(r > 0.0 && r <= 0.25)) return 0;
    // largest m with r^m >= 2^-48 (exact for powers of two such as 1/4)
    long double p = 1.0L;
    int m = 0;
    while (m < 64) {
        p *= (long double)r;
        if (p < 0x1p-48L) break;
        m++;
    }
    return m;
}

// Kind and coefficients of step j (0-based) of an interval of L steps.
inline k::Ftcs2Step ftcs2_step(double r, int64_t j, int64_t L) {
    const int M = ftcs2_max_scaled(r);
    if (M == 0) return {k::kFtcs2Canon, r, 0.0};
    const int64_t P = (int64_t)M + 1, q = j % P, end = std::min<int64_t>(L, j - q + P);
    const long double rl = r, c = 1.0L - 4.0L * rl;
    if (j + 1 < end) return {k::kFtcs2Scaled, (double)(c / rl), 0.0};
    // closing step after q scaled steps: v = u_n / r^q
    const long double rho = std::pow(rl, (long double)q);
    return {k::kFtcs2Close, (double)(rl * rho), (double)(c * rho)};
}

// Interval length of a run of hxc_heat2d_run (0 when there are no steps).
inline int64_t heat2d_interval(const hxc_heat2d_cfg &c) {
    const int64_t n_snap = c.snapshot_every > 0 ? c.steps / c.snapshot_every : 0;
    const bool want_snaps = n_snap > 0 && (c.host_norms || c.gpu_norms);
    return want_snaps ? c.snapshot_every : std::min<int64_t>(c.steps, 100);
}

// Number of canonical, scaled and closing steps of `steps` steps issued in
// intervals of `interval` steps.
inline void ftcs2_count(double r, int64_t steps, int64_t interval, int64_t counts[3]) {
    counts[0] = counts[1] = counts[2] = 0;
    if (steps <= 0 || interval <= 0) return;
    const int M = ftcs2_max_scaled(r);
    const int64_t full = steps / interval, rest = steps % interval;
    for (int64_t L : {interval, rest}) {
        const int64_t times = L == interval ? full : (rest > 0 ? 1 : 0);
        if (L <= 0 || times == 0) continue;
        if (M == 0) {
            counts[k::kFtcs2Canon] += times * L;
            continue;
        }
        const int64_t groups = (L + M) / (M + 1);
        counts[k::kFtcs2Scaled] += times * (L - groups);
        counts[k::kFtcs2Close] += times * groups;
    }
}

}  // namespace drv
}  // namespace hxc
