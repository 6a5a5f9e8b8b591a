// Step schedule of the 1D and 2D FTCS runs (host side).
//
// FTCS in d dimensions is linear: u_{n+1} = (1 - 2d r) u_n + r s(u_n), with
// s the sum of the 2d neighbours, = r ((1 - 2d r)/r u_n + s(u_n)).  A run
// therefore carries the field scaled by r^-m after m steps, v = u_n / r^m,
// and advances it with one FMA after the neighbour sum
// (v' = fma((1 - 2d r)/r, v, s(v)), a "scaled" step: 3 FP64 operations per
// point instead of 4 in 2D, 2 instead of 3 in 1D); a "closing" step takes
// the scaled field back to true values,
// u_{n+1} = fma(r^(m+1), s(v), ((1 - 2d r) r^m) v).
//
// The steps of a run are issued in intervals (2D: between snapshots, or of
// at most 100 steps without them; 1D: of at most 128 steps; a captured
// graph holds one interval).  Each interval is cut into groups of at most
// M + 1 steps: a group's last step closes, the others are scaled, so the
// field is true at every interval end (snapshots, graph boundaries, the
// result).  A step's kind and coefficients depend only on its index in its
// interval, which keeps the bits independent of tiling, partitioning, mode,
// steps per launch and graph replay.
//
// M bounds the growth of the scaled field: for 0 < r <= 1/(2d) the scaled
// step's coefficients (1 - 2d r)/r and 2d 1s are non-negative and sum to
// 1/r, so |v| grows by at most 1/r per step; M is the largest m with
// r^-m <= 2^96.  The scaled field of a field with |u| <= 2^927 therefore
// stays finite.  Outside 0 < r <= 1/(2d), or where M would be 0, every step
// is the canonical one (t = fma(-2d, u, s), u' = fma(r, t, u)).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "hxc.h"
#include "kernels.cuh"

namespace hxc {
namespace drv {

// Largest number of scaled steps in a row for diffusion number r in d
// dimensions (0: none).
inline int ftcs_max_scaled(int dim, double r) {
    if (!(r > 0.0 && r <= 0.5 / dim)) return 0;
    // largest m with r^m >= 2^-96 (exact for powers of two such as 1/4)
    long double p = 1.0L;
    int m = 0;
    while (m < k::kFtcsMaxGroup - 1) {
        p *= (long double)r;
        if (p < 0x1p-96L) break;
        m++;
    }
    return m;
}

// Coefficients of the closing step after q scaled steps: {r^(q+1),
// (1 - 2d r) r^q}, formed in 80-bit long double and rounded once.
inline void ftcs_close_coef(int dim, double r, int q, double *a, double *b) {
    const long double rl = r, c = 1.0L - 2.0L * dim * rl;
    const long double rho = std::pow(rl, (long double)q);
    *a = (double)(rl * rho);
    *b = (double)(c * rho);
}

// The plan of the launches of a run (same kinds and coefficients as
// ftcs_step): a run of `total` steps in intervals of `interval`.
inline k::FtcsPlan ftcs_plan(int dim, double r, int64_t total, int64_t interval) {
    k::FtcsPlan p{};
    const int M = ftcs_max_scaled(dim, r);
    p.r = r;
    p.total = total;
    p.I = (int)std::max<int64_t>(1, interval);
    p.P = M == 0 ? 0 : M + 1;
    if (M > 0) {
        const long double rl = r;
        p.k = (double)((1.0L - 2.0L * dim * rl) / rl);
        for (int q = 0; q <= M; q++) ftcs_close_coef(dim, r, q, &p.a[q], &p.b[q]);
    }
    return p;
}

// Kind and coefficients of step j (0-based) of an interval of L steps.
inline k::FtcsStep ftcs_step(int dim, double r, int64_t j, int64_t L) {
    return k::ftcs_plan_step(ftcs_plan(dim, r, L, L), j);
}
inline k::FtcsStep ftcs2_step(double r, int64_t j, int64_t L) { return ftcs_step(2, r, j, L); }

// Interval length of a run of hxc_heat2d_run (0 when there are no steps).
inline int64_t heat2d_interval(const hxc_heat2d_cfg &c) {
    const int64_t n_snap = c.snapshot_every > 0 ? c.steps / c.snapshot_every : 0;
    const bool want_snaps = n_snap > 0 && (c.host_norms || c.gpu_norms);
    return want_snaps ? c.snapshot_every : std::min<int64_t>(c.steps, 100);
}

// Interval length of a run of hxc_heat1d_run (the steps one graph holds).
inline int64_t heat1d_interval(int64_t steps) { return std::min<int64_t>(steps, 128); }

// Number of canonical, scaled and closing steps of `steps` steps issued in
// intervals of `interval` steps.
inline void ftcs_count(int dim, double r, int64_t steps, int64_t interval, int64_t counts[3]) {
    counts[0] = counts[1] = counts[2] = 0;
    if (steps <= 0 || interval <= 0) return;
    const int M = ftcs_max_scaled(dim, r);
    const int64_t full = steps / interval, rest = steps % interval;
    for (int64_t L : {interval, rest}) {
        const int64_t times = L == interval ? full : (rest > 0 ? 1 : 0);
        if (L <= 0 || times == 0) continue;
        if (M == 0) {
            counts[k::kFtcsCanon] += times * L;
            continue;
        }
        const int64_t groups = (L + M) / (M + 1);
        counts[k::kFtcsScaled] += times * (L - groups);
        counts[k::kFtcsClose] += times * groups;
    }
}

}  // namespace drv
}  // namespace hxc
