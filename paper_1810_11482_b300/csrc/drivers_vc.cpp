// Whole-run entry points of the variable-diffusivity path: batches of
// independent problems, the forward run of one problem, the squared-error
// seed and the checkpointed adjoint.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "drivers_util.hpp"
#include "kernels.cuh"
#include "runtime.hpp"

using namespace hxc;
using namespace hxc::drv;

namespace {

hxc_status need(Ref<Buffer> &b, hxc_buffer h, Device *d, size_t bytes, const char *what) {
    b = buf_from_handle(h);
    if (!b) return HXC_E_INVALID;
    if (b->dev.get() != d || b->bytes < bytes) {
        set_error("%s: buffer on another device or smaller than %zu bytes", what, bytes);
        return HXC_E_INVALID;
    }
    return HXC_OK;
}

hxc_status join_deps(Device *d, const std::vector<FutRef> &dv, FutRef *prev) {
    if (dv.empty()) return HXC_OK;
    return issue_device_op(d, kJoinSlot, dv, StreamOp(), {}, prev);
}

std::vector<FutRef> one(const FutRef &f) {
    std::vector<FutRef> v;
    if (f) v.push_back(f);
    return v;
}

}  // namespace

extern "C" {

hxc_status hxc_varcoef_batch_run(hxc_device dh, hxc_buffer uh, hxc_buffer kh, const int64_t *sides,
                                 const double *cs, int64_t nprob, int steps, hxc_mode mode,
                                 const hxc_future *deps, int ndeps, hxc_future *out,
                                 hxc_run_stats *stats_out) {
    hxc::drv::NvtxRange nvtx_range("hxc_varcoef_batch_run");
    Ref<Device> d = dev_from_handle(dh);
    if (!d) return HXC_E_INVALID;
    if (!sides || !cs || nprob <= 0 || nprob > (1 << 24) || steps < 0 ||
        (mode != HXC_MODE_PLAIN && mode != HXC_MODE_GRAPH && mode != HXC_MODE_FUSED)) {
        set_error("hxc_varcoef_batch_run: invalid arguments");
        return HXC_E_INVALID;
    }
    std::vector<int64_t> off(nprob);
    int64_t total = 0, total_rows = 0;
    for (int64_t p = 0; p < nprob; p++) {
        if (sides[p] <= 0 || sides[p] > (1 << 20) || !(cs[p] >= 0.0)) {
            set_error("hxc_varcoef_batch_run: bad side or c of problem %lld", (long long)p);
            return HXC_E_INVALID;
        }
        off[p] = total;
        total += sides[p] * sides[p];
        total_rows += sides[p];
    }
    Ref<Buffer> u, kap;
    hxc_status st;
    if ((st = need(u, uh, d.get(), (size_t)total * 8, "batch.u"))) return st;
    if ((st = need(kap, kh, d.get(), (size_t)total * 8, "batch.kappa"))) return st;
    if (u->ptr == kap->ptr) {
        set_error("hxc_varcoef_batch_run: u and kappa alias");
        return HXC_E_INVALID;
    }
    std::vector<FutRef> dv;
    if ((st = deps_from_handles(deps, ndeps, &dv))) return st;
    if (stats_out) memset(stats_out, 0, sizeof *stats_out);
    if (has_pending_host(dv)) {
        std::vector<int64_t> sv(sides, sides + nprob);
        std::vector<double> cv(cs, cs + nprob);
        FutRef a, b;
        defer_run(dv,
                  [=](FutRef *ia, FutRef *ib) {
                      hxc_future h = nullptr;
                      hxc_status s2 = hxc_varcoef_batch_run(dh, uh, kh, sv.data(), cv.data(), nprob,
                                                            steps, mode, nullptr, 0, &h, nullptr);
                      if (s2) return s2;
                      *ia = FutRef(reinterpret_cast<Future *>(h), true);
                      *ib = *ia;
                      return HXC_OK;
                  },
                  &a, &b);
        fut_on_done(a, [u, kap](hxc_status) {});
        if (out) *out = to_handle(a);
        return HXC_OK;
    }
    Stats stats{stats_out};
    if ((st = d->make_current())) return st;
    Device *dev = d.get();
    // scratch: second field, coefficients, problem list, row list, queue
    void *pt, *pe, *ps, *pm, *pdesc, *prows, *pq;
    if ((st = dev->scratch_get("batch.tmp", (size_t)total * 8, &pt))) return st;
    if ((st = dev->scratch_get("batch.wE", (size_t)total * 8, &pe))) return st;
    if ((st = dev->scratch_get("batch.wS", (size_t)total * 8, &ps))) return st;
    if ((st = dev->scratch_get("batch.m", (size_t)total * 8, &pm))) return st;
    if ((st = dev->scratch_get("batch.desc", (size_t)nprob * k::vc_problem_bytes(), &pdesc))) return st;
    if ((st = dev->scratch_get("batch.rows", (size_t)(nprob + 1) * 8, &prows))) return st;
    if ((st = dev->scratch_get("batch.queue", 16, &pq))) return st;
    double *U = (double *)u->ptr, *Tm = (double *)pt, *WE = (double *)pe, *WS = (double *)ps,
           *M = (double *)pm;
    const double *K = (const double *)kap->ptr;
    FutRef prev;
    if ((st = join_deps(dev, dv, &prev))) return st;

    if (mode == HXC_MODE_PLAIN) {
        // one coefficient launch and `steps` step launches per problem,
        // problems spread over 16 stream slots
        std::vector<FutRef> finals;
        for (int64_t p = 0; p < nprob; p++) {
            const int slot = (int)(p % 16);
            const int64_t s = sides[p], o = off[p];
            const double c = cs[p];
            FutRef f;
            if ((st = issue_device_op(dev, slot, one(prev),
                                      [=](cudaStream_t q) {
                                          return k::vc_coef(K + o, c, s, s, WE + o, WS + o, M + o, q);
                                      },
                                      {}, &f)))
                return st;
            stats.launch();
            for (int t = 0; t < steps; t++) {
                const double *src = (t & 1) ? Tm + o : U + o;
                double *dst = (t & 1) ? U + o : Tm + o;
                FutRef g;
                if ((st = issue_device_op(dev, slot, one(f),
                                          [=](cudaStream_t q) {
                                              return k::vc_step(src, dst, WE + o, WS + o, M + o, s, s, q);
                                          },
                                          {}, &g)))
                    return st;
                stats.launch();
                f = g;
            }
            if (steps & 1) {
                FutRef g;
                if ((st = issue_device_op(dev, slot, one(f),
                                          [=](cudaStream_t q) {
                                              return cudaMemcpyAsync(U + o, Tm + o, s * s * 8,
                                                                     cudaMemcpyDeviceToDevice, q);
                                          },
                                          {}, &g)))
                    return st;
                stats.copy(0, 0);
                f = g;
            }
            if (p + 16 >= nprob) finals.push_back(f);  // last problem of its slot
        }
        FutRef fin;
        if ((st = issue_device_op(dev, kJoinSlot, finals, StreamOp(),
                                  {AnyRef(u.get(), false), AnyRef(kap.get(), false)}, &fin)))
            return st;
        if (out) *out = to_handle(fin);
        return HXC_OK;
    }

    // problem list: largest first (the persistent kernel's work order)
    std::vector<int64_t> order(nprob);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int64_t a, int64_t b) { return sides[a] > sides[b]; });
    std::vector<char> desc((size_t)nprob * k::vc_problem_bytes());
    std::vector<int64_t> rows(nprob + 1, 0);
    for (int64_t q = 0; q < nprob; q++) {
        const int64_t p = order[q];
        k::vc_pack_problem(desc.data() + q * k::vc_problem_bytes(), off[p], (int32_t)sides[p], cs[p]);
        rows[q + 1] = rows[q] + sides[p];
    }
    // upload on slot 0 (which also runs the kernels) and wait for the copy,
    // so that the host vectors may go out of scope
    {
        FutRef f;
        char *dd = (char *)pdesc;
        int64_t *dr = (int64_t *)prows;
        const char *hd = desc.data();
        const int64_t *hr = rows.data();
        const size_t nd = desc.size(), nr = rows.size() * 8;
        if ((st = issue_device_op(dev, 0, one(prev),
                                  [=](cudaStream_t q) {
                                      cudaError_t e = cudaMemcpyAsync(dd, hd, nd, cudaMemcpyHostToDevice, q);
                                      if (e == cudaSuccess)
                                          e = cudaMemcpyAsync(dr, hr, nr, cudaMemcpyHostToDevice, q);
                                      if (e == cudaSuccess) e = cudaStreamSynchronize(q);
                                      return e;
                                  },
                                  {}, &f)))
            return st;
        prev = f;
    }
    const int np = (int)nprob;
    const int64_t *R = (const int64_t *)prows;
    const void *D = pdesc;
    if (mode == HXC_MODE_FUSED) {
        unsigned *Q = (unsigned *)pq;
        FutRef f;
        if ((st = issue_device_op(dev, 0, one(prev),
                                  [=](cudaStream_t q) {
                                      return k::vc_batch_persistent(D, np, Q, U, Tm, K, WE, WS, M, steps, 0, q);
                                  },
                                  {AnyRef(u.get(), false), AnyRef(kap.get(), false)}, &f)))
            return st;
        stats.launch();
        if (out) *out = to_handle(f);
        return HXC_OK;
    }
    // GRAPH: batched coefficient launch + one batched launch per step
    std::string key = key_of("vcbatch", {(double)nprob, (double)total, (double)steps},
                             {U, K, Tm, WE, D, R});
    Ref<Graph> g;
    auto body = [&](int64_t *kernels) -> hxc_status {
        *kernels = 1 + steps;
        FutRef f;
        hxc_status s2 = issue_device_op(
            dev, 0, {}, [=](cudaStream_t q) { return k::vc_batch_coef(D, R, np, total_rows, K, WE, WS, M, q); },
            {}, &f);
        for (int t = 0; t < steps && !s2; t++) {
            const double *src = (t & 1) ? Tm : U;
            double *dst = (t & 1) ? U : Tm;
            FutRef h;
            s2 = issue_device_op(
                dev, 0, one(f),
                [=](cudaStream_t q) { return k::vc_batch_step(D, R, np, total_rows, src, dst, WE, WS, M, q); },
                {}, &h);
            f = h;
        }
        if (!s2 && (steps & 1)) {
            FutRef h;
            s2 = issue_device_op(
                dev, 0, one(f),
                [=](cudaStream_t q) { return cudaMemcpyAsync(U, Tm, total * 8, cudaMemcpyDeviceToDevice, q); },
                {}, &h);
        }
        return s2;
    };
    if ((st = cached_graph(dev, key, body, &g))) return st;
    FutRef f;
    if ((st = launch_graph(dev, g, 0, one(prev), &f))) return st;
    stats.launch(g->kernels);
    if (stats_out) stats_out->graph_launches++;
    FutRef fin;
    if ((st = issue_device_op(dev, kJoinSlot, one(f), StreamOp(),
                              {AnyRef(u.get(), false), AnyRef(kap.get(), false)}, &fin)))
        return st;
    if (out) *out = to_handle(fin);
    return HXC_OK;
}

hxc_status hxc_sqerr_seed(hxc_device dh, hxc_buffer uh, hxc_buffer th, hxc_buffer lh,
                          hxc_buffer loss_h, int64_t n, int slot, const hxc_future *deps, int ndeps,
                          hxc_future *out) {
    hxc::drv::NvtxRange nvtx_range("hxc_sqerr_seed");
    if (!out) {
        set_error("hxc_sqerr_seed: NULL output");
        return HXC_E_INVALID;
    }
    Ref<Device> d = dev_from_handle(dh);
    if (!d || n < 0 || slot < 0 || slot >= HXC_MAX_SLOTS) {
        set_error("hxc_sqerr_seed: invalid arguments");
        return HXC_E_INVALID;
    }
    Ref<Buffer> u, t, l, ls;
    hxc_status st;
    if ((st = need(u, uh, d.get(), (size_t)n * 8, "sqerr.u"))) return st;
    if ((st = need(t, th, d.get(), (size_t)n * 8, "sqerr.t"))) return st;
    if (lh && (st = need(l, lh, d.get(), (size_t)n * 8, "sqerr.lam"))) return st;
    if ((st = need(ls, loss_h, d.get(), 8, "sqerr.loss"))) return st;
    std::vector<FutRef> dv;
    if ((st = deps_from_handles(deps, ndeps, &dv))) return st;
    // scratch per stream slot: launches on one slot never overlap
    void *scratch;
    if ((st = d->scratch_get("sqerr." + std::to_string(slot), k::sqerr_scratch_bytes(), &scratch)))
        return st;
    const double *up = (const double *)u->ptr, *tp = (const double *)t->ptr;
    double *lp = l ? (double *)l->ptr : nullptr, *lsp = (double *)ls->ptr;
    std::vector<AnyRef> keep{AnyRef(u.get(), false), AnyRef(t.get(), false), AnyRef(ls.get(), false)};
    if (l) keep.push_back(AnyRef(l.get(), false));
    FutRef f;
    if ((st = issue_device_op(d.get(), slot, dv,
                              [=](cudaStream_t q) { return k::sqerr_seed(up, tp, lp, n, scratch, lsp, q); },
                              keep, &f)))
        return st;
    *out = to_handle(f);
    return HXC_OK;
}

hxc_status hxc_varcoef_forward_run(hxc_device dh, hxc_buffer u0h, hxc_buffer kh, int64_t ny,
                                   int64_t nx, double c, int steps, hxc_buffer uTh,
                                   const hxc_future *deps, int ndeps, hxc_future *out,
                                   hxc_run_stats *stats_out) {
    hxc::drv::NvtxRange nvtx_range("hxc_varcoef_forward_run");
    Ref<Device> d = dev_from_handle(dh);
    if (!d || ny <= 0 || nx <= 0 || steps < 0) {
        set_error("hxc_varcoef_forward_run: invalid arguments");
        return HXC_E_INVALID;
    }
    const int64_t n = ny * nx;
    Ref<Buffer> u0, kap, uT;
    hxc_status st;
    if ((st = need(u0, u0h, d.get(), (size_t)n * 8, "forward.u0"))) return st;
    if ((st = need(kap, kh, d.get(), (size_t)n * 8, "forward.kappa"))) return st;
    if ((st = need(uT, uTh, d.get(), (size_t)n * 8, "forward.uT"))) return st;
    if (uT->ptr == kap->ptr || (uT->ptr == u0->ptr && steps > 0)) {
        set_error("hxc_varcoef_forward_run: uT aliases kappa or u0");
        return HXC_E_INVALID;
    }
    std::vector<FutRef> dv;
    if ((st = deps_from_handles(deps, ndeps, &dv))) return st;
    if (stats_out) memset(stats_out, 0, sizeof *stats_out);
    Stats stats{stats_out};
    Device *dev = d.get();
    if ((st = dev->make_current())) return st;
    void *pw, *pe, *ps, *pm;
    if ((st = dev->scratch_get("fwd.w", (size_t)n * 8, &pw))) return st;
    if ((st = dev->scratch_get("fwd.wE", (size_t)n * 8, &pe))) return st;
    if ((st = dev->scratch_get("fwd.wS", (size_t)n * 8, &ps))) return st;
    if ((st = dev->scratch_get("fwd.m", (size_t)n * 8, &pm))) return st;
    double *W = (double *)pw, *WE = (double *)pe, *WS = (double *)ps, *M = (double *)pm;
    const double *K = (const double *)kap->ptr, *U0 = (const double *)u0->ptr;
    double *UT = (double *)uT->ptr;
    FutRef f;
    if ((st = join_deps(dev, dv, &f))) return st;
    FutRef g;
    if ((st = issue_device_op(dev, 0, one(f),
                              [=](cudaStream_t q) { return k::vc_coef(K, c, ny, nx, WE, WS, M, q); }, {}, &g)))
        return st;
    stats.launch();
    f = g;
    // the last step writes uT: the states alternate between W and uT.  The
    // steps are one operation: back-to-back launches, each after the first
    // with programmatic dependent launch
    if (steps > 0) {
        if ((st = issue_device_op(dev, 0, one(f),
                                  [=](cudaStream_t q) {
                                      for (int t = 0; t < steps; t++) {
                                          const bool to_T = ((steps - 1 - t) % 2) == 0;
                                          const double *src = t == 0 ? U0 : (to_T ? W : UT);
                                          double *dst = to_T ? UT : W;
                                          cudaError_t e =
                                              k::vc_step(src, dst, WE, WS, M, ny, nx, q, t > 0);
                                          if (e != cudaSuccess) return e;
                                      }
                                      return cudaSuccess;
                                  },
                                  {}, &g)))
            return st;
        stats.launch(steps);
        f = g;
    }
    if (steps == 0 && UT != U0) {
        if ((st = issue_device_op(dev, 0, one(f),
                                  [=](cudaStream_t q) {
                                      return cudaMemcpyAsync(UT, U0, n * 8, cudaMemcpyDeviceToDevice, q);
                                  },
                                  {}, &g)))
            return st;
        f = g;
    }
    FutRef fin;
    if ((st = issue_device_op(dev, kJoinSlot, one(f), StreamOp(),
                              {AnyRef(u0.get(), false), AnyRef(kap.get(), false), AnyRef(uT.get(), false)},
                              &fin)))
        return st;
    if (out) *out = to_handle(fin);
    return HXC_OK;
}

}  // extern "C"

namespace {

// The checkpointed adjoint.  With u0h it runs its own forward pass to lay
// down the checkpoints; with tapeh (and no u0h, no uTh) it takes them from a
// tape written by hxc_varcoef_forward_tape and starts with the segments.
hxc_status adjoint_impl(hxc_device dh, hxc_buffer u0h, hxc_buffer tapeh, hxc_buffer kh,
                        hxc_buffer lTh, int64_t ny, int64_t nx, double c, int steps, int every,
                        hxc_mode mode, hxc_buffer gkh, hxc_buffer gu0h, hxc_buffer uTh,
                        const hxc_future *deps, int ndeps, hxc_future *out,
                        hxc_run_stats *stats_out) {
    const char *fn = tapeh ? "hxc_varcoef_adjoint_tape" : "hxc_varcoef_adjoint_run";
    Ref<Device> d = dev_from_handle(dh);
    if (!d || ny <= 0 || nx <= 0 || steps < 0 || every < 0 || (!u0h == !tapeh) ||
        (tapeh && uTh) ||
        (mode != HXC_MODE_PLAIN && mode != HXC_MODE_GRAPH && mode != HXC_MODE_FUSED)) {
        set_error("%s: invalid arguments", fn);
        return HXC_E_INVALID;
    }
    const int64_t n = ny * nx;
    const size_t nb = (size_t)n * 8;
    if (every == 0) every = std::max(1, (int)std::ceil(std::sqrt((double)std::max(1, steps))));
    const int nseg = steps > 0 ? (steps + every - 1) / every : 0;
    Ref<Buffer> u0, tape, kap, lT, gk, gu0, uT;
    hxc_status st;
    if (tapeh) {
        if ((st = need(tape, tapeh, d.get(), nb * std::max(1, nseg), "adjoint.tape"))) return st;
        u0 = tape;  // state 0 is the tape's first checkpoint
    } else if ((st = need(u0, u0h, d.get(), nb, "adjoint.u0"))) {
        return st;
    }
    if ((st = need(kap, kh, d.get(), nb, "adjoint.kappa"))) return st;
    if ((st = need(lT, lTh, d.get(), nb, "adjoint.lamT"))) return st;
    if ((st = need(gk, gkh, d.get(), nb, "adjoint.gk"))) return st;
    if ((st = need(gu0, gu0h, d.get(), nb, "adjoint.gu0"))) return st;
    if (uTh && (st = need(uT, uTh, d.get(), nb, "adjoint.uT"))) return st;
    {
        const void *outs[3] = {gk->ptr, gu0->ptr, uT ? uT->ptr : nullptr};
        const void *ins[3] = {u0->ptr, kap->ptr, lT->ptr};
        for (auto o : outs)
            for (auto i : ins)
                if (o && o == i) {
                    set_error("%s: an output aliases an input", fn);
                    return HXC_E_INVALID;
                }
        if (gk->ptr == gu0->ptr || (uT && (uT->ptr == gk->ptr || uT->ptr == gu0->ptr))) {
            set_error("%s: outputs alias", fn);
            return HXC_E_INVALID;
        }
        if (tape) {
            // the gradients must not land inside the tape the run still reads
            const char *t0 = (const char *)tape->ptr, *t1 = t0 + nb * std::max(1, nseg);
            for (const void *o : {(const void *)gk->ptr, (const void *)gu0->ptr, (const void *)lT->ptr})
                if ((const char *)o + nb > t0 && (const char *)o < t1) {
                    set_error("%s: the tape overlaps lamT, gk or gu0", fn);
                    return HXC_E_INVALID;
                }
        }
    }
    std::vector<FutRef> dv;
    if ((st = deps_from_handles(deps, ndeps, &dv))) return st;
    if (stats_out) memset(stats_out, 0, sizeof *stats_out);
    if (has_pending_host(dv)) {
        FutRef a, b;
        defer_run(dv,
                  [=](FutRef *ia, FutRef *ib) {
                      hxc_future h = nullptr;
                      hxc_status s2 = adjoint_impl(dh, u0h, tapeh, kh, lTh, ny, nx, c, steps, every,
                                                   mode, gkh, gu0h, uTh, nullptr, 0, &h, nullptr);
                      if (s2) return s2;
                      *ia = FutRef(reinterpret_cast<Future *>(h), true);
                      *ib = *ia;
                      return HXC_OK;
                  },
                  &a, &b);
        fut_on_done(a, [u0, kap, lT, gk, gu0, uT](hxc_status) {});
        if (out) *out = to_handle(a);
        return HXC_OK;
    }
    Stats stats{stats_out};
    Device *dev = d.get();
    if ((st = dev->make_current())) return st;
    // scratch: coefficients, checkpoints 1..nseg-1 (without a tape), the segment store
    // (states 1..every-1 of a segment), two work fields, two adjoint fields,
    // the per-face gradient sums
    void *pe, *ps, *pm, *pck, *pseg, *pw, *pl, *pf;
    if ((st = dev->scratch_get("adj.wE", nb, &pe))) return st;
    if ((st = dev->scratch_get("adj.wS", nb, &ps))) return st;
    if ((st = dev->scratch_get("adj.m", nb, &pm))) return st;
    if (tape)
        pck = tape->ptr;
    else if ((st = dev->scratch_get("adj.ckpt", nb * std::max(1, nseg), &pck)))
        return st;
    if ((st = dev->scratch_get("adj.seg", nb * std::max(1, every), &pseg))) return st;
    if ((st = dev->scratch_get("adj.work", nb * 2, &pw))) return st;
    if ((st = dev->scratch_get("adj.lam", nb * 2, &pl))) return st;
    const size_t face_bytes = k::vc_face_doubles(ny, nx) * 8;
    if ((st = dev->scratch_get("adj.face", face_bytes, &pf))) return st;
    double *WE = (double *)pe, *WS = (double *)ps, *M = (double *)pm;
    double *CK = (double *)pck, *SEG = (double *)pseg, *WK = (double *)pw, *LM = (double *)pl;
    double *FACE = (double *)pf;
    const double *U0 = (const double *)u0->ptr, *K = (const double *)kap->ptr,
                 *LT = (const double *)lT->ptr;
    double *GK = (double *)gk->ptr, *GU = (double *)gu0->ptr, *UT = uT ? (double *)uT->ptr : nullptr;
    // checkpoint k (state k*every): k = 0 is u0 itself
    auto ckpt = [=](int kk) -> const double * { return kk == 0 ? U0 : CK + (size_t)kk * n; };

    // Issues the whole computation on slot 0 (in stream order).
    auto body = [&](Stats &sc) -> hxc_status {
        hxc_status s2;
        FutRef f;
        auto op = [&](StreamOp o) -> hxc_status {
            FutRef g;
            hxc_status s3 = issue_device_op(dev, 0, one(f), std::move(o), {}, &g);
            if (!s3) f = g;
            return s3;
        };
        // FUSED and GRAPH issue each run of kernel launches as one operation,
        // the launches after the first with programmatic dependent launch;
        // PLAIN issues every launch as an operation of its own
        using Launch = std::function<cudaError_t(cudaStream_t, bool)>;
        std::vector<Launch> pend;
        auto flush = [&]() -> hxc_status {
            if (pend.empty()) return HXC_OK;
            auto ks = std::make_shared<std::vector<Launch>>(std::move(pend));
            pend.clear();
            return op([ks](cudaStream_t q) {
                for (size_t i = 0; i < ks->size(); i++) {
                    cudaError_t e = (*ks)[i](q, i > 0);
                    if (e != cudaSuccess) return e;
                }
                return cudaSuccess;
            });
        };
        auto kern = [&](Launch l) -> hxc_status {
            pend.push_back(std::move(l));
            return mode == HXC_MODE_PLAIN ? flush() : HXC_OK;
        };
        if ((s2 = op([=](cudaStream_t q) { return k::vc_coef(K, c, ny, nx, WE, WS, M, q); }))) return s2;
        sc.launch();
        // forward: states pass through the work fields; segment starts go to
        // their checkpoint, the final state to uT (or a work field); a tape
        // holds the checkpoints already
        const double *cur = U0;
        for (int t = 0; t < (tape ? 0 : steps); t++) {
            double *dst;
            if (t + 1 == steps)
                dst = UT ? UT : WK + (size_t)((t + 1) & 1) * n;
            else if ((t + 1) % every == 0)
                dst = CK + (size_t)((t + 1) / every) * n;
            else
                dst = WK + (size_t)((t + 1) & 1) * n;
            if (dst == cur) dst = WK + (size_t)(((t + 1) & 1) ^ 1) * n;
            const double *src = cur;
            if ((s2 = kern([=](cudaStream_t q, bool pdl) {
                     return k::vc_step(src, dst, WE, WS, M, ny, nx, q, pdl);
                 })))
                return s2;
            sc.launch();
            cur = dst;
        }
        if ((s2 = flush())) return s2;
        // adjoint seed and the per-face gradient sums
        if ((s2 = op([=](cudaStream_t q) {
                 cudaError_t e = cudaMemcpyAsync(LM, LT, nb, cudaMemcpyDeviceToDevice, q);
                 if (e == cudaSuccess) e = cudaMemsetAsync(FACE, 0, face_bytes, q);
                 return e;
             })))
            return s2;
        int li = 0;  // LM + li*n holds lambda^{t+1}
        for (int kk = nseg - 1; kk >= 0; kk--) {
            const int n0 = kk * every, n1 = std::min(steps, n0 + every);
            // recompute states n0+1 .. n1-1 of the segment into SEG[1..]
            for (int t = n0; t + 1 < n1; t++) {
                const double *src = t == n0 ? ckpt(kk) : SEG + (size_t)(t - n0) * n;
                double *dst = SEG + (size_t)(t + 1 - n0) * n;
                if ((s2 = kern([=](cudaStream_t q, bool pdl) {
                         return k::vc_step(src, dst, WE, WS, M, ny, nx, q, pdl);
                     })))
                    return s2;
                sc.launch();
            }
            for (int t = n1 - 1; t >= n0; t--) {
                const double *ut = t == n0 ? ckpt(kk) : SEG + (size_t)(t - n0) * n;
                const double *lin = LM + (size_t)li * n;
                double *lout = (t == 0) ? GU : LM + (size_t)(li ^ 1) * n;
                if (mode == HXC_MODE_PLAIN) {
                    if ((s2 = kern([=](cudaStream_t q, bool pdl) {
                             return k::vc_adjoint(lin, lout, ut, WE, WS, M, FACE, ny, nx, false, true,
                                                  q, pdl);
                         })))
                        return s2;
                    if ((s2 = kern([=](cudaStream_t q, bool pdl) {
                             return k::vc_adjoint(lin, lout, ut, WE, WS, M, FACE, ny, nx, true, false,
                                                  q, pdl);
                         })))
                        return s2;
                    sc.launch(2);
                } else {
                    if ((s2 = kern([=](cudaStream_t q, bool pdl) {
                             return k::vc_adjoint(lin, lout, ut, WE, WS, M, FACE, ny, nx, true, true,
                                                  q, pdl);
                         })))
                        return s2;
                    sc.launch();
                }
                li ^= 1;
            }
        }
        if ((s2 = flush())) return s2;
        if (steps > 0) {
            // dL/dkappa from the face sums
            if ((s2 = op([=](cudaStream_t q) { return k::vc_face_combine(FACE, GK, c, ny, nx, q); })))
                return s2;
            sc.launch();
        }
        if (steps == 0) {
            if ((s2 = op([=](cudaStream_t q) {
                     cudaError_t e = cudaMemcpyAsync(GU, LT, nb, cudaMemcpyDeviceToDevice, q);
                     if (e == cudaSuccess) e = cudaMemsetAsync(GK, 0, nb, q);
                     if (e == cudaSuccess && UT) e = cudaMemcpyAsync(UT, U0, nb, cudaMemcpyDeviceToDevice, q);
                     return e;
                 })))
                return s2;
        }
        return HXC_OK;
    };
    FutRef prev;
    if ((st = join_deps(dev, dv, &prev))) return st;
    FutRef last;
    if (mode == HXC_MODE_GRAPH) {
        std::string key = key_of(tape ? "adjoint_tape" : "adjoint",
                                 {(double)ny, (double)nx, c, (double)steps, (double)every},
                                 {U0, K, LT, GK, GU, UT, WE, CK, SEG, WK, LM, FACE});
        Ref<Graph> g;
        auto capture = [&](int64_t *kernels) {
            hxc_run_stats cnt{};
            Stats counting{&cnt};
            hxc_status s2 = body(counting);
            *kernels = cnt.kernel_launches;
            return s2;
        };
        if ((st = cached_graph(dev, key, capture, &g))) return st;
        if ((st = launch_graph(dev, g, 0, one(prev), &last))) return st;
        if (stats_out) {
            stats_out->graph_launches = 1;
            stats_out->kernel_launches = g->kernels;
        }
    } else {
        if (prev) {
            // make slot 0 wait for the caller's dependencies first
            FutRef g;
            if ((st = issue_device_op(dev, 0, one(prev), StreamOp(), {}, &g))) return st;
        }
        if ((st = body(stats))) return st;
        // everything was issued on slot 0: a marker there closes the run
        if ((st = issue_device_op(dev, 0, {}, StreamOp(), {}, &last))) return st;
    }
    FutRef fin;
    std::vector<AnyRef> keep{AnyRef(u0.get(), false), AnyRef(kap.get(), false), AnyRef(lT.get(), false),
                             AnyRef(gk.get(), false), AnyRef(gu0.get(), false)};
    if (uT) keep.push_back(AnyRef(uT.get(), false));
    if ((st = issue_device_op(dev, kJoinSlot, one(last), StreamOp(), keep, &fin))) return st;
    if (out) *out = to_handle(fin);
    return HXC_OK;
}

}  // namespace

extern "C" {

hxc_status hxc_varcoef_adjoint_run(hxc_device dh, hxc_buffer u0h, hxc_buffer kh, hxc_buffer lTh,
                                   int64_t ny, int64_t nx, double c, int steps, int every,
                                   hxc_mode mode, hxc_buffer gkh, hxc_buffer gu0h, hxc_buffer uTh,
                                   const hxc_future *deps, int ndeps, hxc_future *out,
                                   hxc_run_stats *stats_out) {
    hxc::drv::NvtxRange nvtx_range("hxc_varcoef_adjoint_run");
    if (!u0h) {
        set_error("hxc_varcoef_adjoint_run: u0 is NULL");
        return HXC_E_INVALID;
    }
    return adjoint_impl(dh, u0h, nullptr, kh, lTh, ny, nx, c, steps, every, mode, gkh, gu0h, uTh,
                        deps, ndeps, out, stats_out);
}

hxc_status hxc_varcoef_adjoint_tape(hxc_device dh, hxc_buffer tapeh, hxc_buffer kh, hxc_buffer lTh,
                                    int64_t ny, int64_t nx, double c, int steps, int every,
                                    hxc_mode mode, hxc_buffer gkh, hxc_buffer gu0h,
                                    const hxc_future *deps, int ndeps, hxc_future *out,
                                    hxc_run_stats *stats_out) {
    hxc::drv::NvtxRange nvtx_range("hxc_varcoef_adjoint_tape");
    if (!tapeh) {
        set_error("hxc_varcoef_adjoint_tape: tape is NULL");
        return HXC_E_INVALID;
    }
    return adjoint_impl(dh, nullptr, tapeh, kh, lTh, ny, nx, c, steps, every, mode, gkh, gu0h,
                        nullptr, deps, ndeps, out, stats_out);
}

hxc_status hxc_varcoef_tape_states(int steps, int every, int64_t *states) {
    if (steps < 0 || every < 0 || !states) {
        set_error("hxc_varcoef_tape_states: invalid arguments");
        return HXC_E_INVALID;
    }
    if (every == 0) every = std::max(1, (int)std::ceil(std::sqrt((double)std::max(1, steps))));
    *states = steps > 0 ? (steps + every - 1) / every : 1;
    return HXC_OK;
}

hxc_status hxc_varcoef_forward_tape(hxc_device dh, hxc_buffer u0h, hxc_buffer kh, int64_t ny,
                                    int64_t nx, double c, int steps, int every, hxc_buffer uTh,
                                    hxc_buffer tapeh, const hxc_future *deps, int ndeps,
                                    hxc_future *out, hxc_run_stats *stats_out) {
    hxc::drv::NvtxRange nvtx_range("hxc_varcoef_forward_tape");
    Ref<Device> d = dev_from_handle(dh);
    if (!d || ny <= 0 || nx <= 0 || steps < 0 || every < 0) {
        set_error("hxc_varcoef_forward_tape: invalid arguments");
        return HXC_E_INVALID;
    }
    if (every == 0) every = std::max(1, (int)std::ceil(std::sqrt((double)std::max(1, steps))));
    const int nseg = steps > 0 ? (steps + every - 1) / every : 1;
    const int64_t n = ny * nx;
    const size_t nb = (size_t)n * 8;
    Ref<Buffer> u0, kap, uT, tape;
    hxc_status st;
    if ((st = need(u0, u0h, d.get(), nb, "forward_tape.u0"))) return st;
    if ((st = need(kap, kh, d.get(), nb, "forward_tape.kappa"))) return st;
    if ((st = need(uT, uTh, d.get(), nb, "forward_tape.uT"))) return st;
    if ((st = need(tape, tapeh, d.get(), nb * nseg, "forward_tape.tape"))) return st;
    {
        const char *t0 = (const char *)tape->ptr, *t1 = t0 + nb * nseg;
        auto inside = [&](const void *p) { return (const char *)p + nb > t0 && (const char *)p < t1; };
        if (uT->ptr == kap->ptr || uT->ptr == u0->ptr || inside(u0->ptr) || inside(kap->ptr) ||
            inside(uT->ptr)) {
            set_error("hxc_varcoef_forward_tape: uT, the tape and the inputs must not overlap");
            return HXC_E_INVALID;
        }
    }
    std::vector<FutRef> dv;
    if ((st = deps_from_handles(deps, ndeps, &dv))) return st;
    if (stats_out) memset(stats_out, 0, sizeof *stats_out);
    Stats stats{stats_out};
    Device *dev = d.get();
    if ((st = dev->make_current())) return st;
    void *pw, *pe, *ps, *pm;
    if ((st = dev->scratch_get("fwdt.work", nb * 2, &pw))) return st;
    if ((st = dev->scratch_get("fwd.wE", nb, &pe))) return st;
    if ((st = dev->scratch_get("fwd.wS", nb, &ps))) return st;
    if ((st = dev->scratch_get("fwd.m", nb, &pm))) return st;
    double *WK = (double *)pw, *WE = (double *)pe, *WS = (double *)ps, *M = (double *)pm;
    const double *K = (const double *)kap->ptr, *U0 = (const double *)u0->ptr;
    double *UT = (double *)uT->ptr, *TP = (double *)tape->ptr;
    FutRef f;
    if ((st = join_deps(dev, dv, &f))) return st;
    auto op = [&](StreamOp o) -> hxc_status {
        FutRef g;
        hxc_status s3 = issue_device_op(dev, 0, one(f), std::move(o), {}, &g);
        if (!s3) f = g;
        return s3;
    };
    if ((st = op([=](cudaStream_t q) {
             cudaError_t e = cudaMemcpyAsync(TP, U0, nb, cudaMemcpyDeviceToDevice, q);
             if (e == cudaSuccess) e = k::vc_coef(K, c, ny, nx, WE, WS, M, q);
             return e;
         })))
        return st;
    stats.launch();
    // the same sequence of states as the adjoint run's own forward pass:
    // segment starts into the tape, the final state into uT, the others
    // through two work fields; the steps are one operation, back-to-back
    // launches, each after the first with programmatic dependent launch
    auto seq = std::make_shared<std::vector<std::pair<const double *, double *>>>();
    const double *cur = TP;
    for (int t = 0; t < steps; t++) {
        double *dst;
        if (t + 1 == steps)
            dst = UT;
        else if ((t + 1) % every == 0)
            dst = TP + (size_t)((t + 1) / every) * n;
        else
            dst = WK + (size_t)((t + 1) & 1) * n;
        if (dst == cur) dst = WK + (size_t)(((t + 1) & 1) ^ 1) * n;
        seq->push_back({cur, dst});
        cur = dst;
    }
    if (steps > 0) {
        if ((st = op([=](cudaStream_t q) {
                 for (size_t t = 0; t < seq->size(); t++) {
                     cudaError_t e = k::vc_step((*seq)[t].first, (*seq)[t].second, WE, WS, M, ny, nx,
                                                q, t > 0);
                     if (e != cudaSuccess) return e;
                 }
                 return cudaSuccess;
             })))
            return st;
        stats.launch(steps);
    }
    if (steps == 0 &&
        (st = op([=](cudaStream_t q) {
             return cudaMemcpyAsync(UT, U0, nb, cudaMemcpyDeviceToDevice, q);
         })))
        return st;
    FutRef fin;
    if ((st = issue_device_op(dev, kJoinSlot, one(f), StreamOp(),
                              {AnyRef(u0.get(), false), AnyRef(kap.get(), false),
                               AnyRef(uT.get(), false), AnyRef(tape.get(), false)},
                              &fin)))
        return st;
    if (out) *out = to_handle(fin);
    return HXC_OK;
}

}  // extern "C"
