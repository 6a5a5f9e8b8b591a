"""Benchmark of the partitioned heat-stencil path on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload heat2d|heat1d|...] [--quick]

One "step" is one full pass of the headline workload: a 2D 5-point FTCS
solve on an 8192 x 8192 FP64 Dirichlet grid cut into 64 tiles of 1024^2
(one stream slot per tile, halo dependencies as futures), r = 0.2, 1000
time steps, a snapshot every 100 steps whose tiles are copied to the host
and reduced to L2 norms by host continuations while the GPU keeps stepping,
plus device-side norms.  Each step continues the evolution of the previous
one, so the work per step is identical.  The field (2 x 512 MiB) is larger
than L2, so no L2 flush is needed between steps.

Rank 0 prints one JSON line.  Under torchrun every rank runs an independent
replica on its own GPU (the workload has no exchange between GPUs), and
`value` sums the ranks' updates over the slowest rank's time.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

METRIC = "point-updates/s & HBM fraction of peak; graph/batched/adjoint vs plain, same GPU"
UNIT = "point-updates/s"

# headline workload
NY = NX = 8192
TILES = (8, 8)
R2D = 0.2
STEPS2D = 1000
EVERY = 100
# FP64 pipe operations of one 2D update in the pair-sum form, by step kind
# (canonical, scaled, closing; hxc_heat2d_step_kinds): its own anti-diagonal
# pair sum (the other one is shared with the point up-left), the sum of the
# two pair sums, then 2 fused multiply-adds (canonical), 1 (scaled), or a
# product and a fused multiply-add (closing)
OPS_BY_KIND_2D = (4, 3, 4)
BYTES_PER_UPDATE_2D = 16  # one 8-byte read and one 8-byte write


def bench_config(world):
    """The workload as both arms name it."""
    return {"workload": "heat2d FTCS 8192x8192 FP64, 64 tiles of 1024^2, r=0.2, "
                        "1000 steps, snapshot+host L2 norms every 100 steps",
            "parallelism": "replicas x%d" % world,
            "l2": "field 2x512 MiB > 126 MB L2 (no flush needed)"}


def load_peaks():
    p = os.path.join(HERE, "MEASURED_PEAKS.json")
    peaks = {"hbm_gbs": 6400.0, "hbm_source": "fallback", "sm_max_mhz": 2032.0, "sms": 148}
    if os.path.exists(p):
        d = json.load(open(p))
        peaks["hbm_gbs"] = float(d.get("hbm_gbs", 6400.0))
        peaks["hbm_source"] = "measured"
        peaks["sm_max_mhz"] = float(d.get("sm_max_mhz", 2032.0))
    # nominal FP64 pipe: 2 operations (DADD / DMUL / DFMA) per clock per SM on
    # B300; replaced by the measured rate when a device is at hand
    peaks["fp64_nominal_gops"] = 2 * peaks["sms"] * peaks["sm_max_mhz"] / 1e3
    peaks["fp64_gops"] = peaks["fp64_nominal_gops"]
    peaks["fp64_source"] = "nominal: 2 ops/clk/SM x 148 SMs x %.0f MHz" % peaks["sm_max_mhz"]
    peaks["fp32_nominal_gops"] = 128 * peaks["sms"] * peaks["sm_max_mhz"] / 1e3
    peaks["fp32_gops"] = peaks["fp32_nominal_gops"]
    peaks["fp32_source"] = "nominal: 128 ops/clk/SM x 148 SMs x %.0f MHz" % peaks["sm_max_mhz"]
    return peaks


def measure_pipes(dev, peaks):
    """The FP64 and FP32 pipe rates measured on this device now
    (hxc_pipe_rate: chains of one instruction, CUDA-event timed), which
    become the peaks of the arithmetic-bound rooflines."""
    from paper_1810_11482_b300 import hxc
    res = {}
    for name, kind in (("f64_fma", hxc.HXC_PIPE_F64_FMA), ("f64_add", hxc.HXC_PIPE_F64_ADD),
                       ("f32_fma", hxc.HXC_PIPE_F32_FMA)):
        # the best of three (~0.1 s each): a single run can start before the
        # SM clock has come up from idle
        runs = [hxc.pipe_rate(dev, kind) for _ in range(3)]
        ops, mhz = max(runs)
        res[name] = {"gops": ops / 1e9, "sm_mhz": mhz,
                     "per_sm_clock": ops / (dev.sm_count * mhz * 1e6) if mhz > 0 else None,
                     "runs_gops": [round(o / 1e9, 1) for o, _ in runs]}
    # the rate per SM clock is what the stream measures; the peak is that rate
    # at the maximum SM clock, which the timed regions run at (their clock
    # record says so), whatever clock the short measurement happened to see
    def at_max(r):
        pc = r["per_sm_clock"]
        return pc * dev.sm_count * peaks["sm_max_mhz"] / 1e3 if pc else r["gops"]

    peaks["fp64_gops"] = at_max(res["f64_fma"])
    peaks["fp64_source"] = ("measured here: FP64 FMA stream (hxc_pipe_rate), %.3f ops per SM "
                            "clock (%.1f Gop/s at the %.0f MHz it ran at) x %d SMs x %.0f MHz; "
                            "nominal %.1f Gop/s" % (res["f64_fma"]["per_sm_clock"] or 0.0,
                                                    res["f64_fma"]["gops"],
                                                    res["f64_fma"]["sm_mhz"], dev.sm_count,
                                                    peaks["sm_max_mhz"],
                                                    peaks["fp64_nominal_gops"]))
    peaks["fp32_gops"] = at_max(res["f32_fma"])
    peaks["fp32_source"] = ("measured here: FP32 FMA stream (hxc_pipe_rate), %.2f ops per SM "
                            "clock (%.1f Gop/s at the %.0f MHz it ran at) x %d SMs x %.0f MHz; "
                            "nominal %.1f Gop/s" % (res["f32_fma"]["per_sm_clock"] or 0.0,
                                                    res["f32_fma"]["gops"],
                                                    res["f32_fma"]["sm_mhz"], dev.sm_count,
                                                    peaks["sm_max_mhz"],
                                                    peaks["fp32_nominal_gops"]))
    peaks["pipes"] = res
    return res


class Clocks:
    """Samples SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                mhz.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(n)
        if not mhz:
            return None
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(mhz)}


def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo", init_method="env://")
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def allmax(pg, x):
    if pg is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def allsum(pg, x):
    if pg is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


# ----------------------------------------------------------------- our arm

class Timer:
    """CUDA events on one stream slot of the device; the slot waits for the
    measured future before the end event is recorded."""

    def __init__(self, dev, slot=0):
        import ctypes
        from paper_1810_11482_b300 import hxc
        self.hxc = hxc
        self.dev = dev
        self.stream = dev.stream(slot)
        self.cudart = ctypes.CDLL("libcudart.so.13")
        self.ev = [ctypes.c_void_p(), ctypes.c_void_p()]
        for e in self.ev:
            assert self.cudart.cudaEventCreate(ctypes.byref(e)) == 0
        self.ctypes = ctypes

    def start(self):
        """Records the start event and returns a future the timed work must
        depend on."""
        assert self.cudart.cudaEventRecord(self.ev[0], self.stream) == 0
        out = self.hxc.c_fut()
        self.hxc.check(self.hxc.lib().hxc_future_from_stream(self.dev.h, self.stream,
                                                            self.ctypes.byref(out)))
        return self.hxc.Future(out.value)

    def stop(self, fut):
        self.hxc.check(self.hxc.lib().hxc_future_stream_wait(fut.h, self.stream))
        assert self.cudart.cudaEventRecord(self.ev[1], self.stream) == 0
        assert self.cudart.cudaEventSynchronize(self.ev[1]) == 0
        ms = self.ctypes.c_float()
        assert self.cudart.cudaEventElapsedTime(self.ctypes.byref(ms), self.ev[0], self.ev[1]) == 0
        return ms.value


def ours(args, world, rank, local, pg):
    from paper_1810_11482_b300 import hxc, synth
    devs = hxc.get_all_devices(2, 0)
    if not devs:
        raise RuntimeError("no CUDA device visible")
    dev = devs[local % len(devs)]
    peaks = load_peaks()
    measure_pipes(dev, peaks)
    T = TILES[0] * TILES[1]
    nsnap = STEPS2D // EVERY
    u0 = synth.bumps2d(NY, NX, seed=2)
    field = u0.nbytes
    u, tmp = dev.buffer(field), dev.buffer(field)
    u.write(u0).get()
    hn = np.zeros(nsnap * T)
    gn = np.zeros(nsnap * T)
    upd = NY * NX * STEPS2D
    timer = Timer(dev, 0)
    launches = [0]

    def one(mode, deps=()):
        cfg = hxc.heat2d_cfg(NY, NX, TILES[0], TILES[1], R2D, STEPS2D, EVERY, mode, hn, gn)
        f, fr, st = hxc.heat2d_run(dev, u, tmp, cfg, deps, field_ready=True)
        # a pass that waits on the previous pass's host norms (snapshot ring
        # reuse) is issued later from the worker pool and cannot fill the
        # caller's counters; every pass issues the same launches, so the
        # count of a pass issued directly stands for each of them
        launches[0] = max(launches[0], st.kernel_launches)
        return f, fr

    def timed(mode, k, w):
        for _ in range(w):
            f, _ = one(mode)
            f.get()
        dev.synchronize()
        barrier(pg)
        launches[0] = 0
        start = timer.start()
        ready = start
        alls = []
        for _ in range(k):
            # the next pass starts as soon as the field is final; the host
            # norms of this pass overlap with it
            f, ready = one(mode, deps=[ready])
            alls.append(f)
        ms = timer.stop(hxc.when_all(alls))
        barrier(pg)
        return ms, launches[0] * k

    best_mode = args.mode
    clocks = Clocks(local)
    clocks.start()
    ms, n_launch = timed(best_mode, args.steps, args.warmup)
    clk = clocks.stop()
    ms_max = allmax(pg, ms)
    total_upd = allsum(pg, upd * args.steps)
    value = total_upd / (ms_max / 1e3)

    # the paper's timing protocol (Sec. 5): 11 runs, the first dropped, mean of
    # the other 10 and their minimum
    protocol = None
    if not args.quick:
        runs = [timed(best_mode, 1, 0)[0] for _ in range(11)]
        protocol = {"runs": 11, "mean_ms_of_last_10": statistics.mean(runs[1:]),
                    "min_ms_of_last_10": min(runs[1:]), "first_ms": runs[0]}

    # overlap of the pass: the device work, the snapshot copies and the host
    # norms each measured alone, against the whole pass
    overlap = None
    if not args.quick:
        cfgk = hxc.heat2d_cfg(NY, NX, TILES[0], TILES[1], R2D, STEPS2D, EVERY, best_mode, None, gn)
        fk, _ = hxc.heat2d_run(dev, u, tmp, cfgk)
        fk.get()
        start = timer.start()
        fk, _ = hxc.heat2d_run(dev, u, tmp, cfgk, deps=[start])
        t_dev = timer.stop(fk)
        snap = hxc.host_empty((NY, NX))
        u.read(snap).get()
        t0 = time.perf_counter()
        for _ in range(nsnap):
            u.read(snap).get()
        t_copy = (time.perf_counter() - t0) * 1e3
        tiles = [np.ascontiguousarray(snap[i * (NY // TILES[0]):(i + 1) * (NY // TILES[0]),
                                           j * (NX // TILES[1]):(j + 1) * (NX // TILES[1])])
                 for i in range(TILES[0]) for j in range(TILES[1])]
        hxc.host_norms(tiles)
        t0 = time.perf_counter()
        for _ in range(nsnap):
            hxc.host_norms(tiles)
        t_host = (time.perf_counter() - t0) * 1e3
        t_total = ms_max / args.steps
        overlap = {"total_ms": t_total, "device_ms": t_dev, "snapshot_copies_ms": t_copy,
                   "host_norms_ms": t_host,
                   "efficiency": max(t_dev, t_copy, t_host) / t_total}

    # per-mode comparison (plain per-partition launches vs graph vs fused)
    modes = {}
    if not args.quick:
        for mode in ("plain", "graph", "fused"):
            mms, ml = timed(mode, 1, 1)
            modes[mode] = {"updates_per_s": upd / (mms / 1e3), "ms": mms, "launches": ml}

    # roofline of the dominant kernel: back-to-back whole-domain step launches
    rsteps = 200
    cfg = hxc.heat2d_cfg(NY, NX, 1, 1, R2D, rsteps, 0, "fused", None, None)
    f, _ = hxc.heat2d_run(dev, u, tmp, cfg)
    f.get()
    start = timer.start()
    f, st = hxc.heat2d_run(dev, u, tmp, cfg, deps=[start])
    kms = timer.stop(f) / rsteps
    upd_launch = NY * NX
    kinds = hxc.heat2d_step_kinds(cfg)
    ops_upd = sum(n * o for n, o in zip(kinds, OPS_BY_KIND_2D)) / float(sum(kinds))
    ach_gops = upd_launch * ops_upd / (kms / 1e3) / 1e9
    ach_gbs = upd_launch * BYTES_PER_UPDATE_2D / (kms / 1e3) / 1e9
    traffic = None
    tp = os.path.join(HERE, "profiles", "heat2d_traffic.json")
    if os.path.exists(tp):
        traffic = json.load(open(tp)).get("bytes_per_launch")
    roof = {"bound": "alu", "achieved": ach_gops, "peak": peaks["fp64_gops"], "unit": "Gop/s",
            "frac": ach_gops / peaks["fp64_gops"], "traffic": traffic,
            "kernel": "k_heat2d<2> (whole 8192^2 field, one step per launch, %.3f FP64 "
                      "ops/update: %d scaled steps of 3, %d closing steps of 4)"
                      % (ops_upd, kinds[1], kinds[2] + kinds[0]),
            "ops_per_update": ops_upd, "step_kinds": {"canonical": kinds[0], "scaled": kinds[1],
                                                      "closing": kinds[2]},
            "ms_per_launch": kms,
            "peak_source": peaks["fp64_source"], "nominal_peak": peaks["fp64_nominal_gops"],
            "frac_of_nominal": ach_gops / peaks["fp64_nominal_gops"],
            "hbm": {"achieved_gbs": ach_gbs, "peak_gbs": peaks["hbm_gbs"],
                    "frac": ach_gbs / peaks["hbm_gbs"], "peak_source": peaks["hbm_source"]}}

    # end to end through the host entry points: every step uploads the field
    # from pinned host memory and downloads the result, both inside the timed
    # region.  The headline form issues the steps back to back through the
    # asynchronous entry point (a step's copies overlap its neighbours'
    # stencil steps, as a serving loop would); the synchronous entry point,
    # one call after the other, is reported beside it.
    e2e = None
    if not args.quick:
        hu = hxc.host_empty((NY, NX))
        hu[:] = u0
        hos = [hxc.host_empty((NY, NX)) for _ in range(2)]
        norm_sets = [(np.zeros(nsnap * T), np.zeros(nsnap * T)) for _ in range(2)]
        cfgs = [hxc.heat2d_cfg(NY, NX, TILES[0], TILES[1], R2D, STEPS2D, EVERY, best_mode, a, b)
                for a, b in norm_sets]
        k = max(2, min(args.steps, 20))  # the steps of the resident loop (at most 20)
        for i in range(2):  # warm-up: both device field pairs allocated
            f, _ = hxc.heat2d_run_host_async(dev, hu.ctypes.data, hos[i].ctypes.data, cfgs[i])
            f.get()
        barrier(pg)
        t0 = time.perf_counter()
        futs, sts = [], []
        for i in range(k):
            f, st = hxc.heat2d_run_host_async(dev, hu.ctypes.data, hos[i % 2].ctypes.data,
                                              cfgs[i % 2])
            futs.append(f)
            sts.append(st)
        for f in futs:
            f.get()
        el = allmax(pg, time.perf_counter() - t0)
        ks = max(1, min(args.steps, 3))
        barrier(pg)
        t0 = time.perf_counter()
        for _ in range(ks):
            st_s = hxc.heat2d_run_host(dev, hu.ctypes.data, hos[0].ctypes.data, cfgs[0])
        el_s = allmax(pg, time.perf_counter() - t0)
        # a call issued while the one two before it is still running is
        # issued later from the worker pool and cannot fill the caller's
        # counters; every call copies the same bytes, so the fullest count
        # stands for each of them
        e2e = {"value": allsum(pg, upd * k) / el, "unit": UNIT,
               "h2d_bytes_per_step": int(max(x.h2d_bytes for x in sts)),
               "d2h_bytes_per_step": int(max(x.d2h_bytes for x in sts)),
               "steps": k, "api": "hxc_heat2d_run_host_async, steps issued back to back",
               "sync": {"value": allsum(pg, upd * ks) / el_s, "steps": ks,
                        "api": "hxc_heat2d_run_host, one call after the other",
                        "h2d_bytes_per_step": int(st_s.h2d_bytes),
                        "d2h_bytes_per_step": int(st_s.d2h_bytes)}}

    sec = None
    # the secondary workloads are reported by rank 0 only (no collective in
    # them), so the other replicas skip them
    if not args.quick and not args.no_secondary and rank == 0:
        sec = secondary(dev, timer, peaks)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(world), "launch_mode": best_mode,
        "roofline": roof, "gpu_launches": int(allsum(pg, n_launch)), "modes": modes,
        "clocks": clk, "e2e": e2e, "paper_protocol": protocol, "overlap": overlap,
        "pipe_peaks": peaks.get("pipes"), "secondary": sec,
    }
    if sec:
        out["secondary_summary"] = summarize(sec)
    return out


def summarize(sec):
    """The secondary workloads' key figures in a few numbers (kept at the end
    of the line, where a truncated log still shows them)."""
    r = lambda x: None if x is None else float("%.4g" % x)
    out = {}
    h1 = sec.get("heat1d_2^20_8parts_100steps_f64")
    if h1:
        out["heat1d_ms"] = {m: r(h1[m]["ms"]) for m in ("plain", "graph", "fused")}
    h3 = sec.get("heat3d_512^3_200steps_f32")
    if h3:
        out["heat3d_ms"] = {m: r(h3[m]["ms"]) for m in ("plain", "graph", "fused")}
        out["heat3d_4step_launch"] = {"ms": r(h3["roofline"]["ms_per_launch"]),
                                      "hbm_frac": r(h3["roofline"]["frac"])}
        out["heat3d_1step_launch_hbm_frac"] = r(h3["roofline_one_step"]["frac"])
    b = sec.get("batch_4096_problems_50steps_f64")
    if b:
        out["batch_ms"] = {m: r(b[m]["ms"]) for m in ("plain", "graph", "fused")}
        out["batch_fp64_frac"] = r(b["roofline"]["frac"])
    a = sec.get("adjoint_2048^2_500steps_f64")
    if a:
        out["adjoint_ms"] = {m: r(a[m]["ms"]) for m in ("forward", "plain", "graph", "fused")}
        out["gradient_over_forward"] = r(a["gradient_over_forward_time"])
        out["adjoint_fused_speedup_vs_plain"] = r(a["fused"]["speedup_vs_plain"])
        t = a.get("from_tape")
        if t:
            out["adjoint_from_tape_ms"] = {m: r(t[m]["ms"]) for m in ("forward_tape", "plain",
                                                                      "graph", "fused")}
            out["gradient_from_tape_over_forward"] = r(t["gradient_over_forward_time"])
            e = t.get("every_state")
            if e:
                out["adjoint_every_state_tape_ms"] = {m: r(e[m]["ms"]) for m in (
                    "forward_tape", "plain", "graph", "fused")}
                out["gradient_every_state_over_forward"] = r(e["gradient_over_forward_time"])
    return out


def fp64_roof(ops, ms, peaks, what):
    ach = ops / (ms / 1e3) / 1e9
    return {"bound": "alu", "achieved": ach, "peak": peaks["fp64_gops"], "unit": "Gop/s",
            "frac": ach / peaks["fp64_gops"], "count": what, "peak_source": peaks["fp64_source"]}


def secondary(dev, timer, peaks):
    """The other workloads of the path, each in every launch mode on the same
    GPU: updates/s per mode and the speed-up over the plain per-partition
    (or per-problem / unfused) launch path."""
    from paper_1810_11482_b300 import hxc, synth

    def timed_run(fn, reps=1, warm=1):
        for _ in range(warm):
            f = fn(None)
            f.get()
        start = timer.start()
        f = start
        for _ in range(reps):
            f = fn(f)
        return timer.stop(f) / reps

    def speedups(res, modes=("plain", "graph", "fused")):
        for m in modes:
            res[m]["speedup_vs_plain"] = res["plain"]["ms"] / res[m]["ms"]

    out = {}
    # 1D periodic, 2^20 points in 8 partitions, r = 1/4, 100 steps
    n, parts, st1 = 1 << 20, 8, 100
    u0 = synth.heat1d_input(n, seed=1)
    u, t = dev.buffer(n * 8), dev.buffer(n * 8)
    u.write(u0).get()
    res = {}
    for mode in ("plain", "graph", "fused"):
        ms = timed_run(lambda d, m=mode: hxc.heat1d_run(dev, u, t, n, parts, 0.25, st1, m, 0,
                                                         deps=[d] if d else ())[0], reps=5, warm=2)
        res[mode] = {"ms": ms, "updates_per_s": n * st1 / (ms / 1e3)}
    speedups(res)
    # FP64 operations per update by step kind (canonical, scaled, closing;
    # hxc_heat1d_step_kinds): the sum ul + ur, then 2 FMAs, 1, or a product
    # and an FMA
    k1 = hxc.heat1d_step_kinds(0.25, st1)
    ops1 = sum(c * o for c, o in zip(k1, (3, 2, 3)))
    res["step_kinds"] = {"canonical": k1[0], "scaled": k1[1], "closing": k1[2]}
    res["roofline"] = fp64_roof(ops1 * n, res["graph"]["ms"], peaks,
                                "%.2f FP64 operations per update (%d scaled steps of 2, %d "
                                "closing of 3), graph mode" % (ops1 / st1, k1[1], k1[2] + k1[0]))
    out["heat1d_2^20_8parts_100steps_f64"] = res

    # 3D periodic FP32 512^3, r = 0.15, 200 steps, 4 steps per launch
    n3, st3 = 512, 200
    u3 = synth.heat3d_input(n3, seed=3)
    a, b = dev.buffer(u3.nbytes), dev.buffer(u3.nbytes)
    a.write(u3).get()
    res = {}
    for mode, spl in (("plain", 1), ("graph", 4), ("fused", 4)):
        ms = timed_run(lambda d, m=mode, k=spl: hxc.heat3d_run(dev, a, b, (n3, n3, n3), 0.15, st3, m, k,
                                                                deps=[d] if d else ())[0])
        res[mode] = {"ms": ms, "updates_per_s": n3 ** 3 * st3 / (ms / 1e3), "steps_per_launch": spl}
    speedups(res)
    # per-launch HBM roofline of the 4-step kernel (algorithmic: read + write once)
    launch_ms = res["fused"]["ms"] / (st3 / 4)
    gbs = 2 * u3.nbytes / (launch_ms / 1e3) / 1e9
    traffic3 = None
    tp3 = os.path.join(HERE, "profiles", "heat3d_traffic.json")
    if os.path.exists(tp3):
        traffic3 = json.load(open(tp3)).get("bytes_per_launch")
    res["roofline"] = {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                       "frac": gbs / peaks["hbm_gbs"], "ms_per_launch": launch_ms,
                       "traffic": traffic3,
                       "kernel": "k_heat3d_v7<4> (4 steps of the whole 512^3 field per launch, packed narrow tiles, TMA-fed interior regions)",
                       "effective_gbs_1step_equiv": 2 * u3.nbytes * st3 / (res["fused"]["ms"] / 1e3) / 1e9}
    # the one-step launches of plain mode (streaming kernel): read + write once per step
    ms1 = res["plain"]["ms"] / st3
    gbs1 = 2 * u3.nbytes / (ms1 / 1e3) / 1e9
    res["roofline_one_step"] = {"bound": "hbm", "achieved": gbs1, "peak": peaks["hbm_gbs"],
                                "unit": "GB/s", "frac": gbs1 / peaks["hbm_gbs"], "ms_per_launch": ms1,
                                "kernel": "k_heat3d_s1 (one step of the whole 512^3 field per launch)"}
    out["heat3d_512^3_200steps_f32"] = res
    del u3

    # batch: 4096 variable-diffusivity problems, 50 steps
    sides, offs, kap, ub, cs = synth.batch_input(nprob=4096, seed=4)
    total = ub.size
    bu, bk = dev.buffer(total * 8), dev.buffer(total * 8)
    bk.write(kap).get()
    res, outs = {}, {}
    for mode in ("plain", "graph", "fused"):
        bu.write(ub).get()
        ms = timed_run(lambda d, m=mode: hxc.varcoef_batch_run(dev, bu, bk, sides, cs, 50, m,
                                                                deps=[d] if d else ())[0], warm=1)
        chk = np.empty(1 << 16)
        bu.read_sync(chk, off=(total // 2) * 8)
        outs[mode] = chk
        res[mode] = {"ms": ms, "updates_per_s": total * 50 / (ms / 1e3)}
    speedups(res)
    res["bitwise_equal_modes"] = bool(all(np.array_equal(outs["plain"], outs[m]) for m in outs))
    res["points"] = int(total)
    res["roofline"] = fp64_roof(5 * total * 50, res["fused"]["ms"], peaks,
                                "5 FP64 operations per update (coefficient form), fused mode")
    out["batch_4096_problems_50steps_f64"] = res
    del kap, ub

    # adjoint: 2048^2, 500 steps, sqrt(n) checkpointing
    n2, st4, c = 2048, 500, 0.15
    kref, kap, u0, _ = synth.adjoint_input(n2)
    b0, bkr, bkk = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)
    b0.write(u0).get()
    bkr.write(kref).get()
    bkk.write(kap).get()
    tgt, uT, lam, lb = (dev.buffer(u0.nbytes), dev.buffer(u0.nbytes), dev.buffer(u0.nbytes),
                        dev.buffer(8))
    hxc.varcoef_forward_run(dev, b0, bkr, n2, n2, c, st4, tgt)[0].get()
    hxc.varcoef_forward_run(dev, b0, bkk, n2, n2, c, st4, uT)[0].get()
    hxc.sqerr_seed(dev, uT, tgt, lam, lb, n2 * n2).get()
    gk, gu = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)
    res = {}
    ms = timed_run(lambda d: hxc.varcoef_forward_run(dev, b0, bkk, n2, n2, c, st4, uT,
                                                     deps=[d] if d else ())[0])
    res["forward"] = {"ms": ms, "updates_per_s": n2 * n2 * st4 / (ms / 1e3)}
    for mode in ("plain", "graph", "fused"):
        ms = timed_run(lambda d, m=mode: hxc.varcoef_adjoint_run(dev, b0, bkk, lam, n2, n2, c, st4, gk, gu,
                                                                  None, 0, m, deps=[d] if d else ())[0])
        res[mode] = {"ms": ms, "gradient_updates_per_s": n2 * n2 * st4 / (ms / 1e3)}
    speedups(res)
    res["gradient_over_forward_time"] = res["fused"]["ms"] / res["forward"]["ms"]
    # the training-step form: the forward pass keeps its checkpoint tape and
    # the gradient starts from it (no second forward pass)
    tape = dev.buffer(hxc.varcoef_tape_states(st4) * u0.nbytes)
    ms = timed_run(lambda d: hxc.varcoef_forward_tape(dev, b0, bkk, n2, n2, c, st4, uT, tape,
                                                      deps=[d] if d else ())[0])
    tres = {"forward_tape": {"ms": ms}}
    for mode in ("plain", "graph", "fused"):
        ms = timed_run(lambda d, m=mode: hxc.varcoef_adjoint_tape(dev, tape, bkk, lam, n2, n2, c, st4,
                                                                   gk, gu, 0, m, deps=[d] if d else ())[0])
        tres[mode] = {"ms": ms, "speedup_vs_plain": None}
    for m in ("plain", "graph", "fused"):
        tres[m]["speedup_vs_plain"] = tres["plain"]["ms"] / tres[m]["ms"]
    tres["gradient_over_forward_time"] = tres["fused"]["ms"] / res["forward"]["ms"]
    tres["training_step_ms"] = tres["forward_tape"]["ms"] + tres["fused"]["ms"]
    tres["training_step_ms_without_tape"] = res["forward"]["ms"] + res["fused"]["ms"]
    tres["roofline"] = fp64_roof(16 * n2 * n2 * st4, tres["fused"]["ms"], peaks,
                                 "16 FP64 operations per cell-step: segment recompute 5, adjoint "
                                 "step 5, kappa-gradient face products 6; fused")
    del tape
    # every state on the tape (every = 1: 500 states, 16 GiB at 2048^2; the
    # memory the B300 has room for): the gradient recomputes nothing
    tape1 = dev.buffer(hxc.varcoef_tape_states(st4, 1) * u0.nbytes)
    ms = timed_run(lambda d: hxc.varcoef_forward_tape(dev, b0, bkk, n2, n2, c, st4, uT, tape1, 1,
                                                      deps=[d] if d else ())[0])
    ares = {"tape_bytes": hxc.varcoef_tape_states(st4, 1) * u0.nbytes, "forward_tape": {"ms": ms}}
    for mode in ("plain", "graph", "fused"):
        ms = timed_run(lambda d, m=mode: hxc.varcoef_adjoint_tape(dev, tape1, bkk, lam, n2, n2, c, st4,
                                                                   gk, gu, 1, m, deps=[d] if d else ())[0])
        ares[mode] = {"ms": ms, "speedup_vs_plain": None}
    for m in ("plain", "graph", "fused"):
        ares[m]["speedup_vs_plain"] = ares["plain"]["ms"] / ares[m]["ms"]
    ares["gradient_over_forward_time"] = ares["fused"]["ms"] / res["forward"]["ms"]
    ares["training_step_ms"] = ares["forward_tape"]["ms"] + ares["fused"]["ms"]
    ares["roofline"] = fp64_roof(11 * n2 * n2 * st4, ares["fused"]["ms"], peaks,
                                 "11 FP64 operations per cell-step: adjoint step 5, "
                                 "kappa-gradient face products 6; fused")
    tres["every_state"] = ares
    del tape1
    res["from_tape"] = tres
    res["roofline"] = fp64_roof(21 * n2 * n2 * st4, res["fused"]["ms"], peaks,
                                "21 FP64 operations per cell-step: forward with checkpoints 5, "
                                "segment recompute 5, adjoint step 5, kappa-gradient face "
                                "products 6; fused")
    res["forward"]["roofline"] = fp64_roof(5 * n2 * n2 * st4, res["forward"]["ms"], peaks,
                                           "5 FP64 operations per update")
    out["adjoint_2048^2_500steps_f64"] = res
    del b0, bkr, bkk, tgt, uT, lam, lb, gk, gu
    out["heat2d_streamed_8192_64tiles_f64"] = stream2d_bench(dev)
    out["partition_alg1_p4_f64"] = partition_bench(dev, timer)
    out["mandelbrot_png_f32"] = mandelbrot_bench(dev, timer, peaks)
    return out


def mandelbrot_frames(n, frames, max_iter):
    """Argument sets of a zoom sequence of `frames` n x n images towards the
    point -0.7436 + 0.1318i, the view halving in width from frame to frame
    (from [-2, 1] x [-1.5, 1.5])."""
    F = np.float32
    out = []
    cx, cy = -0.7436439, 0.1318259
    for f in range(frames):
        w = 3.0 * 0.5 ** f
        x0 = -2.0 + (cx + 2.0) * (1 - 0.5 ** f)
        y0 = -1.5 + (cy + 1.5) * (1 - 0.5 ** f)
        out.append((F(x0), F(y0), F(w / n), F(w / n), max_iter))
    return out


def mandelbrot_bench(dev, timer, peaks, sides=(1024, 2048, 4096, 8192), frames=8, max_iter=256,
                     level=1):
    """Sec. 5.1.3: for each image size, a sequence of `frames` images (a zoom)
    computed on the device, copied back and written as PNG files (zlib
    level 1); host-clock time of the sequence with each file written
    synchronously before the next image is issued, and with the writes as
    continuations that overlap the next images and one another.  Plus the
    kernel alone on the first frame of the largest size against the FP32
    issue rate."""
    import shutil
    import tempfile
    import time
    from paper_1810_11482_b300 import hxc
    tmp = tempfile.mkdtemp(prefix="hxc_mandel_")
    try:
        nmax = max(sides)
        bufs = [dev.buffer(nmax * nmax * 3) for _ in range(frames)]
        hosts = [hxc.host_empty(nmax * nmax * 3, np.uint8) for _ in range(frames)]
        res = {"frames": frames, "max_iter": max_iter, "zlib_level": level, "sizes": []}
        for n in sides:
            args = [hxc.mandelbrot_args(bufs[f], n, n, *fr) for f, fr in enumerate(mandelbrot_frames(n, frames, max_iter))]
            row = {"side": n, "image_bytes": 3 * n * n}
            for mode in ("sync", "async"):
                times = []
                for rep in range(3):
                    names = [os.path.join(tmp, "%s%d_%d_%d.png" % (mode, n, rep, f)) for f in range(frames)]
                    t0 = time.perf_counter()
                    futs = [hxc.mandelbrot_png(dev, a, hosts[f], names[f], level, mode == "async",
                                               slot=f % 4)
                            for f, a in enumerate(args)]
                    assert hxc.wait_all(futs) == hxc.HXC_OK
                    times.append((time.perf_counter() - t0) * 1e3)
                    for nm in names:  # new files every time: no truncation inside the timing
                        os.remove(nm)
                row[mode + "_ms"] = float(np.median(times[1:]))
            row["async_speedup"] = row["sync_ms"] / row["async_ms"]
            res["sizes"].append(row)
        # the kernel alone on the first frame of the largest size
        n = nmax
        cnt = dev.buffer(n * n * 4)
        fr = mandelbrot_frames(n, 1, max_iter)[0]
        dev.launch(hxc.HXC_K_MANDELBROT, hxc.mandelbrot_args(bufs[0], n, n, *fr, counts=cnt)).get()
        counts = np.empty(n * n, dtype=np.int32)
        cnt.read_sync(counts)
        a = hxc.mandelbrot_args(bufs[0], n, n, *fr)
        kms = []
        for _ in range(5):
            start = timer.start()
            kms.append(timer.stop(dev.launch(hxc.HXC_K_MANDELBROT, a, deps=[start])))
        kms = float(np.median(kms[1:]))
        # 7 FP32 operations per full iteration, 3 for the final escape test
        ops = 7.0 * counts.astype(np.float64).sum() + 3.0 * float((counts < max_iter).sum())
        peak = peaks["fp32_gops"]
        res["kernel"] = {"side": n, "ms": kms, "iterations": float(counts.astype(np.float64).sum()),
                         "roofline": {"bound": "alu", "achieved": ops / (kms / 1e3) / 1e9,
                                      "peak": peak, "unit": "Gop/s (FP32)",
                                      "frac": ops / (kms / 1e3) / 1e9 / peak,
                                      "peak_source": peaks["fp32_source"]}}
        return res
    finally:
        shutil.rmtree(tmp, ignore_errors=True)


def link_peak(dev, host_in, host_out, buf_in, buf_out, reps=4):
    """The host link alone: host_in copied to the device and buf_out copied to
    host_out at the same time (one copy each way, two stream slots); GB/s of
    both directions together, median of the repetitions after the first."""
    import time
    from paper_1810_11482_b300 import hxc
    ms = []
    for _ in range(reps):
        t0 = time.perf_counter()
        fw = buf_in.write(host_in, slot=0)
        fr = buf_out.read(host_out, slot=1)
        assert hxc.wait_all([fw, fr]) == hxc.HXC_OK
        ms.append((time.perf_counter() - t0) * 1e3)
    return (host_in.nbytes + host_out.nbytes) / (float(np.median(ms[1:])) / 1e3) / 1e9


def stream2d_bench(dev, n=8192, tiles=(8, 8), steps=6):
    """The 2D run streamed through the device every step (host-resident
    field, Algorithm 1 per step): host-clock time per step of the
    asynchronous tile futures and of the native sequential loop, and the host
    link throughput against the link measured alone."""
    import time
    from paper_1810_11482_b300 import hxc, synth
    a, b = hxc.host_empty((n, n)), hxc.host_empty((n, n))
    a[:] = synth.bumps2d(n, n, seed=2)
    res = {"field": [n, n], "tiles": list(tiles), "steps": steps}
    for seq in (False, True):
        hxc.heat2d_stream_run(dev, a, b, tiles, R2D, 2, seq)[0].get()
        t0 = time.perf_counter()
        f, st, _ = hxc.heat2d_stream_run(dev, a, b, tiles, R2D, steps, seq)
        f.get()
        ms = (time.perf_counter() - t0) * 1e3 / steps
        key = "sequential" if seq else "futures"
        res[key] = {"ms_per_step": ms, "updates_per_s": n * n / (ms / 1e3),
                    "host_link_gbs": (st.h2d_bytes + st.d2h_bytes) / steps / (ms / 1e3) / 1e9}
    res["futures_speedup"] = res["sequential"]["ms_per_step"] / res["futures"]["ms_per_step"]
    bi, bo = dev.buffer(a.nbytes), dev.buffer(a.nbytes)
    peak = link_peak(dev, a, b, bi, bo)
    ach = res["futures"]["host_link_gbs"]
    res["roofline"] = {"bound": "host link", "achieved": ach, "peak": peak, "unit": "GB/s",
                       "frac": ach / peak,
                       "peak_source": "measured here: the field in and out concurrently"}
    return res


def partition_bench(dev, timer, ms_exp=range(1, 9), parts=4):
    """Sec. 5.1.2 (Algorithm 1): host-clock time of the three loops (copy in,
    kernel, copy out, per partition) until the results are on the host, on
    the futures layer and as plain CUDA calls on the same streams, for
    n = 2^m * 1024 * 256 * 4; plus the device time of the kernels alone on
    resident data."""
    import time
    from paper_1810_11482_b300 import hxc, synth
    sizes = synth.partition_sizes(ms_exp, 256, parts)
    nmax = max(sizes)
    x_all, r_all = hxc.host_empty(nmax), hxc.host_empty(nmax)
    synth.partition_input(nmax, out=x_all)
    work, side = dev.buffer(nmax * 8), dev.buffer(nmax * 8)
    rows = []
    for m, n in zip(ms_exp, sizes):
        x, r = x_all[:n], r_all[:n]
        reps = max(3, min(20, (1 << 27) // n))
        res = {"m": m, "n": n}
        outs = {}
        for path in ("futures", "native"):
            def once():
                if path == "futures":
                    hxc.partition_run(dev, x, r, parts, work).get()
                else:
                    hxc.partition_run_native(dev, x, r, parts, work)
            once()
            best = []
            for _ in range(reps):
                t0 = time.perf_counter()
                once()
                best.append((time.perf_counter() - t0) * 1e3)
            res[path + "_ms"] = float(np.median(best))
            outs[path] = r[:: max(1, n // 65536)].copy()
        res["futures_over_native"] = res["futures_ms"] / res["native_ms"]
        res["bitwise_equal_paths"] = bool(np.array_equal(outs["futures"], outs["native"]))
        res["max_abs_err_vs_1"] = float(np.max(np.abs(r - 1.0)))
        res["host_link_gbs"] = 16.0 * n / (res["futures_ms"] / 1e3) / 1e9  # 8 B in + 8 B out
        # the kernels alone, data resident (a fresh copy of x before each timing)
        kms = []
        bounds = [i * n // parts for i in range(parts + 1)]
        for _ in range(3):
            work.write(x).get()
            start = timer.start()
            fs = [dev.launch(hxc.HXC_K_PARTITION,
                             hxc.hxc_partition_args(work.h, bounds[i + 1] - bounds[i], bounds[i]),
                             slot=i, deps=[start]) for i in range(parts)]
            kms.append(timer.stop(hxc.when_all(fs)))
        res["kernels_only_ms"] = float(np.median(kms))
        rows.append(res)
    n = nmax
    link_gbs = link_peak(dev, x_all, r_all, work, side)
    last = rows[-1]
    return {"sizes": rows,
            "roofline": {"bound": "host link", "achieved": last["host_link_gbs"], "peak": link_gbs,
                         "unit": "GB/s", "frac": last["host_link_gbs"] / link_gbs, "n": n,
                         "peak_source": "measured here: 8n bytes host->device and 8n bytes "
                                        "device->host copied concurrently on two streams"}}


def cpu_info():
    """Host CPU model and the number of logical CPUs this process may use."""
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    try:
        usable = len(os.sched_getaffinity(0))
    except AttributeError:
        usable = os.cpu_count()
    return {"cpu_model": model, "nproc": usable, "cpu_count": os.cpu_count()}


class OracleRun:
    """The oracle's 2D FTCS stepping routine on the headline field, stepping
    two caller-owned arrays (both touched before any timing, so no allocation,
    copy or page fault is inside a timed call).  omp=True is the OpenMP build
    of the same loop (all host threads), omp=False the serial build."""

    def __init__(self, omp):
        import oracle
        from paper_1810_11482_b300 import synth
        self.oracle = oracle
        self.omp = omp
        self.a = synth.bumps2d(NY, NX, seed=2)
        self.b = np.zeros_like(self.a)
        self.threads = oracle.threads(omp)

    def run(self, steps):
        """Advances the field `steps` time steps in one call; seconds taken."""
        t0 = time.perf_counter()
        res = self.oracle.heat2d_steps(self.a, self.b, R2D, steps, omp=self.omp)
        el = time.perf_counter() - t0
        if res is self.b:
            self.a, self.b = self.b, self.a
        return el

    def steps_for(self, seconds, cap):
        """Time steps per call that take about `seconds` (one calibration step)."""
        t1 = self.run(1)
        return max(1, min(cap, int(round(seconds / max(t1, 1e-6)))))


def oracle_protocol(warmup, steps):
    """The oracle (OpenMP build, all host threads) timed on the headline
    workload: each bench step advances the full 8192^2 field `k` = 10 time
    steps in one call (0.2-0.3 s on an 8-core host), continuing the evolution; `warmup`
    untimed bench steps, then the mean of `steps` timed ones.  The serial
    build is timed once beside it.  The field's far tails pass through
    subnormal values, which the host's FP64 unit handles slowly, so the rate
    depends on the stretch of the evolution sampled: the benchmark's CPU
    baseline and its reference arm therefore take the same stretch."""
    info = cpu_info()
    o = OracleRun(True)
    k = 10
    times = []
    for i in range(warmup + steps):
        el = o.run(k)
        if i >= warmup:
            times.append(el)
    per = statistics.mean(times)
    threads = o.threads
    del o
    st = OracleRun(False)
    ks = st.steps_for(2.0, 20)
    el_s = st.run(ks)
    return {"value": NY * NX * k / per, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "full 8192^2 field from u0, %d + %d bench steps of %d time steps each "
                      "(one call each, continuing the evolution), OpenMP build (row loop on %d "
                      "threads; C, -O2, no FMA)" % (warmup, steps, k, threads),
            "seconds_per_step": per, "time_steps_per_step": k,
            "seconds_per_step_min_median_max": [min(times), statistics.median(times), max(times)],
            "note": "the host is shared with other GPUs' jobs: its timings vary from run to run",
            "single_thread": {"value": NY * NX * ks / el_s, "cores": 1,
                              "sample": "full field from u0, %d time steps in one call" % ks},
            **info}


def cpu_baseline(warmup, steps):
    """The oracle as it stands on the host cores, on the same bounded sample
    as the reference arm (oracle_protocol)."""
    return oracle_protocol(warmup, steps)


def reference(args, world, rank):
    """The reference arm: the oracle on the headline workload
    (oracle_protocol); under torchrun rank 0 alone runs it."""
    if rank != 0:
        return None
    b = oracle_protocol(args.warmup, args.steps)
    value = b["value"]
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": b["seconds_per_step"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": bench_config(world), "cpu_baseline": b,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="fused", choices=["plain", "graph", "fused"])
    ap.add_argument("--quick", action="store_true", help="skip mode comparison and e2e")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the 1D/3D/batch/adjoint comparisons")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local, pg = dist_setup(args.gpus)
    if args.impl == "reference":
        out = reference(args, world, rank)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    out = ours(args, world, rank, local, pg)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args.warmup, args.steps)
        if "secondary_summary" in out:  # keep it last
            out["secondary_summary"] = out.pop("secondary_summary")
        print(json.dumps(out), flush=True)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
