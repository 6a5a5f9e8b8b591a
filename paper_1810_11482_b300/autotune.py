"""Autotuner: measures the launch-shape knobs of the kernels on the current
GPU and writes them to a JSON tuning cache.

    python -m paper_1810_11482_b300.autotune [--out PATH] [--quick]

Knobs (see hxc_tune_set in include/hxc.h) change speed only -- every value
gives bit-identical results -- so the search simply times each candidate on
representative synthetic work with CUDA events and keeps the fastest: launch
shapes of the 2D, 3D, 1D and batch kernels, the 3D kernel form, the steps
per fused launch of the 1D and 3D runs, and the side below which the batch
kernel keeps a problem in shared memory.  The
cache maps "sm_<major><minor>" to {knob: value}; the library loads it when it
first opens a device (HXC_TUNE_CACHE, else tune_cache.json beside
libhxc.so).
"""
import argparse
import ctypes
import json
import os

import numpy as np

from . import hxc, synth

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(HERE, "tune_cache.json")


class _Timer:
    def __init__(self, dev):
        self.dev = dev
        self.stream = dev.stream(0)
        self.rt = ctypes.CDLL("libcudart.so.13")
        self.ev = [ctypes.c_void_p(), ctypes.c_void_p()]
        for e in self.ev:
            assert self.rt.cudaEventCreate(ctypes.byref(e)) == 0

    def time(self, issue, reps=3):
        """Best time in ms of issue(deps) -> Future, after one warm-up."""
        issue(()).get()
        best = float("inf")
        for _ in range(reps):
            assert self.rt.cudaEventRecord(self.ev[0], ctypes.c_void_p(self.stream)) == 0
            out = hxc.c_fut()
            hxc.check(hxc.lib().hxc_future_from_stream(self.dev.h, ctypes.c_void_p(self.stream),
                                                      ctypes.byref(out)))
            f = issue((hxc.Future(out.value),))
            hxc.check(hxc.lib().hxc_future_stream_wait(f.h, ctypes.c_void_p(self.stream)))
            assert self.rt.cudaEventRecord(self.ev[1], ctypes.c_void_p(self.stream)) == 0
            assert self.rt.cudaEventSynchronize(self.ev[1]) == 0
            ms = ctypes.c_float()
            self.rt.cudaEventElapsedTime(ctypes.byref(ms), self.ev[0], self.ev[1])
            best = min(best, ms.value)
        return best


def _search(timer, knobs, issue, log):
    """Times every combination of knob values (dict key -> list) and sets
    the fastest; returns {key: value}."""
    keys = list(knobs)
    best, best_ms = None, float("inf")

    def rec(i, chosen):
        nonlocal best, best_ms
        if i == len(keys):
            for k, v in chosen.items():
                hxc.tune_set(k, v)
            ms = timer.time(issue)
            log(f"  {chosen} {ms:.3f} ms")
            if ms < best_ms:
                best, best_ms = dict(chosen), ms
            return
        for v in knobs[keys[i]]:
            chosen[keys[i]] = v
            rec(i + 1, chosen)

    rec(0, {})
    for k, v in best.items():
        hxc.tune_set(k, v)
    return best


def tune(quick=False, log=print):
    dev = hxc.get_all_devices(2, 0)[0]
    timer = _Timer(dev)
    result = {}
    # 2D: rows per warp x compiled occupancy (fused whole-field steps)
    n = 4096 if quick else 8192
    u0 = synth.bumps2d(n, n, seed=2)
    u, t = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)
    u.write(u0).get()
    cfg = hxc.heat2d_cfg(n, n, 1, 1, 0.2, 100, 0, "fused", None, None)
    log("heat2d")
    result.update(_search(timer, {"heat2d.occupancy": [4, 5, 6], "heat2d.rows": [8, 16, 32, 64]},
                          lambda d: hxc.heat2d_run(dev, u, t, cfg, d)[0], log))
    del u, t
    # 3D: z chunks of the 4-step kernel
    n3 = 256 if quick else 512
    u3 = synth.uniform(6, n3 ** 3).astype(np.float32)
    a, b = dev.buffer(u3.nbytes), dev.buffer(u3.nbytes)
    a.write(u3).get()
    log("heat3d")
    run3 = lambda d: hxc.heat3d_run(dev, a, b, (n3, n3, n3), 0.15, 8, "fused", 4, d)[0]
    hxc.tune_set("heat3d.zchunks", 0)
    best3 = _search(timer, {"heat3d.variant": [2, 3, 4, 6, 7]}, run3, log)
    # the z split applies to the form that cuts z into chunks (2); forms 3, 4,
    # 6 and 7 split the (region, plane) pairs evenly over the SMs themselves
    if best3["heat3d.variant"] <= 2:
        best3.update(_search(timer, {"heat3d.zchunks": [0, 1, 2, 3, 4, 6, 8]}, run3, log))
    result.update(best3)
    # one-step launches (PLAIN mode) choose their form separately
    run31 = lambda d: hxc.heat3d_run(dev, a, b, (n3, n3, n3), 0.15, 8, "plain", 1, d)[0]
    result.update(_search(timer, {"heat3d.variant1": [2, 3, 4, 5, 6, 7]}, run31, log))
    # steps per fused launch when the caller passes 0 (12 steps: whole
    # launches for 2, 3 and 4)
    run3t = lambda d: hxc.heat3d_run(dev, a, b, (n3, n3, n3), 0.15, 12, "fused", 0, d)[0]
    result.update(_search(timer, {"heat3d.steps_per_launch": [2, 3, 4]}, run3t, log))
    del a, b
    # 1D: CTAs per partition of the temporally blocked kernel
    n1 = 1 << 20
    v0 = synth.heat1d_input(n1, seed=1)
    p, q = dev.buffer(n1 * 8), dev.buffer(n1 * 8)
    p.write(v0).get()
    log("heat1d")
    run1 = lambda d: hxc.heat1d_run(dev, p, q, n1, 8, 0.25, 100, "fused", 0, d)[0]
    result.update(_search(timer, {"heat1d.tb_ctas": [0, 8, 12, 16, 18, 24, 32]}, run1, log))
    # steps per fused launch (the caller's 0): all steps, or launches of
    # fewer steps (smaller halos, more launches)
    result.update(_search(timer, {"heat1d.steps_per_launch": [0, 10, 25, 50]}, run1, log))
    # batch: CTAs per SM of the persistent kernel, on the full batch (its
    # largest problems set the critical path of the
    # persistent kernel, so a subset would tune for a different balance)
    sides, offs, kap, ub, cs = synth.batch_input(nprob=256 if quick else 4096, seed=4)
    bu, bk = dev.buffer(ub.nbytes), dev.buffer(kap.nbytes)
    bu.write(ub).get()
    bk.write(kap).get()
    log("batch")
    runb = lambda d: hxc.varcoef_batch_run(dev, bu, bk, sides, cs, 50, "fused", d)[0]
    result.update(_search(timer, {"batch.block": [256, 512], "batch.ctas_per_sm": [1, 2, 3, 4]},
                          runb, log))
    # shared-memory residency threshold of small problems (the CTAs per SM
    # chosen above must still fit: 2 side^2 doubles per CTA)
    fit = [v for v in (0, 32, 40, 48, 59)
           if 2 * v * v * 8 * result["batch.ctas_per_sm"] <= 200 * 1024]
    result.update(_search(timer, {"batch.smem_side": fit}, runb, log))
    return dev, result


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.environ.get("HXC_TUNE_CACHE", DEFAULT_CACHE))
    ap.add_argument("--quick", action="store_true")
    a = ap.parse_args()
    dev, result = tune(a.quick)
    arch = "sm_%d%d" % (dev.major, dev.minor)
    cache = {}
    if os.path.exists(a.out):
        with open(a.out) as fh:
            cache = json.load(fh)
    cache[arch] = {k: int(v) for k, v in result.items()}
    with open(a.out, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    print(arch, cache[arch], "->", a.out)


if __name__ == "__main__":
    main()
