"""The autotuner end to end: a quick search on this GPU, its cache written
and loaded back through hxc_tune_load, and runs under the tuned knobs
bit-identical to runs under the previous ones (knobs change speed only)."""
import json

import numpy as np
import pytest

from paper_1810_11482_b300 import autotune, hxc, synth

pytestmark = pytest.mark.gpu

KNOBS = ["heat2d.emul", "heat2d.rows", "heat2d.occupancy", "heat3d.zchunks", "heat3d.variant",
         "heat3d.variant1", "heat3d.steps_per_launch", "heat1d.tb_ctas",
         "heat1d.steps_per_launch", "mandel.pair", "batch.ctas_per_sm", "batch.block",
         "batch.smem_side"]


@pytest.fixture(scope="module")
def dev():
    devs = hxc.get_all_devices(2, 0)
    assert devs
    return devs[0]


def runs(dev):
    """A small run of every tuned workload, with the caller's steps per
    launch left to the knobs (0)."""
    out = {}
    n1 = 1 << 16
    v0 = synth.heat1d_input(n1, seed=1)
    p, q = dev.buffer(n1 * 8), dev.buffer(n1 * 8)
    p.write(v0).get()
    hxc.heat1d_run(dev, p, q, n1, 8, 0.25, 61, "fused", 0)[0].get()
    out["heat1d"] = np.empty(n1)
    p.read_sync(out["heat1d"])
    u3 = synth.heat3d_input(48, seed=3, nz=40, ny=36)
    a, b = dev.buffer(u3.nbytes), dev.buffer(u3.nbytes)
    a.write(u3).get()
    hxc.heat3d_run(dev, a, b, u3.shape, 0.15, 11, "fused", 0)[0].get()
    out["heat3d"] = np.empty(u3.shape, np.float32)
    a.read_sync(out["heat3d"])
    sides, offs, kap, ub, cs = synth.batch_input(nprob=40, seed=412, smin=8, smax=90)
    bu, bk = dev.buffer(ub.nbytes), dev.buffer(kap.nbytes)
    bu.write(ub).get()
    bk.write(kap).get()
    hxc.varcoef_batch_run(dev, bu, bk, sides, cs, 7, "fused")[0].get()
    out["batch"] = np.empty(ub.size)
    bu.read_sync(out["batch"])
    u0 = synth.bumps2d(300, 260, seed=2, nbumps=5, sigma=0.05)
    u, t = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)
    u.write(u0).get()
    cfg = hxc.heat2d_cfg(300, 260, 3, 2, 0.2, 13, 0, "fused", None, None)
    hxc.heat2d_run(dev, u, t, cfg)[0].get()
    out["heat2d"] = np.empty(u0.shape)
    u.read_sync(out["heat2d"])
    return out


def test_quick_search_cache_round_trip(dev, tmp_path):
    saved = {k: hxc.tune_get(k) for k in KNOBS}
    try:
        before = runs(dev)
        _, result = autotune.tune(quick=True, log=lambda *a: None)
        for k in ("heat3d.steps_per_launch", "heat1d.steps_per_launch", "batch.smem_side"):
            assert k in result
        path = tmp_path / "tune_cache.json"
        arch = "sm_%d%d" % (dev.major, dev.minor)
        path.write_text(json.dumps({arch: {k: int(v) for k, v in result.items()}}))
        for k, v in saved.items():
            hxc.tune_set(k, v)
        hxc.tune_load(str(path), dev.major, dev.minor)
        for k, v in result.items():
            assert hxc.tune_get(k) == v, k
        after = runs(dev)
        for name in before:
            assert np.array_equal(before[name], after[name]), name
    finally:
        for k, v in saved.items():
            hxc.tune_set(k, v)


def test_steps_per_launch_knobs_keep_bits(dev):
    """Every steps-per-launch value of the 1D and 3D fused runs, set through
    the knobs (caller passes 0), gives the bits of the default."""
    saved = {k: hxc.tune_get(k) for k in KNOBS}
    try:
        ref = runs(dev)
        for t3, t1 in ((1, 1), (2, 7), (3, 60), (4, 0)):
            hxc.tune_set("heat3d.steps_per_launch", t3)
            hxc.tune_set("heat1d.steps_per_launch", t1)
            got = runs(dev)
            for name in ref:
                assert np.array_equal(ref[name], got[name]), (name, t3, t1)
    finally:
        for k, v in saved.items():
            hxc.tune_set(k, v)
