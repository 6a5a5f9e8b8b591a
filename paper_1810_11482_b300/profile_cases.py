"""Small, self-contained cases for profiling one kernel at a time.

    python -m paper_1810_11482_b300.profile_cases heat1d [log2 n] [parts] [steps] [fused 0/1]
    python -m paper_1810_11482_b300.profile_cases heat2d [n] [launches]
    python -m paper_1810_11482_b300.profile_cases heat3d [nz ny nx] [steps]
    python -m paper_1810_11482_b300.profile_cases heat3d_step [nz ny nx] [steps]
    python -m paper_1810_11482_b300.profile_cases batch [nprob] [steps]
    python -m paper_1810_11482_b300.profile_cases adjoint [n] [steps]
    python -m paper_1810_11482_b300.profile_cases partition [n] [parts]
    python -m paper_1810_11482_b300.profile_cases mandelbrot [side] [max_iter]

Each case uploads seeded synthetic inputs, runs the path once through the C
ABI and exits 0; sizes default to fields larger than the 126 MB L2 but small
enough for a profiler capture.
"""
import sys

import numpy as np

from . import hxc, synth


def heat1d(log2n=20, parts=8, steps=100, fused=0):
    dev = hxc.get_all_devices(2, 0)[0]
    n = 1 << log2n
    u0 = synth.heat1d_input(n, seed=1)
    u, t = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)
    u.write(u0).get()
    f, st = hxc.heat1d_run(dev, u, t, n, parts, 0.25, steps, "fused" if fused else "plain", 0)
    f.get()
    return st.kernel_launches


def heat2d(n=4096, launches=3):
    dev = hxc.get_all_devices(2, 0)[0]
    u0 = synth.uniform(5, n * n).reshape(n, n)
    u, t = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)
    u.write(u0).get()
    cfg = hxc.heat2d_cfg(n, n, 1, 1, 0.2, launches, 0, "fused", None, None)
    f, st = hxc.heat2d_run(dev, u, t, cfg)
    f.get()
    return st.kernel_launches


def heat3d(nz=256, ny=512, nx=512, steps=8):
    dev = hxc.get_all_devices(2, 0)[0]
    u0 = synth.uniform(6, nz * ny * nx).astype(np.float32)
    u, t = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)
    u.write(u0).get()
    f, st = hxc.heat3d_run(dev, u, t, (nz, ny, nx), 0.15, steps, "fused", 4)
    f.get()
    return st.kernel_launches


def heat3d_step(nz=512, ny=512, nx=512, steps=4):
    """One step per launch (PLAIN mode): the one-step kernel form."""
    dev = hxc.get_all_devices(2, 0)[0]
    u0 = synth.uniform(6, nz * ny * nx).astype(np.float32)
    u, t = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)
    u.write(u0).get()
    f, st = hxc.heat3d_run(dev, u, t, (nz, ny, nx), 0.15, steps, "plain", 1)
    f.get()
    return st.kernel_launches


def batch(nprob=512, steps=10):
    dev = hxc.get_all_devices(2, 0)[0]
    sides, offs, kap, u0, cs = synth.batch_input(nprob=nprob, seed=4)
    u, k = dev.buffer(u0.nbytes), dev.buffer(kap.nbytes)
    u.write(u0).get()
    k.write(kap).get()
    f, st = hxc.varcoef_batch_run(dev, u, k, sides, cs, steps, "fused")
    f.get()
    return st.kernel_launches


def adjoint(n=2048, steps=20):
    dev = hxc.get_all_devices(2, 0)[0]
    kref, kap, u0, c = synth.adjoint_input(n)
    bu, bk, bl = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)
    bu.write(u0).get()
    bk.write(kap).get()
    bl.write(u0).get()
    gk, gu = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)
    f, st = hxc.varcoef_adjoint_run(dev, bu, bk, bl, n, n, c, steps, gk, gu)
    f.get()
    return st.kernel_launches


def partition(n=1 << 24, parts=4):
    dev = hxc.get_all_devices(2, 0)[0]
    x, r = hxc.host_empty(n), hxc.host_empty(n)
    synth.partition_input(n, out=x)
    hxc.partition_run(dev, x, r, parts, dev.buffer(n * 8)).get()
    return parts


def mandelbrot(side=4096, max_iter=256):
    dev = hxc.get_all_devices(2, 0)[0]
    f32 = np.float32
    rgb = dev.buffer(side * side * 3)
    a = hxc.mandelbrot_args(rgb, side, side, f32(-2.0), f32(-1.5), f32(3.0 / side), f32(3.0 / side),
                            max_iter)
    dev.launch(hxc.HXC_K_MANDELBROT, a).get()
    return 1


CASES = {"heat1d": heat1d, "heat2d": heat2d, "heat3d": heat3d, "heat3d_step": heat3d_step, "batch": batch,
         "adjoint": adjoint,
         "partition": partition, "mandelbrot": mandelbrot}

if __name__ == "__main__":
    name = sys.argv[1]
    args = [int(a) for a in sys.argv[2:]]
    print(name, "launches:", CASES[name](*args))
