"""Run-time compiled programs (the paper's `program`, Sec. 4, Listing 2).

A program is created from a file or a string, built into a future, and run
with buffers and values as arguments on a user grid; runs follow the build.
"""
import ctypes

import numpy as np
import pytest

from paper_1810_11482_b300 import hxc

pytestmark = pytest.mark.gpu

# One block of threads sums an array of unsigned ints into *result (the
# worked example of Listing 2: 1000 ones on a 1x1x1 grid of 32 threads).
SUM_SRC = r'''
extern "C" __global__ void sum(const unsigned int *a, unsigned int *result, unsigned int n) {
    unsigned int s = 0;
    for (unsigned int i = threadIdx.x; i < n; i += blockDim.x) s += a[i];
    atomicAdd(result, s);
}
'''

# A templated kernel (C++ name expression) with value arguments and a 2D grid.
AXPY_SRC = r'''
template <class T>
__global__ void axpy2d(T *y, const T *x, T alpha, int ny, int nx) {
    int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i < ny && j < nx) y[(long long)i * nx + j] = alpha * x[(long long)i * nx + j] + y[(long long)i * nx + j];
}
'''


@pytest.fixture(scope="module")
def dev():
    devs = hxc.get_all_devices(2, 0)
    assert devs
    return devs[0]


def test_listing2_sum_from_file(dev, tmp_path):
    path = tmp_path / "example_kernel.cu"
    path.write_text(SUM_SRC)
    n = 1000
    a = np.ones(n, dtype=np.uint32)
    zero = np.zeros(1, dtype=np.uint32)
    buf_a, buf_r = dev.buffer(a.nbytes), dev.buffer(4)
    prog = hxc.Program.from_file(dev, path)
    futs = [prog.build("sum"), buf_a.write(a), buf_r.write(zero)]
    assert hxc.wait_all(futs) == hxc.HXC_OK, prog.log()
    run = prog.run("sum", [buf_a, buf_r, ctypes.c_uint32(n)], (1, 1, 1), (32, 1, 1))
    out = np.zeros(1, dtype=np.uint32)
    buf_r.read(out, deps=[run]).get()
    assert int(out[0]) == n
    prog.close()


def test_templated_kernel_values_and_2d_grid(dev):
    ny, nx = 300, 517  # ragged against the 32x8 block
    rng = np.random.default_rng(7)
    x = rng.standard_normal((ny, nx))
    y = rng.standard_normal((ny, nx))
    bx, by = dev.buffer(x.nbytes), dev.buffer(y.nbytes)
    prog = hxc.Program.from_source(dev, AXPY_SRC, "axpy.cu")
    b = prog.build("axpy2d<double>")
    w = [bx.write(x), by.write(y)]
    # the run depends on the writes explicitly and on the build implicitly
    run = prog.run("axpy2d<double>", [by, bx, ctypes.c_double(-0.75), ctypes.c_int(ny), ctypes.c_int(nx)],
                   ((nx + 31) // 32, (ny + 7) // 8, 1), (32, 8, 1), slot=1, deps=w)
    out = np.empty_like(y)
    by.read(out, deps=[run]).get()
    b.get()
    want = -0.75 * x + y  # one rounding each way: multiply then add, or a fused multiply-add
    assert np.max(np.abs(out - want)) <= 2 * np.finfo(float).eps * np.max(np.abs(want))
    prog.close()


def test_compile_error_fails_the_build_future_and_its_runs(dev):
    prog = hxc.Program.from_source(dev, "extern \"C\" __global__ void k(int *p) { p[0] = undefined_name; }")
    f = prog.build("k")
    assert f.wait() == hxc.HXC_E_INVALID
    assert "undefined_name" in prog.log()
    buf = dev.buffer(4)
    r = prog.run("k", [buf], (1, 1, 1), (32, 1, 1))
    assert r.wait() != hxc.HXC_OK  # a run after a failed build does not launch
    prog.close()


def test_unknown_kernel_name(dev):
    prog = hxc.Program.from_source(dev, SUM_SRC)
    assert prog.build("nope").wait() == hxc.HXC_E_INVALID
    assert "nope" in prog.log()
    prog.close()


def test_build_options_and_chained_builds(dev):
    src = r'''
extern "C" __global__ void fill(int *p) { p[threadIdx.x] = VALUE; }
'''
    prog = hxc.Program.from_source(dev, src)
    buf = dev.buffer(32 * 4)
    prog.build("fill", "-DVALUE=41").get()
    r1 = prog.run("fill", [buf], (1, 1, 1), (32, 1, 1))
    out = np.zeros(32, dtype=np.int32)
    buf.read(out, deps=[r1]).get()
    assert (out == 41).all()
    # a rebuild with other options replaces the kernel for later runs only
    b2 = prog.build("fill", "-DVALUE=42", deps=[r1])
    r2 = prog.run("fill", [buf], (1, 1, 1), (32, 1, 1))
    buf.read(out, deps=[r2]).get()
    b2.get()
    assert (out == 42).all()
    prog.close()


def test_run_argument_checks(dev):
    prog = hxc.Program.from_source(dev, SUM_SRC)
    prog.build("sum").get()
    buf = dev.buffer(4)
    with pytest.raises(hxc.HxcError):
        prog.run("sum", [buf], (1, 1, 1), (2048, 1, 1))  # more than 1024 threads
    with pytest.raises(hxc.HxcError):
        prog.run("sum", [buf], (0, 1, 1), (32, 1, 1))  # empty grid
    prog.close()
