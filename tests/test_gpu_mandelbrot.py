"""Sec. 5.1.3 Mandelbrot: the device kernel against the binary32 oracle
(escape counts and colours bit for bit), and PNG files written
synchronously and as continuations, decoded back here."""
import os

import numpy as np
import pytest

import oracle
from paper_1810_11482_b300 import hxc

from test_png_cpu import decode_png

pytestmark = pytest.mark.gpu
F = np.float32


@pytest.fixture(scope="module")
def dev():
    devs = hxc.get_all_devices(2, 0)
    assert devs
    return devs[0]


def device_image(dev, w, h, x0, y0, dx, dy, it, cfg=None):
    rgb, cnt = dev.buffer(max(1, w * h * 3)), dev.buffer(max(1, w * h * 4))
    dev.launch(hxc.HXC_K_MANDELBROT, hxc.mandelbrot_args(rgb, w, h, x0, y0, dx, dy, it, cnt),
               cfg=cfg).get()
    out_rgb = np.empty((h, w, 3), dtype=np.uint8)
    out_cnt = np.empty((h, w), dtype=np.int32)
    if w * h:
        rgb.read_sync(out_rgb)
        cnt.read_sync(out_cnt)
    return out_rgb, out_cnt


CASES = [
    (333, 251, F(-2.0), F(-1.5), F(3.0 / 333), F(3.0 / 251), 300),   # whole set, ragged tiles
    (257, 129, F(-0.7485), F(0.0999), F(2e-5), F(2e-5), 1001),       # near the boundary
    (8, 4, F(-2.0), F(-1.0), F(0.4), F(0.5), 1),                     # one tile, max_iter 1
    (1, 1, F(0.0), F(0.0), F(1.0), F(1.0), 7),
    (64, 48, F(-1.9), F(-1.2), F(0.05), F(0.05), 6),                  # groups of 4 + a tail of 2
    # across |c|^2 = 3.99, where the kernel switches between testing every
    # fourth iterate and testing every iterate: on the circle near c = -2
    # (slow escapes along the real axis), near 1.41 + 1.41i and near 2i
    (200, 120, F(-2.02), F(-0.03), F(2.5e-4), F(5e-4), 700),
    (150, 150, F(1.395), F(1.395), F(1e-4), F(1e-4), 300),
    (160, 100, F(-0.04), F(1.985), F(5e-4), F(2e-4), 300),
]


@pytest.mark.parametrize("case", CASES)
def test_kernel_matches_oracle(dev, case):
    w, h, x0, y0, dx, dy, it = case
    rgb, cnt = device_image(dev, w, h, x0, y0, dx, dy, it)
    want_rgb, want_cnt = oracle.mandelbrot_image(w, h, x0, y0, dx, dy, it)
    assert np.array_equal(cnt, want_cnt)
    assert np.array_equal(rgb, want_rgb)


@pytest.mark.parametrize("case", CASES)
def test_one_and_two_pixel_forms_agree(dev, case):
    """The kernel's two forms (one pixel per thread; two adjacent pixels per
    thread on paired FP32 instructions) give the same counts and colours."""
    w, h, x0, y0, dx, dy, it = case
    old = hxc.tune_get("mandel.pair")
    try:
        outs = []
        for pair in (0, 1):
            hxc.tune_set("mandel.pair", pair)
            outs.append(device_image(dev, w, h, x0, y0, dx, dy, it))
        assert np.array_equal(outs[0][1], outs[1][1]) and np.array_equal(outs[0][0], outs[1][0])
    finally:
        hxc.tune_set("mandel.pair", old)


def test_launch_shapes_do_not_change_bits(dev):
    w, h, x0, y0, dx, dy, it = CASES[0]
    a = device_image(dev, w, h, x0, y0, dx, dy, it)
    for grid, block in (((1, 1, 1), (32, 1, 1)), ((7, 1, 1), (64, 1, 1)), ((300, 1, 1), (256, 1, 1))):
        b = device_image(dev, w, h, x0, y0, dx, dy, it, cfg=hxc.hxc_launch_cfg(grid, block))
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_empty_image_and_argument_checks(dev):
    rgb = dev.buffer(64)
    dev.launch(hxc.HXC_K_MANDELBROT, hxc.mandelbrot_args(rgb, 0, 5, F(0), F(0), F(1), F(1), 10)).get()
    with pytest.raises(hxc.HxcError):  # buffer too small
        dev.launch(hxc.HXC_K_MANDELBROT, hxc.mandelbrot_args(rgb, 10, 10, F(0), F(0), F(1), F(1), 10))
    with pytest.raises(hxc.HxcError):  # more than 256 threads per block
        dev.launch(hxc.HXC_K_MANDELBROT, hxc.mandelbrot_args(rgb, 4, 4, F(0), F(0), F(1), F(1), 10),
                   cfg=hxc.hxc_launch_cfg((1, 1, 1), (512, 1, 1)))


@pytest.mark.parametrize("async_write", [False, True])
def test_png_pipeline(dev, tmp_path, async_write):
    """Three images of different sizes in flight at once (async) or one after
    another (sync); every file decodes to the oracle's image."""
    sizes = [(640, 480), (1000, 1000), (123, 77)]
    futs, want = [], []
    keep = []
    for q, (w, h) in enumerate(sizes):
        buf, host = dev.buffer(w * h * 3), hxc.host_empty(w * h * 3, np.uint8)
        args = hxc.mandelbrot_args(buf, w, h, F(-2.0), F(-1.25), F(3.0 / w), F(2.5 / h), 256)
        path = tmp_path / f"m{q}.png"
        futs.append(hxc.mandelbrot_png(dev, args, host, path, level=1, async_write=async_write,
                                       slot=q))
        keep.append((buf, host))
        want.append((path, oracle.mandelbrot_image(w, h, F(-2.0), F(-1.25), F(3.0 / w),
                                                   F(2.5 / h), 256)[0]))
    if not async_write:
        assert all(f.is_ready() for f in futs)
    assert hxc.wait_all(futs) == hxc.HXC_OK
    for path, img in want:
        got, _ = decode_png(path)
        assert np.array_equal(got, img)


def test_png_pipeline_reports_write_errors(dev, tmp_path):
    w = h = 64
    buf, host = dev.buffer(w * h * 3), hxc.host_empty(w * h * 3, np.uint8)
    args = hxc.mandelbrot_args(buf, w, h, F(-2.0), F(-1.5), F(3.0 / w), F(3.0 / h), 50)
    bad = os.path.join(str(tmp_path), "missing_dir", "m.png")
    f = hxc.mandelbrot_png(dev, args, host, bad, async_write=True)
    assert f.wait() == hxc.HXC_E_INVALID
    with pytest.raises(hxc.HxcError):
        hxc.mandelbrot_png(dev, args, host, bad, async_write=False)


def test_full_size_image_sampled(dev):
    """The largest image of the benchmark (8192 x 8192, 256 iterations):
    sampled rows and columns against the oracle's per-point counts."""
    n, it = 8192, 256
    x0, y0, d = F(-2.0), F(-1.5), F(3.0 / n)
    rgb, cnt = device_image(dev, n, n, x0, y0, d, d, it)
    rows = np.array([0, 1, 2047, 4095, 4096, 6000, n - 1])
    for j in rows:
        i = np.arange(n)
        cr = x0 + i.astype(F) * d
        ci = np.full(n, y0 + F(j) * d, dtype=F)
        assert np.array_equal(cnt[j], oracle.mandelbrot_counts(cr, ci, it))
    i = 3000
    cr = np.full(n, x0 + F(i) * d, dtype=F)
    ci = y0 + np.arange(n).astype(F) * d
    assert np.array_equal(cnt[:, i], oracle.mandelbrot_counts(cr, ci, it))
    assert abs((cnt == it).mean() * 9.0 - 1.5066) < 0.03
