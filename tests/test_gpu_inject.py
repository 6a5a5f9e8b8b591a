"""Failure handling of the future layer with host-side fault injection
(hxc_debug_inject): one device operation is made to fail at issue, as if its
CUDA call had returned an error, without any fault on the device.  The
failure must reach the run's future, operations and continuations that
depend on it must not run, no wait may hang (every wait here is bounded),
and the device must stay usable: the same run afterwards matches the oracle."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1810_11482_b300 import hxc, synth

pytestmark = pytest.mark.gpu
WAIT_NS = 60 * 10**9  # bounded waits: a hang fails the test instead of stalling it


@pytest.fixture(scope="module")
def dev():
    devs = hxc.get_all_devices(2, 0)
    assert devs
    yield devs[0]
    hxc.debug_inject(-1)


def run2d(dev, u0, mode, tiles=(2, 3), steps=12, every=4, inject=None):
    """A 2D run with snapshots and host norms; `inject` arms the injection
    (counted from the run's first device operation) after the upload."""
    ny, nx = u0.shape
    u, t = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)
    u.write(u0).get()
    if inject is not None:
        hxc.debug_inject(inject)
    T = tiles[0] * tiles[1]
    hn = np.zeros(steps // every * T)
    cfg = hxc.heat2d_cfg(ny, nx, tiles[0], tiles[1], 0.2, steps, every, mode, hn, None)
    f, _ = hxc.heat2d_run(dev, u, t, cfg)
    return f, u


def test_injected_failure_reaches_the_run_and_spares_the_device(dev):
    u0 = synth.bumps2d(96, 130, seed=260, nbumps=4, sigma=0.1)
    want = oracle.heat2d(u0, 0.2, 12)
    for after in (0, 5, 37):
        f, _ = run2d(dev, u0, "plain", inject=after)
        st = f.wait(WAIT_NS)
        assert st in (hxc.HXC_E_CUDA, hxc.HXC_E_DEP_FAILED), (after, st)
        hxc.debug_inject(-1)
        dev.synchronize()
        f, u = run2d(dev, u0, "plain")
        assert f.wait(WAIT_NS) == hxc.HXC_OK
        got = np.empty_like(u0)
        u.read_sync(got)
        assert np.max(np.abs(got - want)) / np.max(np.abs(want)) <= 1e-12


def test_dependants_and_continuations_of_a_failed_copy_do_not_run(dev):
    n = 4096
    x = np.arange(n, dtype=np.float64)
    a = dev.buffer(n * 8)
    a.write(np.zeros(n)).get()
    ran = []
    hxc.debug_inject(0, hxc.HXC_E_NOMEM)
    w = a.write(x)  # the next device operation: fails with the injected status
    assert w.wait(WAIT_NS) == hxc.HXC_E_NOMEM
    args = hxc.hxc_partition_args(a.h, n, 0)
    k = dev.launch(hxc.HXC_K_PARTITION, args, deps=[w])
    assert k.wait(WAIT_NS) == hxc.HXC_E_DEP_FAILED
    c = k.then(lambda: ran.append(1))
    assert c.wait(WAIT_NS) == hxc.HXC_E_DEP_FAILED
    j = hxc.when_all([k, dev.buffer(8).write(np.zeros(1))])
    assert j.wait(WAIT_NS) == hxc.HXC_E_DEP_FAILED
    assert ran == []
    # the buffer still holds what was there before the failed write
    out = np.empty(n)
    a.read_sync(out)
    assert np.array_equal(out, np.zeros(n))


def test_injected_failure_inside_a_graph_capture(dev):
    """A failure while a run captures its graph fails the run synchronously or
    through its future; no broken graph is cached: the next run in graph mode
    replays a fresh capture and matches the plain run bit for bit."""
    u0 = synth.bumps2d(80, 64, seed=261, nbumps=3, sigma=0.1)
    try:
        f, _ = run2d(dev, u0, "graph", tiles=(2, 2), steps=10, every=5, inject=3)
        assert f.wait(WAIT_NS) != hxc.HXC_OK
    except hxc.HxcError:
        pass
    hxc.debug_inject(-1)
    dev.synchronize()
    f, u = run2d(dev, u0, "graph", tiles=(2, 2), steps=10, every=5)
    assert f.wait(WAIT_NS) == hxc.HXC_OK
    g = np.empty_like(u0)
    u.read_sync(g)
    f, u = run2d(dev, u0, "plain", tiles=(2, 2), steps=10, every=5)
    assert f.wait(WAIT_NS) == hxc.HXC_OK
    p = np.empty_like(u0)
    u.read_sync(p)
    assert np.array_equal(g, p)


def test_injection_argument_checks(dev):
    L = hxc.lib()
    assert L.hxc_debug_inject(ctypes.c_int64(0), hxc.HXC_OK) == hxc.HXC_E_INVALID
    assert L.hxc_debug_inject(ctypes.c_int64(-1), hxc.HXC_OK) == hxc.HXC_OK
    # disarmed: the next operations run normally
    b = dev.buffer(64)
    b.write(np.ones(8)).get()


# ------------------------------------------- every run entry point

def _case_heat1d(dev, mode):
    n = 5003
    u0 = synth.heat1d_input(n, seed=270)
    u, t = dev.buffer(n * 8), dev.buffer(n * 8)

    def prepare():
        u.write(u0).get()

    def issue():
        return hxc.heat1d_run(dev, u, t, n, 4, 0.25, 20, mode)[0]

    def result():
        out = np.empty(n)
        u.read_sync(out)
        return out
    return prepare, issue, result


def _case_heat3d(dev, mode):
    shape = (24, 40, 56)
    u0 = np.ascontiguousarray(synth.heat3d_input(56, seed=271, nz=24, ny=40), dtype=np.float32)
    u, t = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)

    def prepare():
        u.write(u0).get()

    def issue():
        return hxc.heat3d_run(dev, u, t, shape, 0.15, 8, mode, 4)[0]

    def result():
        out = np.empty_like(u0)
        u.read_sync(out)
        return out
    return prepare, issue, result


def _case_batch(dev, mode):
    sides, offs, kap, ub, cs = synth.batch_input(nprob=20, seed=272)
    bu, bk = dev.buffer(ub.nbytes), dev.buffer(kap.nbytes)
    bk.write(kap).get()

    def prepare():
        bu.write(ub).get()

    def issue():
        return hxc.varcoef_batch_run(dev, bu, bk, sides, cs, 6, mode)[0]

    def result():
        out = np.empty_like(ub)
        bu.read_sync(out)
        return out
    return prepare, issue, result


def _case_adjoint(dev, mode):
    n = 64
    kref, kap, u0, c = synth.adjoint_input(n)
    b0, bk, bl = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)
    gk, gu, ut = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)
    b0.write(u0).get()
    bk.write(kap).get()
    bl.write(u0).get()

    def prepare():
        pass

    def issue():
        return hxc.varcoef_adjoint_run(dev, b0, bk, bl, n, n, c, 30, gk, gu, ut, 0, mode)[0]

    def result():
        a, b = np.empty_like(u0), np.empty_like(u0)
        gk.read_sync(a)
        gu.read_sync(b)
        return np.concatenate([a.ravel(), b.ravel()])
    return prepare, issue, result


def _case_forward(dev, mode):
    n = 72
    kref, kap, u0, c = synth.adjoint_input(n)
    b0, bk, ut = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)
    b0.write(u0).get()
    bk.write(kap).get()

    def prepare():
        pass

    def issue():
        return hxc.varcoef_forward_run(dev, b0, bk, n, n, c, 25, ut)[0]

    def result():
        out = np.empty_like(u0)
        ut.read_sync(out)
        return out
    return prepare, issue, result


def _case_forward_tape(dev, mode):
    """The forward that keeps its checkpoints (tape) for a later gradient."""
    n, steps, every = 66, 27, 5
    kref, kap, u0, c = synth.adjoint_input(n)
    ns = hxc.varcoef_tape_states(steps, every)
    b0, bk, ut = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)
    tape = dev.buffer(ns * u0.nbytes)
    b0.write(u0).get()
    bk.write(kap).get()

    def prepare():
        pass

    def issue():
        return hxc.varcoef_forward_tape(dev, b0, bk, n, n, c, steps, ut, tape, every)[0]

    def result():
        out, tp = np.empty_like(u0), np.empty(ns * n * n)
        ut.read_sync(out)
        tape.read_sync(tp)
        return np.concatenate([out.ravel(), tp])
    return prepare, issue, result


def _case_adjoint_tape(dev, mode):
    """The gradient that starts from a forward's checkpoints; the tape is
    written once, before the runs under test, and is only read by them."""
    n, steps, every = 60, 23, 6
    kref, kap, u0, c = synth.adjoint_input(n)
    ns = hxc.varcoef_tape_states(steps, every)
    b0, bk, bl = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)
    ut, gk, gu = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)
    tape = dev.buffer(ns * u0.nbytes)
    b0.write(u0).get()
    bk.write(kap).get()
    bl.write(u0).get()
    f, _ = hxc.varcoef_forward_tape(dev, b0, bk, n, n, c, steps, ut, tape, every)
    assert f.wait(WAIT_NS) == hxc.HXC_OK

    def prepare():
        pass

    def issue():
        return hxc.varcoef_adjoint_tape(dev, tape, bk, bl, n, n, c, steps, gk, gu, every, mode)[0]

    def result():
        a, b = np.empty_like(u0), np.empty_like(u0)
        gk.read_sync(a)
        gu.read_sync(b)
        return np.concatenate([a.ravel(), b.ravel()])
    return prepare, issue, result


def _case_stream2d(dev, mode):
    u0 = synth.bumps2d(70, 90, seed=273, nbumps=3, sigma=0.1)
    ha, hb = hxc.host_empty(u0.shape), hxc.host_empty(u0.shape)
    res = {}

    def prepare():
        ha[:] = u0
        hb[:] = 0.0

    def issue():
        f, _, out = hxc.heat2d_stream_run(dev, ha, hb, (2, 2), 0.2, 3, sequential=(mode == "plain"))
        res["out"] = out
        return f

    def result():
        return np.array(res["out"])
    return prepare, issue, result


def _case_partition(dev, mode):
    n = 1 << 16
    hx, hr = hxc.host_empty(n), hxc.host_empty(n)
    work = dev.buffer(n * 8)

    def prepare():
        hx[:] = np.arange(n, dtype=np.float64)
        hr[:] = 0.0

    def issue():
        return hxc.partition_run(dev, hx, hr, 4, work)

    def result():
        return np.array(hr)
    return prepare, issue, result


def _case_heat2d(dev, mode):
    """The resident 2D run with host and device norms."""
    u0 = synth.bumps2d(72, 100, seed=275, nbumps=3, sigma=0.1)
    u, t = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)
    hn, gn = np.zeros(3 * 6), np.zeros(3 * 6)

    def prepare():
        u.write(u0).get()
        hn[:] = 0.0
        gn[:] = 0.0

    def issue():
        cfg = hxc.heat2d_cfg(72, 100, 2, 3, 0.2, 12, 4, mode, hn, gn)
        issue.cfg = cfg  # the run writes the norms through it
        return hxc.heat2d_run(dev, u, t, cfg)[0]

    def result():
        out = np.empty_like(u0)
        u.read_sync(out)
        return np.concatenate([out.ravel(), hn, gn])
    return prepare, issue, result


def _case_host2d(dev, mode):
    """The synchronous host entry point: the field in and out of host memory,
    snapshots with host norms."""
    u0 = synth.bumps2d(64, 96, seed=274, nbumps=3, sigma=0.1)
    hu, ho = hxc.host_empty(u0.shape), hxc.host_empty(u0.shape)
    hn = np.zeros(2 * 4)

    def prepare():
        hu[:] = u0
        ho[:] = 0.0

    def issue():
        cfg = hxc.heat2d_cfg(64, 96, 2, 2, 0.2, 10, 5, mode, hn, None)
        hxc.heat2d_run_host(dev, hu.ctypes.data, ho.ctypes.data, cfg)
        f = hxc.promise()
        hxc.promise_set(f, hxc.HXC_OK)
        return f

    def result():
        return np.concatenate([np.array(ho).ravel(), hn])
    return prepare, issue, result


def _case_mandelbrot(dev, mode):
    """An image computed, copied back and written as a PNG file, the write
    synchronous ("plain") or a continuation ("fused"); the result is the
    file's bytes."""
    import tempfile
    w, h = 257, 123
    path = tempfile.mkdtemp(prefix="hxc_inject_") + "/m.png"
    rgb = dev.buffer(w * h * 3)
    host = np.zeros(w * h * 3, dtype=np.uint8)
    args = hxc.mandelbrot_args(rgb, w, h, -2.0, -1.2, 3.0 / w, 2.4 / h, 200)

    def prepare():
        host[:] = 0

    def issue():
        issue.rgb = rgb  # the argument block holds its handle only
        return hxc.mandelbrot_png(dev, args, host, path, level=1, async_write=(mode == "fused"))

    def result():
        with open(path, "rb") as fh:
            return np.frombuffer(fh.read(), dtype=np.uint8).copy()
    return prepare, issue, result


PROG_SRC = r"""
extern "C" __global__ void axpb(double *x, double a, double b, long long n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) x[i] = a * x[i] + b;
}
"""


def _case_program(dev, mode):
    """A run-time compiled kernel (the paper's program.run) on a buffer."""
    import ctypes
    n = 10007
    x0 = np.linspace(-1.0, 1.0, n)
    buf = dev.buffer(n * 8)
    prog = hxc.Program.from_source(dev, PROG_SRC, "axpb.cu")
    assert prog.build("axpb").wait(WAIT_NS) == hxc.HXC_OK, prog.log()

    def prepare():
        buf.write(x0).get()

    def issue():
        issue.prog = prog  # kept alive with the case
        return prog.run("axpb", [buf, ctypes.c_double(0.5), ctypes.c_double(0.25),
                                 ctypes.c_longlong(n)], ((n + 255) // 256, 1, 1), (256, 1, 1))

    def result():
        out = np.empty(n)
        buf.read_sync(out)
        return out
    return prepare, issue, result


CASES = [("heat1d", _case_heat1d, m) for m in ("plain", "graph", "fused")] + \
        [("heat2d", _case_heat2d, m) for m in ("plain", "graph", "fused")] + \
        [("host2d", _case_host2d, m) for m in ("plain", "graph", "fused")] + \
        [("heat3d", _case_heat3d, m) for m in ("plain", "graph", "fused")] + \
        [("batch", _case_batch, m) for m in ("plain", "graph", "fused")] + \
        [("adjoint", _case_adjoint, m) for m in ("plain", "graph", "fused")] + \
        [("adjoint_tape", _case_adjoint_tape, m) for m in ("plain", "graph", "fused")] + \
        [("forward", _case_forward, "fused"), ("forward_tape", _case_forward_tape, "fused"),
         ("stream2d", _case_stream2d, "plain"),
         ("stream2d", _case_stream2d, "fused"), ("partition", _case_partition, "fused"),
         ("mandelbrot", _case_mandelbrot, "plain"), ("mandelbrot", _case_mandelbrot, "fused"),
         ("program", _case_program, "plain")]


@pytest.mark.parametrize("name,case,mode", CASES, ids=["%s-%s" % (c[0], c[2]) for c in CASES])
def test_every_run_survives_an_injected_failure(dev, name, case, mode):
    """For every run entry point and mode: a run with one device operation
    failing at issue reports the failure (synchronously or in its future,
    within a bounded wait), and the same run afterwards gives the bits of a
    run that never saw a failure."""
    prepare, issue, result = case(dev, mode)
    prepare()
    f = issue()
    assert f.wait(WAIT_NS) == hxc.HXC_OK
    want = result()
    for after in (0, 3, 11):
        prepare()
        hxc.debug_inject(after)
        try:
            f = issue()
            st = f.wait(WAIT_NS)
            assert st != hxc.HXC_E_TIMEOUT, (after, st)
        except hxc.HxcError:
            pass
        hxc.debug_inject(-1)
        dev.synchronize()
        prepare()
        f = issue()
        assert f.wait(WAIT_NS) == hxc.HXC_OK, after
        got = result()
        assert np.array_equal(got, want), after


def test_runs_of_every_kind_issued_together(dev):
    """Every run entry point and mode issued back to back without waiting
    (they share the device's streams, scratch and staging buffers), twice:
    each result has the bits of the same run issued alone."""
    cases = [case(dev, mode) for _, case, mode in CASES]
    wants = []
    for prepare, issue, result in cases:
        prepare()
        assert issue().wait(WAIT_NS) == hxc.HXC_OK
        wants.append(result())
    for rep in range(2):
        for prepare, _, _ in cases:
            prepare()
        futs = [issue() for _, issue, _ in cases]
        for f in futs:
            assert f.wait(WAIT_NS) == hxc.HXC_OK
        for i, ((_, _, result), want) in enumerate(zip(cases, wants)):
            assert np.array_equal(result(), want), (rep, CASES[i][0], CASES[i][2])


def test_runs_issued_from_several_threads(dev):
    """Host threads issue resident and host-memory 2D runs (with host and
    device norms, every mode) and 3D runs at the same time, each on its own
    buffers; every result has the bits of the same run issued alone."""
    import threading
    kinds = [(_case_heat2d, m) for m in ("plain", "graph", "fused")] + \
            [(_case_host2d, "fused"), (_case_heat3d, "fused"), (_case_heat2d, "fused")]
    cases = [case(dev, mode) for case, mode in kinds]
    wants = []
    for prepare, issue, result in cases:
        prepare()
        assert issue().wait(WAIT_NS) == hxc.HXC_OK
        wants.append(result())
    errors = []
    start = threading.Barrier(len(cases))

    def worker(i):
        prepare, issue, result = cases[i]
        try:
            start.wait()
            for rep in range(6):
                prepare()
                st = issue().wait(WAIT_NS)
                if st != hxc.HXC_OK:
                    errors.append((i, rep, "status %d" % st))
                elif not np.array_equal(result(), wants[i]):
                    errors.append((i, rep, "bits differ"))
        except Exception as e:  # reported below, not lost in the thread
            errors.append((i, -1, repr(e)))

    threads = [threading.Thread(target=worker, args=(i,)) for i in range(len(cases))]
    for t in threads:
        t.start()
    for t in threads:
        t.join(300)
    assert not any(t.is_alive() for t in threads)
    assert errors == []


# ------------------------------------------------- graph capture and threads

def _heat1d_chain(dev, a, b, n, steps, r=0.25, slot=0):
    """`steps` one-step 1D launches ping-ponging between a and b (the result
    is in a for even steps); the future of the last."""
    f = None
    src, dst = a, b
    for _ in range(steps):
        args = hxc.hxc_heat1d_args(src.h, dst.h, n, 0, n, r, 1)
        f = dev.launch(hxc.HXC_K_HEAT1D, args, slot, deps=[f] if f is not None else ())
        src, dst = dst, src
    return f


def test_graph_api_capture_and_replay(dev):
    """hxc_graph_begin/end/launch: 20 captured 1D launches replayed three
    times give the bits of 60 launches issued directly."""
    n = 4099
    u0 = synth.heat1d_input(n, seed=280)
    a, b = dev.buffer(n * 8), dev.buffer(n * 8)
    a.write(u0).get()
    hxc.graph_begin(dev)
    try:
        _heat1d_chain(dev, a, b, n, 20)
    finally:
        g = hxc.graph_end(dev)
    assert g.node_count() >= 20
    f = None
    for _ in range(3):
        f = g.launch(0, deps=[f] if f is not None else ())
    assert f.wait(WAIT_NS) == hxc.HXC_OK
    got = np.empty(n)
    a.read_sync(got)
    c, d = dev.buffer(n * 8), dev.buffer(n * 8)
    c.write(u0).get()
    assert _heat1d_chain(dev, c, d, n, 60).wait(WAIT_NS) == hxc.HXC_OK
    want = np.empty(n)
    c.read_sync(want)
    assert np.array_equal(got, want)
    assert np.max(np.abs(got - oracle.heat1d(u0, 0.25, 60))) <= 1e-12 * np.max(np.abs(u0))
    g.close()


def test_user_graph_of_fused_2d_runs(dev):
    """A user capture (hxc_graph_begin/end) of a fused 2D run, whose step
    launches follow each other by programmatic dependent launch, replayed
    twice gives the bits of two fused runs of the same length issued
    directly."""
    u0 = synth.bumps2d(96, 130, seed=282, nbumps=4, sigma=0.1)
    ny, nx = u0.shape
    cfg = hxc.heat2d_cfg(ny, nx, 1, 1, 0.2, 30, 0, "fused", None, None)
    a, b = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)
    a.write(u0).get()
    assert hxc.heat2d_run(dev, a, b, cfg)[0].wait(WAIT_NS) == hxc.HXC_OK  # no allocation later
    a.write(u0).get()
    hxc.graph_begin(dev)
    try:
        hxc.heat2d_run(dev, a, b, cfg)
    finally:
        g = hxc.graph_end(dev)
    assert g.node_count() >= 30
    f = None
    for _ in range(2):
        f = g.launch(0, deps=[f] if f is not None else ())
    assert f.wait(WAIT_NS) == hxc.HXC_OK
    got = np.empty_like(u0)
    a.read_sync(got)
    c, d = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)
    c.write(u0).get()
    for _ in range(2):
        assert hxc.heat2d_run(dev, c, d, cfg)[0].wait(WAIT_NS) == hxc.HXC_OK
    want = np.empty_like(u0)
    c.read_sync(want)
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))
    assert np.max(np.abs(got - oracle.heat2d(u0, 0.2, 60))) <= 1e-12 * np.max(np.abs(u0))
    g.close()


def test_capture_holds_other_threads_operations(dev):
    """While one thread captures a graph, operations that another thread and
    the worker pool issue to the device wait for the capture to end instead
    of landing in the graph (or failing): they run afterwards with the right
    results, and the graph holds only the capturing thread's launches."""
    import threading
    import time
    n = 2048
    u0 = synth.heat1d_input(n, seed=281)
    a, b = dev.buffer(n * 8), dev.buffer(n * 8)
    c, d = dev.buffer(n * 8), dev.buffer(n * 8)
    e, f_ = dev.buffer(n * 8), dev.buffer(n * 8)
    a.write(u0).get()
    e.write(u0).get()
    hxc.graph_begin(dev)  # the same capture alone, for its node count
    try:
        _heat1d_chain(dev, a, b, n, 10)
    finally:
        solo = hxc.graph_end(dev)
    gate = hxc.promise()
    # a launch deferred on a host promise, set while the capture runs
    deferred = dev.launch(hxc.HXC_K_HEAT1D, hxc.hxc_heat1d_args(e.h, f_.h, n, 0, n, 0.25, 1), 3,
                          deps=[gate])
    capturing, res = threading.Event(), {}

    def capturer():
        hxc.graph_begin(dev)
        try:
            capturing.set()
            _heat1d_chain(dev, a, b, n, 10)
            hxc.promise_set(gate, hxc.HXC_OK)
            time.sleep(0.3)
            res["t_end"] = time.perf_counter()
        finally:
            res["graph"] = hxc.graph_end(dev)

    def other():
        capturing.wait(30)
        c.write(u0).get()
        res["t_other"] = time.perf_counter()
        res["other"] = _heat1d_chain(dev, c, d, n, 10, slot=5).wait(WAIT_NS)

    ts = [threading.Thread(target=capturer), threading.Thread(target=other)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(120)
    assert not any(t.is_alive() for t in ts)
    assert res["t_other"] >= res["t_end"]
    assert res["other"] == hxc.HXC_OK
    assert deferred.wait(WAIT_NS) == hxc.HXC_OK
    g = res["graph"]
    assert g.node_count() == solo.node_count() >= 10
    solo.close()
    assert g.launch(0).wait(WAIT_NS) == hxc.HXC_OK
    want = oracle.heat1d(u0, 0.25, 10)
    for buf in (a, c):
        got = np.empty(n)
        buf.read_sync(got)
        assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(u0))
    got = np.empty(n)
    f_.read_sync(got)
    assert np.max(np.abs(got - oracle.heat1d(u0, 0.25, 1))) <= 1e-12 * np.max(np.abs(u0))
    g.close()
