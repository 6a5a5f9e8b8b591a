"""CPU checks of the C-ABI library: it loads, exports every function that
include/hxc.h declares, its structs match the binding's layouts, and the
host side of the future layer (promises, then, when_all, wait_all, error
propagation, timeouts) behaves as specified without touching a GPU."""
import ctypes
import os
import re
import subprocess
import tempfile
import threading
import time

import numpy as np
import pytest

from paper_1810_11482_b300 import hxc, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def _declared_functions():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        # declarations: "<return type> hxc_name(" at the start of a line
        for m in re.finditer(r"^\s*(?!typedef)(?:const\s+)?\w+\s*\**\s*(hxc_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def L():
    from paper_1810_11482_b300 import build
    build.build()
    return hxc.lib()


def test_exports_every_declared_function(L):
    names = _declared_functions()
    assert len(names) > 40
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # the binding covers the same set
    unbound = [n for n in names if n not in hxc._SIGS]
    assert not unbound, unbound


def test_struct_layouts_match_header(L):
    structs = ["hxc_launch_cfg", "hxc_sum_args", "hxc_prk_args", "hxc_heat1d_args",
               "hxc_heat2d_args", "hxc_tile_norm2_args", "hxc_partition_args", "hxc_run_stats",
               "hxc_heat2d_cfg"]
    structs += [s for s in getattr(hxc, "EXTRA_STRUCTS", [])]
    prog = "#include <stdio.h>\n#include \"hxc.h\"\nint main(void){\n"
    for s in structs:
        prog += 'printf("%%s %%zu\\n", "%s", sizeof(%s));\n' % (s, s)
    prog += "return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(prog)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = subprocess.check_output([exe], text=True)
    sizes = dict(line.split() for line in out.strip().splitlines())
    for s in structs:
        assert int(sizes[s]) == ctypes.sizeof(getattr(hxc, s)), s


def test_status_strings_and_version(L):
    assert L.hxc_abi_version() == 1
    assert L.hxc_status_string(hxc.HXC_E_TIMEOUT) == b"timeout"
    assert L.hxc_status_string(hxc.HXC_E_DEP_FAILED) == b"dependency failed"


def test_invalid_handles_rejected(L):
    bogus = ctypes.c_void_p(0)
    assert L.hxc_future_wait(bogus, 0) == hxc.HXC_E_INVALID
    assert L.hxc_buffer_release(bogus) == hxc.HXC_E_INVALID
    r = ctypes.c_int()
    assert L.hxc_future_is_ready(bogus, ctypes.byref(r)) == hxc.HXC_E_INVALID
    assert L.hxc_future_then(bogus, hxc.HOST_FN(lambda u: 0), None, None) == hxc.HXC_E_INVALID


def test_promise_then_chain_runs_in_order(L):
    log = []
    p = hxc.promise()
    a = p.then(lambda: log.append("a"))
    b = a.then(lambda: log.append("b"))
    time.sleep(0.05)
    assert log == [] and not b.is_ready()
    hxc.promise_set(p)
    b.get(timeout_ns=5_000_000_000)
    assert log == ["a", "b"]


def test_continuation_runs_on_worker_thread(L):
    main = threading.get_ident()
    seen = []
    f = hxc.make_ready_future().then(lambda: seen.append(threading.get_ident()))
    f.get(5_000_000_000)
    assert seen and seen[0] != main


def test_failure_propagates_and_skips_continuations(L):
    ran = []
    p = hxc.promise()
    c = p.then(lambda: ran.append(1))
    d = c.then(lambda: ran.append(2))
    hxc.promise_set(p, hxc.HXC_E_CUDA)  # inject a host-side failure
    assert p.wait(5_000_000_000) == hxc.HXC_E_CUDA
    assert c.wait(5_000_000_000) == hxc.HXC_E_DEP_FAILED
    assert d.wait(5_000_000_000) == hxc.HXC_E_DEP_FAILED
    assert ran == []


def test_callback_error_becomes_callback_status(L):
    def boom():
        raise ValueError("x")
    f = hxc.make_ready_future().then(boom)
    assert f.wait(5_000_000_000) == hxc.HXC_E_CALLBACK
    g = f.then(lambda: None)
    assert g.wait(5_000_000_000) == hxc.HXC_E_DEP_FAILED


def test_when_all_joins_and_propagates(L):
    ps = [hxc.promise() for _ in range(5)]
    j = hxc.when_all(ps)
    for p in ps[:4]:
        hxc.promise_set(p)
    assert j.wait(20_000_000) == hxc.HXC_E_TIMEOUT  # one input still open
    hxc.promise_set(ps[4])
    assert j.wait(5_000_000_000) == hxc.HXC_OK
    qs = [hxc.promise() for _ in range(3)]
    k = hxc.when_all(qs)
    hxc.promise_set(qs[0])
    hxc.promise_set(qs[1], hxc.HXC_E_NOMEM)
    hxc.promise_set(qs[2])
    assert k.wait(5_000_000_000) == hxc.HXC_E_DEP_FAILED
    assert hxc.when_all([]).wait(0) == hxc.HXC_OK


def test_wait_timeout_then_success(L):
    p = hxc.promise()
    t0 = time.time()
    assert p.wait(50_000_000) == hxc.HXC_E_TIMEOUT
    assert time.time() - t0 >= 0.04
    assert b"timeout" in L.hxc_last_error()
    threading.Timer(0.05, lambda: hxc.promise_set(p)).start()
    assert p.wait(5_000_000_000) == hxc.HXC_OK


def test_wait_all_reports_first_failure(L):
    fs = [hxc.make_ready_future(), hxc.make_ready_future(hxc.HXC_E_CALLBACK),
          hxc.make_ready_future(hxc.HXC_E_NOMEM)]
    assert hxc.wait_all(fs, 1_000_000_000) == hxc.HXC_E_CALLBACK
    assert hxc.wait_all([hxc.promise()], 10_000_000) == hxc.HXC_E_TIMEOUT


def test_promise_set_twice_rejected(L):
    p = hxc.promise()
    hxc.promise_set(p)
    with pytest.raises(hxc.HxcError):
        hxc.promise_set(p)


def test_many_concurrent_continuations(L):
    n = 2000
    count = []
    lock = threading.Lock()

    def inc():
        with lock:
            count.append(1)
    root = hxc.promise()
    leaves = [root.then(inc) for _ in range(n)]
    hxc.promise_set(root)
    assert hxc.wait_all(leaves, 10_000_000_000) == hxc.HXC_OK
    assert len(count) == n


def test_get_all_devices_without_gpu(L):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    assert hxc.get_all_devices(2, 0) == []
    n = ctypes.c_int(-1)
    assert L.hxc_get_all_devices(2, 0, None, 0, ctypes.byref(n)) == hxc.HXC_E_NODEV
    assert n.value == 0


def test_tuning_registry_and_cache(L, tmp_path):
    old = hxc.tune_get("heat2d.rows")
    try:
        hxc.tune_set("heat2d.rows", 16)
        assert hxc.tune_get("heat2d.rows") == 16
        hxc.tune_set("heat2d.occupancy", 99)  # clamped to the range 4..6
        assert hxc.tune_get("heat2d.occupancy") == 6
        with pytest.raises(hxc.HxcError):
            hxc.tune_set("no.such.knob", 1)
        nested = tmp_path / "t.json"
        nested.write_text('{"sm_90": {"heat2d.rows": 3}, "sm_103": {"heat2d.rows": 64, '
                          '"batch.ctas_per_sm": 6, "future.knob": 1}}')
        hxc.tune_load(nested, 10, 3)
        assert hxc.tune_get("heat2d.rows") == 64 and hxc.tune_get("batch.ctas_per_sm") == 6
        flat = tmp_path / "f.json"
        flat.write_text('{"heat2d.rows": 24}')
        hxc.tune_load(flat, 10, 3)
        assert hxc.tune_get("heat2d.rows") == 24
        bad = tmp_path / "b.json"
        bad.write_text('{"heat2d.rows": }')
        with pytest.raises(hxc.HxcError):
            hxc.tune_load(bad, 10, 3)
    finally:
        hxc.tune_set("heat2d.rows", old)
        hxc.tune_set("heat2d.occupancy", 4)
        hxc.tune_set("batch.ctas_per_sm", 4)


def test_shipped_tuning_cache_parses(L):
    import json
    path = os.path.join(ROOT, "paper_1810_11482_b300", "tune_cache.json")
    data = json.load(open(path))
    assert "sm_103" in data and set(data["sm_103"]) <= {"heat2d.emul", "heat2d.rows",
                                                        "heat2d.occupancy", "heat3d.zchunks",
                                                        "heat3d.variant", "heat3d.variant1",
                                                        "heat3d.steps_per_launch",
                                                        "heat1d.tb_ctas",
                                                        "heat1d.steps_per_launch", "mandel.pair",
                                                        "batch.ctas_per_sm", "batch.block",
                                                        "batch.smem_side"}
    hxc.tune_load(path, 10, 3)
    for k, v in data["sm_103"].items():
        assert hxc.tune_get(k) == v


def test_program_calls_reject_bad_handles():
    L = hxc.lib()
    out = ctypes.c_void_p()
    assert L.hxc_program_create_with_source(None, b"x", b"x.cu", ctypes.byref(out)) == hxc.HXC_E_INVALID
    assert L.hxc_program_create_with_file(None, b"/nonexistent/x.cu", ctypes.byref(out)) == hxc.HXC_E_INVALID
    n = ctypes.c_size_t()
    assert L.hxc_program_build_log(None, None, 0, ctypes.byref(n)) == hxc.HXC_E_INVALID
    assert L.hxc_program_release(None) == hxc.HXC_E_INVALID


def test_host_norms_on_the_worker_pool():
    """hxc_host_norms needs no device: against a long-double sum, on empty,
    short, ragged and long arrays."""
    arrays = [np.zeros(0), np.array([3.0, 4.0]), synth.uniform(50, 1025, lo=-1, hi=1),
              synth.uniform(51, 1 << 20, lo=-2, hi=2), synth.uniform(52, 8191)]
    got = hxc.host_norms(arrays)
    want = [float(np.sqrt(np.sum(a.astype(np.longdouble) ** 2))) for a in arrays]
    assert got[0] == 0.0 and got[1] == 5.0
    assert np.max(np.abs(got[2:] - want[2:]) / np.array(want[2:])) <= 2e-15  # bound 1.4e-15
    L = hxc.lib()
    assert L.hxc_host_norms(None, None, 2, None) == hxc.HXC_E_INVALID


def test_debug_inject_arguments():
    """hxc_debug_inject needs a failure status to arm and disarms with a
    negative count; arming and disarming need no device."""
    L = hxc.lib()
    assert L.hxc_debug_inject(ctypes.c_int64(0), hxc.HXC_OK) == hxc.HXC_E_INVALID
    assert L.hxc_debug_inject(ctypes.c_int64(5), hxc.HXC_E_CUDA) == hxc.HXC_OK
    assert L.hxc_debug_inject(ctypes.c_int64(-1), hxc.HXC_OK) == hxc.HXC_OK
    hxc.debug_inject(-1)


def test_debug_wait_errors_arguments(L):
    """hxc_debug_wait_errors rejects a NULL output and an invalid device
    before touching any device."""
    flags = ctypes.c_uint32()
    assert L.hxc_debug_wait_errors(None, None) == hxc.HXC_E_INVALID
    assert L.hxc_debug_wait_errors(None, ctypes.byref(flags)) == hxc.HXC_E_INVALID


def test_host_run_and_graph_calls_reject_bad_arguments(L):
    """Argument checks of the host-memory run entry points and the graph
    calls come before any device work, so they hold without a GPU."""
    bogus = ctypes.c_void_p(0)
    cfg = hxc.heat2d_cfg(64, 64, 2, 2, 0.2, 4, 2, "fused", None, None)
    host = np.zeros((64, 64))
    out = hxc.c_fut()
    st = hxc.hxc_run_stats()
    assert L.hxc_heat2d_run_host_async(bogus, host.ctypes.data, host.ctypes.data, ctypes.byref(cfg),
                                       None, 0, ctypes.byref(out), ctypes.byref(st)) == hxc.HXC_E_INVALID
    assert L.hxc_heat2d_run_host(bogus, host.ctypes.data, host.ctypes.data, ctypes.byref(cfg),
                                 ctypes.byref(st)) == hxc.HXC_E_INVALID
    assert L.hxc_graph_begin(bogus) == hxc.HXC_E_INVALID
    g = hxc.c_graph()
    assert L.hxc_graph_end(bogus, ctypes.byref(g)) == hxc.HXC_E_INVALID
    assert L.hxc_graph_launch(bogus, 0, None, 0, ctypes.byref(out)) == hxc.HXC_E_INVALID


@pytest.mark.parametrize("r,steps,every,norms,want", [
    # r = 0.2: at most 41 scaled steps in a row (0.2^-41 <= 2^96 < 0.2^-42), so
    # an interval of 100 steps is 3 groups (42 + 42 + 16), each closed once
    (0.2, 1000, 100, True, (0, 970, 30)),
    (0.2, 1000, 100, False, (0, 970, 30)),  # no norms: intervals of 100 all the same
    (0.2, 200, 0, False, (0, 194, 6)),
    (0.2, 43, 0, False, (0, 41, 2)),        # 42 + 1
    (0.2, 42, 0, False, (0, 41, 1)),
    (0.2, 1000, 1, True, (0, 0, 1000)),     # a snapshot after every step
    (0.2, 10, 3, True, (0, 6, 4)),          # intervals 3, 3, 3 (2 scaled + 1) and a last 1
    # r = 1/4: (1/4)^48 = 2^-96 exactly, so 48 scaled steps: 100 = 49 + 49 + 2
    (0.25, 100, 0, False, (0, 97, 3)),
    # r = 0.01: 14 (0.01^-14 = 1e28 <= 2^96 < 1e30): 250 = 100 + 100 + 50,
    # 7 + 7 + 4 groups of at most 15
    (0.01, 250, 0, False, (0, 232, 18)),
    (1e-17, 10, 0, False, (0, 5, 5)),       # 1e17 <= 2^96 < 1e34: groups of 2
    (0.3, 50, 0, False, (50, 0, 0)),        # beyond the stability bound: canonical
    (1e-30, 10, 0, False, (10, 0, 0)),      # one scaled step would grow 1e30 > 2^96
    (-0.1, 5, 0, False, (5, 0, 0)),
    (0.2, 0, 0, False, (0, 0, 0)),
])
def test_heat2d_step_kinds(L, r, steps, every, norms, want):
    """The 2D runs' schedule of scaled and closing steps (host only)."""
    hn = np.zeros(max(1, steps // max(every, 1))) if norms else None
    cfg = hxc.heat2d_cfg(64, 64, 1, 1, r, steps, every, "fused", hn, None)
    assert hxc.heat2d_step_kinds(cfg) == want
    assert sum(want) == steps


def test_heat2d_step_kinds_arguments(L):
    cfg = hxc.heat2d_cfg(64, 64, 1, 1, 0.2, -1, 0, "fused", None, None)
    assert L.hxc_heat2d_step_kinds(ctypes.byref(cfg), (ctypes.c_int64 * 3)()) == hxc.HXC_E_INVALID
    assert L.hxc_heat2d_step_kinds(None, (ctypes.c_int64 * 3)()) == hxc.HXC_E_INVALID


@pytest.mark.parametrize("r,steps,want", [
    # r = 1/4: (1/4)^48 = 2^-96, so 48 scaled steps in a row; an interval of
    # 100 steps is 3 groups (49 + 49 + 2)
    (0.25, 100, (0, 97, 3)),
    # 300 steps: intervals of 128, 128, 44; 3 + 3 + 1 groups
    (0.25, 300, (0, 293, 7)),
    (0.25, 1, (0, 0, 1)),
    # r = 1/2: (1 - 2r)/r = 0, 96 scaled steps in a row: 100 = 97 + 3
    (0.5, 100, (0, 98, 2)),
    (0.6, 10, (10, 0, 0)),     # beyond the stability bound: canonical
    (1e-30, 10, (10, 0, 0)),   # one scaled step would grow 1e30 > 2^96
    (0.25, 0, (0, 0, 0)),
])
def test_heat1d_step_kinds(L, r, steps, want):
    """The 1D runs' schedule of scaled and closing steps (host only)."""
    assert hxc.heat1d_step_kinds(r, steps) == want
    assert sum(want) == steps


def test_heat1d_step_kinds_arguments(L):
    assert L.hxc_heat1d_step_kinds(0.25, -1, (ctypes.c_int64 * 3)()) == hxc.HXC_E_INVALID
    assert L.hxc_heat1d_step_kinds(0.25, 5, None) == hxc.HXC_E_INVALID
