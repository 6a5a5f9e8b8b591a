"""The host side of the library (future layer, worker pool, tuning registry,
host norms, PNG writer) under ThreadSanitizer and under AddressSanitizer +
UndefinedBehaviorSanitizer, without a GPU.

The C++ sources are recompiled here with g++ and the sanitizer, linked with
the library's CUDA objects (built by paper_1810_11482_b300.build, not
instrumented) into a test program that drives the public C API from many
threads: promises set from other threads, chains of then-continuations,
when_all over mixed ready / pending / failing futures, bounded waits that
time out, dependency failure propagation, concurrent knob updates.  Any
sanitizer report fails the test."""
import glob
import os
import shutil
import subprocess
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1810_11482_b300", "csrc")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")

DRIVER = r"""
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <thread>
#include <vector>

#include "hxc.h"

#define CHECK(c)                                                        \
    do {                                                                \
        if (!(c)) {                                                     \
            std::fprintf(stderr, "check failed at line %d: %s\n", __LINE__, #c); \
            std::exit(3);                                               \
        }                                                               \
    } while (0)

static std::atomic<int> g_calls{0};
static hxc_status count_fn(void *) { g_calls++; return HXC_OK; }
static hxc_status fail_fn(void *) { return HXC_E_INVALID; }
static hxc_status add_fn(void *p) { static_cast<std::atomic<int> *>(p)->fetch_add(1); return HXC_OK; }

static void chains(int id) {
    for (int round = 0; round < 40; round++) {
        hxc_future p;
        CHECK(hxc_promise_create(&p) == HXC_OK);
        std::atomic<int> hits{0};
        std::vector<hxc_future> tails;
        hxc_future prev = p;
        hxc_future_retain(prev);
        for (int k = 0; k < 6; k++) {
            hxc_future nx;
            CHECK(hxc_future_then(prev, add_fn, &hits, &nx) == HXC_OK);
            hxc_future_release(prev);
            prev = nx;
        }
        tails.push_back(prev);
        hxc_future ready, bad, failing;
        CHECK(hxc_make_ready_future(HXC_OK, &ready) == HXC_OK);
        CHECK(hxc_promise_create(&bad) == HXC_OK);
        CHECK(hxc_future_then(p, fail_fn, nullptr, &failing) == HXC_OK);
        hxc_future parts[3] = {prev, ready, p}, all, all_bad;
        CHECK(hxc_when_all(parts, 3, &all) == HXC_OK);
        hxc_future parts2[2] = {all, bad};
        CHECK(hxc_when_all(parts2, 2, &all_bad) == HXC_OK);
        // a bounded wait on an unset promise times out
        CHECK(hxc_future_wait(bad, 1000000) == HXC_E_TIMEOUT);
        std::thread setter([&] {
            std::this_thread::sleep_for(std::chrono::microseconds(50 * (id % 3)));
            CHECK(hxc_promise_set(p, HXC_OK) == HXC_OK);
            CHECK(hxc_promise_set(bad, HXC_E_CUDA) == HXC_OK);
        });
        CHECK(hxc_future_wait(all, -1) == HXC_OK);
        CHECK(hits.load() == 6);
        CHECK(hxc_future_wait(failing, -1) == HXC_E_CALLBACK);
        CHECK(hxc_future_wait(all_bad, -1) == HXC_E_DEP_FAILED);
        hxc_future after_bad;
        CHECK(hxc_future_then(all_bad, count_fn, nullptr, &after_bad) == HXC_OK);
        CHECK(hxc_future_wait(after_bad, -1) == HXC_E_DEP_FAILED);  // never ran
        setter.join();
        for (hxc_future f : {prev, ready, bad, failing, all, all_bad, after_bad, p})
            hxc_future_release(f);
    }
}

static void knobs(int id) {
    for (int i = 0; i < 2000; i++) {
        CHECK(hxc_tune_set("heat2d.rows", 8 + (i + id) % 9) == HXC_OK);
        int64_t v = 0;
        CHECK(hxc_tune_get("batch.ctas_per_sm", &v) == HXC_OK);
    }
}

static void norms(int id) {
    std::vector<double> a(100000 + 37 * id), b(1025);
    for (size_t i = 0; i < a.size(); i++) a[i] = std::sin(0.001 * (double)(i + id));
    for (size_t i = 0; i < b.size(); i++) b[i] = 1.0;
    const double *arrs[2] = {a.data(), b.data()};
    const int64_t counts[2] = {(int64_t)a.size(), (int64_t)b.size()};
    double out[2];
    for (int r = 0; r < 20; r++) {
        CHECK(hxc_host_norms(arrs, counts, 2, out) == HXC_OK);
        CHECK(out[1] == std::sqrt(1025.0));
    }
}

static void png(int id, const char *dir) {
    std::vector<uint8_t> img(3 * 97 * 61);
    for (size_t i = 0; i < img.size(); i++) img[i] = (uint8_t)(i * 7 + id);
    char path[4096];
    std::snprintf(path, sizeof path, "%s/t%d.png", dir, id);
    for (int r = 0; r < 5; r++) CHECK(hxc_png_write(img.data(), 97, 61, 1, path) == HXC_OK);
}

int main(int argc, char **argv) {
    std::vector<std::thread> th;
    for (int i = 0; i < 8; i++) th.emplace_back(chains, i);
    for (int i = 0; i < 4; i++) th.emplace_back(knobs, i);
    for (int i = 0; i < 4; i++) th.emplace_back(norms, i);
    for (int i = 0; i < 4; i++) th.emplace_back(png, i, argv[1]);
    for (auto &t : th) t.join();
    hxc_tune_set("heat2d.rows", 8);
    std::printf("ok %d\n", g_calls.load());
    return 0;
}
"""


def cuda_objects():
    from paper_1810_11482_b300 import build
    build.build()
    objs = sorted(glob.glob(os.path.join(ROOT, "_build", "*.cu.o")))
    assert objs, "no CUDA objects were built"
    return objs


def build_and_run(san, tmp):
    flags = ["-O1", "-g", "-std=c++17", "-fno-omit-frame-pointer", "-fsanitize=" + san,
             "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-I", os.path.join(CUDA, "include")]
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cpp"))) + [os.path.join(tmp, "driver.cpp")]
    with open(srcs[-1], "w") as fh:
        fh.write(DRIVER)

    def cc(src):
        obj = os.path.join(tmp, os.path.basename(src) + ".o")
        subprocess.check_call(["g++"] + flags + ["-c", src, "-o", obj])
        return obj

    with ThreadPoolExecutor(max_workers=8) as ex:
        objs = list(ex.map(cc, srcs))
    exe = os.path.join(tmp, "t")
    subprocess.check_call(["g++", "-fsanitize=" + san, "-o", exe] + objs + cuda_objects() +
                          ["-L", os.path.join(CUDA, "lib64"), "-lcudart", "-lz", "-ldl",
                           "-lpthread"])
    out = os.path.join(tmp, "png")
    os.makedirs(out)
    env = dict(os.environ)
    env["TSAN_OPTIONS"] = "halt_on_error=1 exitcode=66"
    env["ASAN_OPTIONS"] = "detect_leaks=0 halt_on_error=1"
    env["UBSAN_OPTIONS"] = "halt_on_error=1 print_stacktrace=1"
    r = subprocess.run([exe, out], capture_output=True, text=True, timeout=600, env=env)
    return r


@pytest.mark.parametrize("san", ["thread", "address,undefined"])
def test_host_runtime_under_sanitizer(san):
    if not shutil.which("g++"):
        pytest.skip("g++ not available")
    with tempfile.TemporaryDirectory() as tmp:
        r = build_and_run(san, tmp)
    report = r.stdout + r.stderr
    assert r.returncode == 0 and "WARNING: ThreadSanitizer" not in report and \
        "runtime error" not in report and "ERROR: AddressSanitizer" not in report, report[-4000:]
    assert r.stdout.startswith("ok")
