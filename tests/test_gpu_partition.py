"""Sec. 5.1.2 partition benchmark (Algorithm 1) against the oracle: the
futures path and the native-stream path on ragged and empty partitions, in
place, with dependencies, and on the largest vector of the benchmark."""
import time

import numpy as np
import pytest

import oracle
from paper_1810_11482_b300 import hxc, synth

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps
TOL = 8 * EPS  # sin, cos: a few ulp each; squares, sum and root: one rounding each


@pytest.fixture(scope="module")
def dev():
    devs = hxc.get_all_devices(2, 0)
    assert devs
    return devs[0]


@pytest.mark.parametrize("n,parts", [(0, 4), (3, 4), ((1 << 21) + 77, 4), ((1 << 21) + 77, 3),
                                     (100003, 7), (1 << 20, 1)])
def test_futures_and_native_match_oracle(dev, n, parts):
    x = hxc.host_empty(max(n, 1))[:n]
    synth.partition_input(n, out=x)
    want = oracle.partition_k(x)
    work = dev.buffer(max(n, 1) * 8)
    r1 = hxc.host_empty(max(n, 1))[:n]
    r1[:] = -1.0
    hxc.partition_run(dev, x, r1, parts, work).get()
    r2 = hxc.host_empty(max(n, 1))[:n]
    r2[:] = -2.0
    hxc.partition_run_native(dev, x, r2, parts, work)
    assert np.array_equal(r1, r2)  # same kernel, same partitions: identical bits
    if n:
        assert np.max(np.abs(r1 - want)) <= TOL
        assert np.max(np.abs(r1 - 1.0)) <= TOL
    assert np.array_equal(x, synth.partition_input(n))  # the input is left alone


def test_in_place_and_pageable_host_memory(dev):
    n = 3 * 65536 + 5
    x = synth.partition_input(n)  # pageable: correct, without overlap
    want = oracle.partition_k(x)
    work = dev.buffer(n * 8)
    hxc.partition_run(dev, x, x, 4, work).get()
    assert np.max(np.abs(x - want)) <= TOL


def test_first_writes_wait_for_dependencies(dev):
    n = 1 << 20
    x = hxc.host_empty(n)
    x[:] = np.nan
    r = hxc.host_empty(n)
    gate = hxc.promise()
    f = hxc.partition_run(dev, x, r, 4, dev.buffer(n * 8), deps=[gate])
    time.sleep(0.05)
    assert not f.is_ready()
    synth.partition_input(n, out=x)  # the input is written before the gate opens
    hxc.promise_set(gate)
    f.get()
    assert not np.isnan(r).any()
    assert np.max(np.abs(r - 1.0)) <= TOL


def test_largest_vector_of_the_benchmark(dev):
    """n = 2^8 * 1024 * 256 * 4 = 2^28 (2 GiB each way): every element is 1
    within the bound, and sampled elements match the oracle."""
    n = synth.partition_sizes([8])[0]
    x = hxc.host_empty(n)
    synth.partition_input(n, out=x)
    r = hxc.host_empty(n)
    hxc.partition_run(dev, x, r, 4, dev.buffer(n * 8)).get()
    assert np.max(np.abs(r - 1.0)) <= TOL
    idx = np.concatenate([np.arange(1000), n - 1 - np.arange(1000),
                          (synth.uniform(12, 4000) * n).astype(np.int64)])
    assert np.max(np.abs(r[idx] - oracle.partition_k(x[idx]))) <= TOL


def test_argument_checks(dev):
    x = np.zeros(16)
    with pytest.raises(hxc.HxcError):
        hxc.partition_run(dev, x, x, 4, dev.buffer(8))  # work buffer too small
    with pytest.raises(hxc.HxcError):
        hxc.partition_run(dev, x, x, 0, dev.buffer(16 * 8))  # no partition
