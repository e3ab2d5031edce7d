"""Failure paths, injected on the host (FSPARSE_FAULT): an allocation that
fails, and a look-back wait that runs out because a predecessor tile never
publishes.  Nothing faults, traps or hangs the GPU: the bounded wait gives up,
the call returns its status, and the next call on the same context is exact."""
import time

import numpy as np
import pytest

import oracle
from gpu_util import assert_same, config, gpu_assemble, to_dev
from paper_1406_1066_gb300 import fsparse, inputs

pytestmark = pytest.mark.gpu


def test_injected_allocation_failure(monkeypatch):
    t = inputs.random_small(5000, 60, 50, 71, dup=0.3)
    monkeypatch.setenv("FSPARSE_FAULT", "alloc")
    with pytest.raises(fsparse.FsparseError) as e:
        fsparse.assemble(to_dev(t.ii), to_dev(t.jj), to_dev(t.s), t.m, t.n)
    assert e.value.status == fsparse.ERR_NOMEM
    monkeypatch.delenv("FSPARSE_FAULT")
    assert_same(gpu_assemble(t.ii, t.jj, t.s, t.m, t.n), oracle.assemble(t.ii, t.jj, t.s, t.m, t.n))


def test_injected_bad_index(monkeypatch):
    """FSPARSE_FAULT=index seeds the status word: a valid input takes the
    bad-index return (no plan), and the next call is exact."""
    t = inputs.random_small(6000, 70, 50, 76, dup=0.3)
    monkeypatch.setenv("FSPARSE_FAULT", "index")
    for strategy in (1, 2):
        with config(strategy=strategy):
            with pytest.raises(fsparse.FsparseError) as e:
                fsparse.assemble(to_dev(t.ii), to_dev(t.jj), to_dev(t.s), t.m, t.n)
            assert e.value.status == fsparse.ERR_INDEX
    monkeypatch.delenv("FSPARSE_FAULT")
    assert_same(gpu_assemble(t.ii, t.jj, t.s, t.m, t.n), oracle.assemble(t.ii, t.jj, t.s, t.m, t.n))


def test_injected_lookback_timeout(monkeypatch):
    """The column-pointer scan of the onesweep path spans several tiles
    (8000 columns); with tile 0 withheld the others wait out their bound."""
    t = inputs.mesh3d(20, 72)
    with config(strategy=1):
        monkeypatch.setenv("FSPARSE_FAULT", "timeout")
        t0 = time.perf_counter()
        with pytest.raises(fsparse.FsparseError) as e:
            fsparse.symbolic(to_dev(t.ii), to_dev(t.jj), t.m, t.n)
        waited = time.perf_counter() - t0
        assert e.value.status == fsparse.ERR_TIMEOUT
        assert waited < 60.0
        monkeypatch.delenv("FSPARSE_FAULT")
        g = gpu_assemble(t.ii, t.jj, t.s, t.m, t.n)
    assert_same(g, oracle.assemble(t.ii, t.jj, t.s, t.m, t.n))


def test_injected_digit_pass_timeout(monkeypatch):
    """The first digit pass of the onesweep sort withholds tile 0's counts:
    the following tiles' waits run out, the pass leaves positions unwritten,
    and the kernels after it read whatever the pool memory held.  The call
    returns FSPARSE_ERR_TIMEOUT with every access in bounds, and the next
    call on the same context is exact."""
    wide = inputs.random_small(200_000, 2**30 - 1, 2**30 - 1, 74, dup=0.2)   # 60-bit keys first
    t = inputs.random_small(80_000, 500, 300, 75, dup=0.4)
    with config(strategy=1):
        assert_same(gpu_assemble(wide.ii, wide.jj, wide.s, wide.m, wide.n),
                    oracle.assemble(wide.ii, wide.jj, wide.s, wide.m, wide.n))
        monkeypatch.setenv("FSPARSE_FAULT", "timeout_sort")
        t0 = time.perf_counter()
        with pytest.raises(fsparse.FsparseError) as e:
            fsparse.assemble(to_dev(t.ii), to_dev(t.jj), to_dev(t.s), t.m, t.n)
        waited = time.perf_counter() - t0
        assert e.value.status == fsparse.ERR_TIMEOUT
        assert waited < 60.0
        monkeypatch.delenv("FSPARSE_FAULT")
        g = gpu_assemble(t.ii, t.jj, t.s, t.m, t.n)
    assert_same(g, oracle.assemble(t.ii, t.jj, t.s, t.m, t.n))


@pytest.mark.parametrize("strategy,phases", [
    (2, ["bucket_count", "bucket_scatter", "bucket_emit", "numeric_fold"]),
    (1, ["digit_hist", "digit_passes", "emit", "jcS_scan", "numeric_fold"])], ids=["bucket", "onesweep"])
def test_phase_timing(monkeypatch, strategy, phases):
    """FSPARSE_TIMING=1 records the device time of every phase of the call."""
    t = inputs.mesh3d(16, 73)
    with config(strategy=strategy):
        monkeypatch.setenv("FSPARSE_TIMING", "1")
        gpu_assemble(t.ii, t.jj, t.s, t.m, t.n)
        got = fsparse.fsparse_last_timings()
        monkeypatch.delenv("FSPARSE_TIMING")
        assert [n for n, _ in got] == phases
        assert all(ms >= 0.0 for _, ms in got) and sum(ms for _, ms in got) > 0.0
        gpu_assemble(t.ii, t.jj, t.s, t.m, t.n)
        assert fsparse.fsparse_last_timings() == []          # a call without it records nothing
