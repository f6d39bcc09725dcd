"""Host logic of the benchmark that needs no GPU: the roofline's DRAM traffic
is taken from the committed ncu summary only while the kernel source and the
2D tiling are the ones that summary was captured with."""

from __future__ import annotations

import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_host_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_traffic_only_for_the_profiled_source_and_tiling(tmp_path):
    b = _bench()
    t = b._profile_traffic((1, 0, 0))
    assert t is not None and 4e8 < t < 7e8  # bytes per 2D L = 16384 launch
    assert b._profile_traffic((1, 1, 0)) is None  # another tiling
    # a kernel source other than the one profiled
    src = tmp_path / "stream.cu"
    src.write_bytes(open(b.KERNEL_SRC, "rb").read() + b"\n")
    b.KERNEL_SRC = str(src)
    assert b._profile_traffic((1, 0, 0)) is None


def test_attempts_per_step_matches_the_workload():
    b = _bench()
    assert b.ATTEMPTS_PER_STEP == 3 * 200 * 16384 ** 2 + 100 * 512 ** 3
