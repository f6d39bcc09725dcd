"""Host logic of the benchmark that needs no GPU: the roofline's DRAM traffic
is taken from the committed ncu summary only while the kernel source and the
2D tiling are the ones that summary was captured with."""

from __future__ import annotations

import hashlib
import importlib.util
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_host_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_traffic_only_for_the_profiled_source_and_tiling(tmp_path):
    b = _bench()
    src = tmp_path / "stream.cu"
    src.write_bytes(b"// kernel source as profiled\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    prof = tmp_path / "prof.md"
    prof.write_text(f"source_sha256: {sha}\ntraffic_bytes_per_launch: 5.251e8\ntiling: 1,0,0\n")
    b.KERNEL_SRC, b.PROFILE_2D = str(src), str(prof)
    assert b._profile_traffic((1, 0, 0)) == 5.251e8  # bytes per 2D L = 16384 launch
    assert b._profile_traffic((1, 1, 0)) is None  # another tiling
    src.write_bytes(b"// kernel source as profiled\n\n")  # a kernel source other than the one profiled
    assert b._profile_traffic((1, 0, 0)) is None


def test_committed_profile_names_a_source_and_tiling():
    b = _bench()
    text = open(b.PROFILE_2D).read()
    assert re.search(r"source_sha256:\s*[0-9a-f]{64}", text)
    assert re.search(r"traffic_bytes_per_launch:\s*[0-9.eE+]+", text)
    assert re.search(r"tiling:\s*\d+,\d+,\d+", text)


def test_attempts_per_step_matches_the_workload():
    b = _bench()
    assert b.ATTEMPTS_PER_STEP == 3 * 200 * 16384 ** 2 + 100 * 512 ** 3


def test_reference_line_carries_the_same_config(capsys, monkeypatch):
    """Both arms print `_config(ws)`: the workload of a step and nothing
    measured, so the two lines name the same configuration."""
    import argparse
    import json

    b = _bench()
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.setattr(b, "_cpu_baseline", lambda sample=1: {"value": 1.0})
    b.run_reference(argparse.Namespace(steps=2, warmup=1))
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["config"] == b._config(1)
    assert set(b._config(1)) == {"workload", "attempts_per_step", "l2", "parallelism"}
    assert line["metric"] == b.METRIC and line["unit"] == b.UNIT and line["higher_is_better"] is True
    src = open(os.path.join(ROOT, "bench.py")).read()
    assert src.count('"config": _config(ws)') == 2  # the reference line and this arm's line
