"""The benchmark's multi-rank path on CPU: two gloo ranks launched the way
torchrun does (RANK / WORLD_SIZE / MASTER_* in the environment) agree on the
slowest rank's time, report the whole-job value from it, and the reference arm
prints exactly one line, from rank 0."""

from __future__ import annotations

import json
import os
import socket
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _launch(code: str, world: int = 2, extra_env=None, timeout=180):
    port = _free_port()
    procs = []
    for rank in range(world):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), SPN_BENCH_BACKEND="gloo",
                   PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
        env.update(extra_env or {})
        procs.append(subprocess.Popen([sys.executable, "-c", code], cwd=ROOT, env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=timeout)
        assert p.returncode == 0, err
        outs.append(out)
    return outs


def test_max_over_ranks_and_job_value_with_gloo():
    code = textwrap.dedent("""
        import json, bench
        dist, rank, ws, local = bench._dist()
        ms = [12.5, 40.0][rank]  # rank 1 is the slow one
        slow = bench.max_over_ranks(dist, ms, device="cpu")
        print(json.dumps({"rank": rank, "ws": ws, "ms": slow, "value": bench.job_value(ws, 5, 10**9, slow)}))
        dist.destroy_process_group()
    """)
    outs = [json.loads(o.strip().splitlines()[-1]) for o in _launch(code)]
    assert [o["rank"] for o in outs] == [0, 1]
    assert all(o["ws"] == 2 and o["ms"] == 40.0 for o in outs)
    assert all(o["value"] == pytest.approx(2 * 5 * 10**9 / (40.0 * 1e6)) for o in outs)


def test_reference_arm_prints_once_from_rank_zero():
    code = textwrap.dedent("""
        import sys, bench
        sys.argv = ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"]
        bench.L2D, bench.L3D = 64, 16          # a tiny sample keeps the CPU oracle quick
        bench.main()
    """)
    outs = _launch(code)
    lines = [[ln for ln in o.splitlines() if ln.startswith("{")] for o in outs]
    assert len(lines[0]) == 1 and lines[1] == []
    rec = json.loads(lines[0][0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0
