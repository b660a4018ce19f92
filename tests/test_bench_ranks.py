"""bench.py's multi-rank path, on CPU: two gloo ranks launched by
torch.distributed.run as bench.py is under torchrun.  The workload runs as
independent replicas (a single graph does not shard), so what crosses the
ranks is only the timing: every rank must report the slowest rank's time,
the whole-job rate must count every rank's units over that time, and the
reference arm must leave ranks other than 0 idle."""
import json
import os
import socket
import subprocess
import sys

import pytest

pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_single_rank_helpers():
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_rate(520_765_898, 5, 1, 0.6128) == pytest.approx(520.765898 * 5 / 0.6128)
    assert bench.job_rate(1_000, 2, 4, 0.5) == pytest.approx(1e-6 * 1_000 * 2 * 4 / 0.5)


def test_two_gloo_ranks_report_the_slowest_rank(tmp_path):
    env = dict(os.environ, OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(ROOT, "tests", "rank_worker.py"), str(tmp_path)]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    outs = [json.loads((tmp_path / f"rank{k}.json").read_text()) for k in range(2)]
    for o in outs:
        assert o["world"] == 2
        assert o["slowest_ms"] == 150.0
        assert o["rate"] == pytest.approx(1_000_000 * 5 * 2 / 0.150 / 1e6)
    assert outs[0]["ref"] is None and outs[1]["ref"] == 0
