"""Host logic of bench.py that needs no GPU."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

MOVE_KERNELS = ["move_thread", "move_group", "move_half", "move_warp", "move_mid", "move_block", "move_wide",
                "move_hub"]


def test_move_bins_tile_the_degrees():
    """For every valid threshold triple the local-moving bins cover degrees
    1.. without gaps or overlaps (empty bins have hi < lo), in the library's
    bin order."""
    for gm in (16, 32, 48, 64):
        for hm in sorted({gm, 96, 128}):
            if hm < gm:
                continue
            for wm in (128, 256):
                if wm < hm:
                    continue
                sched = dict(group_max=gm, half_max=hm, warp_max=wm)
                nxt = 1
                for k in MOVE_KERNELS:
                    lo, hi = bench.move_bin_degrees(k, sched)
                    assert lo == nxt, (sched, k)
                    if hi is None:
                        assert k == "move_hub"
                        break
                    assert hi >= lo - 1
                    nxt = hi + 1
    assert bench.move_bin_degrees("merge_big", dict(group_max=64, half_max=128, warp_max=256)) is None


def test_reference_arm_line_on_cpu():
    """The reference arm times the CPU oracle only; its JSON line carries the
    contract's keys (run here on the small planted-partition workload)."""
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "sbm1000",
                        "--steps", "2", "--warmup", "3"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 3
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_first_launch_entries_follow_the_bucket_schedule():
    """The entries of the first launches of a bin kernel (iteration 0 of
    pass 0, every vertex unprocessed), used to scale a small ncu capture,
    follow the schedule's bucket hash: checked against the oracle's bucket
    function vertex by vertex."""
    import numpy as np
    import oracle
    from paper_2501_19004_gb300 import graphgen as gg
    g = gg.rmat(13, 16, seed=7)
    deg = np.diff(g.offsets)
    sched = dict(group_max=64, half_max=128, warp_max=256)
    for kern, (lo, hi) in (("move_block", (1025, 4096)), ("move_mid", (257, 1024))):
        want = [0] * 4
        for i in range(g.n):
            if lo <= deg[i] <= hi:
                want[oracle.bucket(i, 0, 0, 0, 4)] += int(deg[i])
        assert bench.first_launch_entries(g, kern, sched, 4) == want


def test_stored_traffic_describes_the_current_wide_kernel():
    """profiles/traffic.json holds the DRAM bytes per entry of the dominant
    kernel of the default workload; it must have been taken on the current
    move.cu and headers (the bench reports no traffic figure otherwise)."""
    per_entry, rec = bench.stored_traffic("move_wide")
    assert per_entry is not None and rec is not None
    assert 0 < per_entry < 100
    assert "move.cu" in bench.kernel_sources("move_wide")
    assert bench.kernel_sources("move_hub")[0] == "big.cu" and bench.kernel_sources("merge_mid")[0] == "aggr.cu"
