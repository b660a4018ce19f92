"""Host logic of bench.py that needs no GPU."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

MOVE_KERNELS = ["move_thread", "move_group", "move_half", "move_warp", "move_mid", "move_block", "move_xl",
                "move_cluster", "move_hub"]


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


def test_stored_traffic_matches_its_capture_range():
    tj = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    default = dict(group_max=64, half_max=128, warp_max=256)
    for wl, ents in tj.items():
        if wl.startswith("_"):
            continue
        for kern, ent in ents.items():
            assert ent["bin_degrees"] == bench.move_bin_degrees(kern, default), (wl, kern)
            assert ent["dram_bytes_per_launch"] == ent["dram_read_per_launch"] + ent["dram_write_per_launch"] or \
                abs(ent["dram_bytes_per_launch"] - ent["dram_read_per_launch"] - ent["dram_write_per_launch"]) <= 1
