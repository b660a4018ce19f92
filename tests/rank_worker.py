"""One rank of the two-rank gloo job in tests/test_bench_ranks.py, launched
by torch.distributed.run on CPU the way bench.py is launched under torchrun
(RANK, WORLD_SIZE and MASTER_* from the environment).  Writes what it saw to
<out_dir>/rank<r>.json."""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch.distributed as dist  # noqa: E402

import bench  # noqa: E402


def main(out_dir: str) -> None:
    world = int(os.environ["WORLD_SIZE"])
    rank = int(os.environ["RANK"])
    dist.init_process_group("gloo")
    try:
        dist.barrier()
        ms = [120.0, 150.0][rank]  # rank 1 is the slower one
        slowest = bench.max_over_ranks(ms, world, "cpu")
        rate = bench.job_rate(1_000_000, 5, world, slowest / 1e3)
        dist.barrier()
        # the reference arm: every rank but 0 returns at once, without work
        ref = bench.run_reference(None, "rmat24") if rank != 0 else None
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"rank": rank, "world": world, "slowest_ms": slowest, "rate": rate, "ref": ref}, f)
    finally:
        dist.destroy_process_group()


if __name__ == "__main__":
    main(sys.argv[1])
