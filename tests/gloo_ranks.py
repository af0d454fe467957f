"""Rank program for tests/test_multiprocess.py (run under torch.distributed.run): the
bench's multi-process helpers over gloo on the CPU -- process-group set-up from the
launcher's environment, the barrier, and the max over ranks of a per-rank time."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def main():
    world = int(os.environ["WORLD_SIZE"])
    rank, w, local = bench.dist_setup(world)
    bench.barrier(w)
    t = bench.max_over_ranks(1.5 + rank, w)      # per-rank "times" 1.5, 2.5, ...
    bench.barrier(w)
    print(json.dumps({"rank": rank, "world": w, "local": local, "max": t}), flush=True)
    import torch.distributed as dist
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
