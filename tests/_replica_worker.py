"""One rank of the world-size-2 replica test (launched by torchrun with the gloo backend on CPU):
combines a rank-dependent duration, checks the reference arm's rank rule and writes one JSON
file per rank into $CS_REPLICA_OUT."""
import json
import os
import sys

import torch.distributed as dist

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2305_06482_gb300 import replicas  # noqa: E402


def main():
    rank = int(os.environ["RANK"])
    world = int(os.environ["WORLD_SIZE"])
    dist.init_process_group("gloo")
    ms_local = 10.0 + 15.0 * rank          # rank 1 is the slowest
    ms = replicas.slowest_ms(ms_local, dist)
    value = replicas.seconds_per_recon(ms, 3, world)
    seed = replicas.replica_seed(1, rank)
    seeds = [None] * world
    dist.all_gather_object(seeds, seed)
    # the reference arm: every rank but 0 returns without work or output
    ref_silent = None
    if rank != 0:
        import contextlib
        import io
        import bench
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            bench.run_reference(None, dict(bench.WORKLOAD), rank, world)
        ref_silent = buf.getvalue() == ""
    dist.barrier()
    with open(os.path.join(os.environ["CS_REPLICA_OUT"], f"rank{rank}.json"), "w") as fh:
        json.dump({"rank": rank, "world": world, "slowest_ms": ms, "value": value, "seeds": seeds,
                   "ref_silent": ref_silent}, fh)
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
