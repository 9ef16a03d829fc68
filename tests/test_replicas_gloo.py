"""The multi-rank path of the benchmark on CPU: two ranks under torchrun with the gloo backend.
Each rank keeps its own duration; the job's time is the slowest rank's, the throughput counts
every rank's reconstructions, seeds differ per rank, and the reference arm runs on rank 0 only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_two_rank_replicas_with_gloo(tmp_path):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--standalone", "--local-addr", "127.0.0.1",
           "--nnodes=1", "--nproc-per-node=2", os.path.join(ROOT, "tests", "_replica_worker.py")]
    env = dict(os.environ, OMP_NUM_THREADS="1", CS_REPLICA_OUT=str(tmp_path))
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(open(tmp_path / f"rank{k}.json").read()) for k in range(2)]
    assert sorted(d["rank"] for d in lines) == [0, 1]
    for d in lines:
        assert d["world"] == 2
        assert d["slowest_ms"] == 25.0                       # max over ranks
        assert abs(d["value"] - 25.0 / 1e3 / (3 * 2)) < 1e-15   # 2 ranks x 3 steps in 25 ms
        assert d["seeds"] == [1, 18] and len(set(d["seeds"])) == 2
    assert [d["ref_silent"] for d in lines if d["rank"] == 1] == [True]
