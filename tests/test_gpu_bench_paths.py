"""The benchmark's multi-GPU step (LPT-sharded partitions, score gather,
K-means block-sum exchange) run on one GPU: with one rank it owns every
partition, so it must pick the same best model as the one-GPU step; both
lines are well formed.  The exchanges themselves are covered with two gloo
ranks on CPU (tests/test_dist.py)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*extra):
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "2", "--warmup", "1", "--no-cpu-baseline",
           "--no-fp64-path", "--no-serve", *extra]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


@pytest.mark.parametrize("workload,size", [("bkrr2", ["--n", "8192", "--p", "4", "--t", "512"]),
                                           ("kkrr2", ["--n", "16384", "--p", "8", "--t", "1024"])])
def test_sharded_step_on_one_gpu_matches_the_plain_step(workload, size):
    plain = _bench("--workload", workload, *size)
    shard = _bench("--workload", workload, "--shard", *size)
    for line in (plain, shard):
        assert line["value"] > 0 and line["failed_solves"] == 0
        assert line["roofline"]["kernel"] in line["stages_ms_per_step"]
    assert shard["best_model"] == plain["best_model"]
    assert shard["best_mse"] == pytest.approx(plain["best_mse"], rel=1e-9)
