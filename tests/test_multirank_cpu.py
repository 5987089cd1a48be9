"""Host-side logic of the multi-GPU path (independent replicas), run as two
gloo ranks on the CPU: the job time is the slowest rank's, the throughput
counts every rank's maps, replicas draw disjoint seeds, and the reference arm
runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import bench
rank, world, _ = bench.dist_env()
d = bench.init_dist(world, None)
t = bench.max_over_ranks(d, 10.0 * (rank + 1), None)        # rank r "took" 10 (r + 1) ms
base = bench.rank_seed_base(rank)
print(json.dumps({"rank": rank, "world": world, "t_max": t, "seeds": [base, base + 505],
                  "value": bench.job_throughput(world, 100, t)}), flush=True)
bench.finish_dist(d)
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def run_ranks(code, world, extra_args=()):
    port = free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", code, ROOT, *extra_args], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=240)
        assert p.returncode == 0, err[-2000:]
        outs.append(out)
    return outs


def test_two_gloo_ranks_max_time_throughput_and_seeds():
    outs = run_ranks(WORKER, 2)
    res = sorted((json.loads(o.strip().splitlines()[-1]) for o in outs), key=lambda d: d["rank"])
    assert [d["t_max"] for d in res] == [20.0, 20.0]              # the slowest rank's time on every rank
    assert all(d["value"] == pytest.approx(2 * 100 / 0.020) for d in res)
    (a0, a1), (b0, b1) = res[0]["seeds"], res[1]["seeds"]
    assert a1 < b0 or b1 < a0                                      # disjoint seed ranges


REF_WORKER = r"""
import sys
sys.path.insert(0, sys.argv[1])
sys.argv = ["bench.py", "--impl", "reference", "--workload", "box64_cap0.1_trilinear", "--steps", "2",
            "--warmup", "1", "--ref-budget-s", "30"]
import bench
bench.main()
"""


def test_reference_arm_prints_on_rank_zero_only():
    outs = run_ranks(REF_WORKER, 2)
    lines = [[l for l in o.splitlines() if l.startswith("{")] for o in outs]
    assert len(lines[0]) == 1 and lines[1] == []
    d = json.loads(lines[0][0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
