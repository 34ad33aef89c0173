"""The multi-GPU form of the bench splits the workload's nets over the ranks
(one process per GPU) with one demand all-reduce per round: its host logic
on 2 gloo ranks on the CPU - max-over-ranks timing, counts summed over the
ranks, each rank's node-balanced net range of the one forest - and the
reference arm: its ranks other than 0 exit without work, rank 0 prints the
bench line."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    import forestgen as fg
    from paper_2507_13375_gb300 import shard as sh

    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 50.0 * rank
    m = bench.max_over_ranks(local_ms, dist, "cpu")
    total = bench.sum_over_ranks(10.0 + rank, dist, "cpu")
    wl = fg.WORKLOADS[1].scaled(40)
    f = fg.make_forest(wl, 0)
    lo, hi = sh.shard_ranges(f["net_ptr"], world)[rank]
    mine = sh.shard_forest(f, lo, hi)
    parts = [None] * world
    dist.all_gather_object(parts, (lo, hi, int(mine["num_nodes"])))
    if rank == 0:
        with open(out, "w") as fh:
            json.dump({"max_ms": m, "total": total, "parts": parts, "V": int(f["num_nodes"]),
                       "N": int(f["num_nets"])}, fh)
    dist.barrier()
    dist.destroy_process_group()


def test_ranks_on_two_gloo_ranks(tmp_path):
    out = str(tmp_path / "r.json")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    with open(out) as fh:
        r = json.load(fh)
    assert r["max_ms"] == 150.0                     # the slower rank's time
    assert r["total"] == 21.0                       # a count of both ranks
    (lo0, hi0, v0), (lo1, hi1, v1) = r["parts"]     # one forest, split by nets
    assert lo0 == 0 and hi0 == lo1 and hi1 == r["N"] and v0 + v1 == r["V"]


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0
    assert p.stdout.strip() == ""


def test_reference_arm_line_on_rank0():
    """Rank 0 of the reference arm (the oracle on the host cores) prints one JSON
    line with the bench keys, a cpu_baseline describing the run and an e2e of
    its own value with no host-device bytes."""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--workload", "1"], env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "nets/s" and d["higher_is_better"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "nets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "plain-64x64x6-2k"
