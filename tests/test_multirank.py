"""The N > 1 path of bench.py on CPU: one process per rank over gloo, world size 2.

The replicas share no data-path collective; what crosses ranks is the barrier,
the whole-job reduction (slowest rank's time, sum of every rank's work) and, for
the reference arm, the rule that rank 0 alone runs and prints.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _combine_worker(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    # rank r took 10 + 5r ms for (r + 1) * 1e6 evals over (r + 1) * 100 universes
    res = bench._combine_ranks(dist, 10.0 + 5.0 * rank, (rank + 1) * 1e6, (rank + 1) * 100.0)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, res))


def test_combine_ranks_gloo_world_2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_combine_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the same whole-job figures: max time, summed work
    assert got[0] == got[1] == (15.0, 3e6, 300.0)


def test_replica_seeds_are_distinct():
    import bench

    seeds = [bench.replica_seed(r) for r in range(8)]
    assert len(set(seeds)) == 8 and seeds[0] == 0


@pytest.mark.timeout(600)
def test_reference_arm_under_torchrun_two_ranks():
    """bench.py --impl reference launched as the driver launches N > 1: rank 0 alone runs the
    CPU oracle and prints one JSON line; rank 1 exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
