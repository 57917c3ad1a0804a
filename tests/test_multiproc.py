"""The multi-rank path of bench.py on CPU: two gloo ranks aggregate their
timed regions into one whole-job throughput (max over ranks), solve
independent seeded systems, and the reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r pretends its timed region took (r + 1) * 100 ms for 4 solves
    value, total = bench.aggregate_throughput((rank + 1) * 100.0, 4, world, "cpu")
    seed = bench.rank_source_seed("wilson_16x16x16x32_exp0.4", rank)
    dist.destroy_process_group()
    q.put((rank, value, total, seed))


def test_two_gloo_ranks_aggregate_throughput():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    # max over ranks: 200 ms for 2 ranks x 4 solves = 40 solves/s, on every rank
    for rank, value, total, seed in out:
        assert total == 200.0
        assert abs(value - 40.0) < 1e-12
    assert out[0][3] != out[1][3]  # independent systems per rank


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
