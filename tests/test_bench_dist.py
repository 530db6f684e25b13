"""The benchmark's multi-rank path on CPU: two gloo ranks, barrier,
max-over-ranks timing and the whole-job value; the reference arm exits on
ranks other than 0."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as td

    import bench
    r, ws = bench.init_dist("gloo")
    bench.barrier()
    t_local = 1.0 + 0.5 * rank          # rank 1 is the slower one
    t_max = bench.max_over_ranks(t_local)
    seeds = [bench.rank_seed(r, k, 1_000_000) for k in range(3)]
    q.put((r, ws, t_max, bench.step_value(1000, 10, ws, t_max), seeds))
    bench.barrier()
    td.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for r, ws, t_max, value, _ in out:
        assert ws == 2 and t_max == 1.5
        assert value == pytest.approx(1000 * 10 * 2 / 1.5)
    s0, s1 = out[0][4], out[1][4]
    assert not set(s0) & set(s1)          # replicas draw disjoint streams


def test_reference_arm_exits_on_other_ranks():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference"], env=env,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
