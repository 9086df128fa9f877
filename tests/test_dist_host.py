"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): replicas report the slowest
rank's time and the whole-job value; only rank 0 prints the reference arm's line."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_local = 1.0 + rank  # rank 1 is the slow one
    t_max = bench.reduce_max_time(t_local, world, "cpu")
    value = bench.weak_scaling_value(1e9, 10, world, t_max)
    q.put((rank, t_max, value))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_max_over_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t_max, value in got:
        assert t_max == 2.0
        assert value == pytest.approx(2 * 1e9 * 10 / 2.0 / 1e9)


def test_reference_arm_only_rank0_prints(tmp_path):
    """Under torchrun, non-zero ranks of the reference arm exit 0 without work or output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1"], env=env, capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def _dying_worker(rank, world, port, q):
    import datetime
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        os._exit(0)  # the rank is lost between steps, with nothing in flight
    try:
        bench.reduce_max_time(1.0, world, "cpu")
        q.put((rank, "no error"))
    except Exception as e:  # gloo reports the lost peer instead of waiting forever
        q.put((rank, type(e).__name__))


def test_lost_rank_is_reported_not_hung():
    """A rank that exits between steps: the survivor's max-over-ranks reduction ends with an
    error within the process-group timeout instead of hanging."""
    import time
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dying_worker, args=(r, 2, port, q)) for r in range(2)]
    t0 = time.time()
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    rank, outcome = q.get(timeout=10)
    assert rank == 0 and outcome != "no error"
    assert time.time() - t0 < 100
