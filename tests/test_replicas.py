"""The multi-GPU form of the benchmark is independent replicas (one process per
GPU, no data-path collective): its host logic - the rank environment and the
max-over-ranks job time - run here as two gloo processes on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    ms_max, value = bench.replica_throughput(10.0 * (rank + 1), steps=5, world=w, device="cpu")
    out.put((r, w, local, ms_max, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [(r, w, loc) for r, w, loc, _, _ in results] == [(0, 2, 0), (1, 2, 1)]
    for _, _, _, ms_max, value in results:
        assert ms_max == 20.0                       # the slower rank's time
        assert abs(value - 2 * 5 / 0.020) < 1e-9     # both ranks' applies over that time


def test_single_process_defaults():
    torch = pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    env = {k: os.environ.pop(k) for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK") if k in os.environ}
    try:
        assert bench.dist_env() == (0, 1, 0)
        ms, v = bench.replica_throughput(4.0, steps=2, world=1, device="cpu")
        assert ms == 4.0 and abs(v - 500.0) < 1e-9
    finally:
        os.environ.update(env)
