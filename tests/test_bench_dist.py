"""The multi-rank plumbing of bench.py on CPU: two gloo ranks (world_size 2) run the same
setup, barrier and max-reduce of the timed region that the NCCL ranks run on the GPUs, and
each replica renders its own frames (no frame is shared, no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_setup(world, backend="gloo")
    bench.barrier(w)
    # the slowest rank's time is the job's time
    t = bench.reduce_max(1.5 + rank, w)
    q.put((r, w, local, t, bench.frame_seeds(r)))
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1] and all(g[1] == world for g in got)
    assert all(g[3] == 2.5 for g in got)  # max over ranks of 1.5 and 2.5
    seeds0, seeds1 = got[0][4], got[1][4]
    assert len(seeds0) == len(seeds1) == 4 and not set(seeds0) & set(seeds1)


def test_world_size_must_match_gpus(monkeypatch):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    with pytest.raises(SystemExit):
        bench.dist_setup(1)
