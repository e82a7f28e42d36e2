"""The multi-GPU form is replicas only: each rank solves its own instance, and
the only collectives are the benchmark's max-over-ranks elapsed time and sum of
processed iterations.  Exercised with two gloo ranks on the CPU."""

import multiprocessing as mp
import os
import socket
import types

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, u = bench.aggregate(dist, world, 10.0 + rank, 5.0 * (rank + 1), "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, u, bench.rank_seed(0, rank)))


def test_two_ranks_aggregate_and_independent_instances():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [11.0, 11.0]  # the slowest rank's time
    assert [o[2] for o in out] == [15.0, 15.0]  # every rank's units
    assert out[0][3] != out[1][3]  # each rank draws its own instance


def test_single_rank_aggregate_is_identity():
    import bench
    assert bench.aggregate(None, 1, 3.5, 7, "cpu") == (3.5, 7.0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import bench
    a = types.SimpleNamespace(n=10, r=2, alpha=0.1, seed=0, variant="R", steps=1, warmup=0, gpus=2)
    bench.run_reference(a, rank=1, world=2)  # returns before any work
    assert capsys.readouterr().out == ""
