"""The multi-GPU path of the bench is replicas only (samples are independent; no
data-path collective): each rank runs its own estimate with disjoint noise, the
step time is the slowest rank's, and the job's value is seconds per trace over
all replicas.  Its host logic runs here on CPU as two `gloo` ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as tmp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_local = 0.1 * (rank + 1)
    t = bench.max_over_ranks(t_local, "cpu")
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.replica_seed(0, rank))
    dist.barrier()
    out[rank] = (t, bench.job_value(t, world), tuple(seeds))
    dist.destroy_process_group()


def test_two_replicas_max_time_and_disjoint_seeds():
    world, port = 2, _free_port()
    mgr = tmp.get_context("spawn").Manager()
    out = mgr.dict()
    tmp.start_processes(_rank_main, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    assert sorted(out.keys()) == [0, 1]
    for r in range(world):
        t, value, seeds = out[r]
        assert t == pytest.approx(0.2)                 # the slowest replica's step time
        assert value == pytest.approx(0.1)             # seconds per trace over both replicas
        assert len(set(seeds)) == world                # disjoint noise streams
    # the seeds give different Philox noise (the sample streams do not overlap)
    from oracle.philox import rademacher
    a, b = rademacher(4096, out[0][2][0], 1, 0), rademacher(4096, out[0][2][1], 1, 0)
    assert np.mean(a == b) < 0.6


def test_single_process_is_the_identity():
    import bench
    assert bench.max_over_ranks(0.25, "cpu") == 0.25
    assert bench.job_value(0.25, 1) == 0.25


def test_reference_arm_other_ranks_exit_without_output(monkeypatch, capsys):
    """Under torchrun the reference (oracle) arm runs on rank 0 only."""
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(workload="laplace1024", warmup=3, steps=1, gpus=2, impl="reference")
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""
