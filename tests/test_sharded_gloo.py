"""One estimate with its samples spread over ranks (paper_2108_11281_gb300/sharded.py):
the host logic of the multi-GPU path, run here on CPU as two `gloo` ranks with the
oracle's exact-solve samples standing in for the GPU's blocks.  Ranks draw disjoint
blocks of one sample stream and merge the gathered block statistics in block
order, so two ranks give bit for bit the estimate one rank gives over the same
sample indices."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as tmp

from oracle import estimator as E
from oracle.hierarchy import SetupParams, build_hierarchy
from oracle.operators import laplace2d
from paper_2108_11281_gb300 import sharded as S

N, SEED, EPS, WIDTHS = 32, 2, 1e-2, [8, 8]


def levels():
    return build_hierarchy(laplace2d(N, N), N, N, 1, SetupParams(levels=3, n_tv=4, sweeps=20, coarse_sweeps=10))


class OracleSampler:
    """Blocks of exact-solve samples (oracle) with their (N, mean, M2).  The samples are
    computed once (NS per level) and handed to every rank, so that all ranks and runs see
    the same floating-point values whatever the BLAS threading of each process."""
    NS = 256

    def __init__(self, table):
        self.table = table
        self.n_differences = len(table["samples"])

    @staticmethod
    def make_table():
        lv = levels()
        sv = E.LevelSolvers(lv)
        return {"samples": [E.level_samples(lv, sv, l, "rademacher", SEED, 0, OracleSampler.NS)
                            for l in range(1, len(lv))],
                "costs": [E.nominal_sample_cost(lv, l) for l in range(1, len(lv))],
                "term": float(np.real(E.exact_coarse_trace(lv)))}

    def width(self, l):
        return WIDTHS[l - 1]

    def cost(self, l):
        return self.table["costs"][l - 1]

    def coarse_term(self):
        return self.table["term"]

    def block(self, l, first, k):
        assert first + k <= self.NS
        s = self.table["samples"][l - 1][first:first + k]
        m = s.mean()
        return s, (k, complex(m), float(np.sum(np.abs(s - m) ** 2)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, table, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r = S.sharded_trace_estimate(OracleSampler(table), S.torch_allgather("cpu"), rank, world, eps=EPS)
    dist.barrier()
    out[rank] = r
    dist.destroy_process_group()


@pytest.fixture(scope="module")
def table():
    return OracleSampler.make_table()


def single(table, allocation="optimal", n_fixed=None):
    return S.sharded_trace_estimate(OracleSampler(table), lambda v: [v], 0, 1, eps=EPS, allocation=allocation,
                                    n_fixed=n_fixed)


def test_merge_is_the_two_pass_statistics():
    """Merging block statistics in order gives the mean and the sum of squared deviations
    of all samples (computed here directly in two passes)."""
    rng = np.random.default_rng(0)
    x = rng.normal(size=50) + 1j * rng.normal(size=50)
    acc = (0, 0j, 0.0)
    for a, b in ((0, 7), (7, 20), (20, 21), (21, 50)):
        blk = x[a:b]
        m = blk.mean()
        acc = S.merge(acc, (b - a, m, float(np.sum(np.abs(blk - m) ** 2))))
    assert acc[0] == 50
    assert abs(acc[1] - x.mean()) <= 1e-14
    assert abs(acc[2] - np.sum(np.abs(x - x.mean()) ** 2)) <= 1e-12 * acc[2]


def test_one_rank_follows_the_oracle_allocation_loop(table):
    """One rank: the same N_l, tau and trace as the oracle's Sec. 2 loop on the same samples."""
    r = single(table)
    ref = E.optimal_trace_estimate(levels(), "rademacher", seed=SEED, eps=EPS, widths=WIDTHS)
    assert r["n_samples"] == ref.n_samples
    assert abs(r["tau"] - ref.tau) <= 1e-12 * abs(ref.tau)
    assert abs(r["trace"] - ref.trace) <= 1e-12 * abs(ref.trace)


def test_two_ranks_equal_one_rank_over_the_same_samples(table):
    world, port = 2, _free_port()
    mgr = tmp.get_context("spawn").Manager()
    out = mgr.dict()
    tmp.start_processes(_rank_main, args=(world, port, table, out), nprocs=world, start_method="spawn", join=True)
    r0, r1 = out[0], out[1]
    assert r0 == r1                                          # every rank holds the same estimate
    assert all(n % (2 * w) == 0 for n, w in zip(r0["n_samples"], WIDTHS))   # whole rounds of two blocks
    one = single(table, "fixed", r0["n_samples"])            # one rank, the same sample indices
    for key in ("trace", "tau", "std_err", "coarse_term", "n_samples", "mean", "variance"):
        assert one[key] == r0[key], key
