"""Sharded sweeps on CPU: the cost-balanced partition of the rows and the exchange of
updated rows between world-size-2 gloo ranks, with the FP64 oracle standing in for a
GPU chain.  Two ranks, each updating its own ranges and all-gathering the rest after
every half-sweep, end with the factors, hyper-parameters and RMSEs of one oracle chain
over all rows, bit for bit."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import workloads
from paper_1705_10633_gb300.shard import (COST_FIXED, COST_PER_RATING, MOVIE, USER,
                                          ShardedChain, cost_balanced_ranges)


def _problem():
    return workloads.random_small(240, 90, 6, 3000, seed=19, n_test=80, long_rows=3, long_deg=60)


class OracleBackend:
    """The FP64 oracle as a sharding backend (host tensors, for gloo)."""

    def __init__(self, prob):
        self.orc = oracle.Oracle(prob, nthreads=2)
        self.deg = {USER: prob.degrees(), MOVIE: prob.col_degrees()}
        self.n = {USER: prob.M, MOVIE: prob.N}
        self.shard = {USER: (0, prob.M), MOVIE: (0, prob.N)}
        self.rmse = None

    def rows(self, side):
        return self.n[side]

    def degrees(self, side):
        return self.deg[side]

    def set_shard(self, side, lo, hi):
        self.shard[side] = (lo, hi)

    def hyper(self, side):
        self.orc.hyper(side)

    def rows_phase(self, side):
        self.orc.rows_range(side, *self.shard[side])

    def predict(self):
        self.rmse = self.orc.predict()

    def advance(self):
        self.orc.set_counters(self.orc.sweep_index + 1, self.orc.n_avg)

    def get_rows(self, side, lo, hi):
        import torch
        return torch.from_numpy(np.ascontiguousarray(self.orc.get_factors(side)[lo:hi]))

    def put_rows(self, side, lo, hi, rows):
        X = self.orc.get_factors(side)
        X[lo:hi] = rows.numpy()
        self.orc.set_factors(side, X)


def test_ranges_tile_the_rows_and_balance_the_cost():
    rng = np.random.default_rng(3)
    deg = rng.lognormal(4.5, 1.2, 5000).astype(np.int64) + 1
    for world in (1, 2, 3, 8):
        ranges = cost_balanced_ranges(deg, world)
        assert len(ranges) == world and ranges[0][0] == 0 and ranges[-1][1] == len(deg)
        assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
        cost = COST_FIXED + COST_PER_RATING * deg
        per = [cost[lo:hi].sum() for lo, hi in ranges]
        # each range is within one row's cost of its share
        assert max(per) - cost.sum() / world <= cost.max() + 1e-9
    # more ranks than rows: the ranges still tile, some are empty
    ranges = cost_balanced_ranges(np.array([5, 1]), 4)
    assert ranges[0][0] == 0 and ranges[-1][1] == 2
    assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, sweeps, q):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = OracleBackend(_problem())
        chain = ShardedChain(b, rank, world)
        chain.sweep(sweeps)
        q.put((rank, chain.ranges, b.orc.get_factors(USER), b.orc.get_factors(MOVIE),
               b.orc.get_hyper(USER), b.orc.get_hyper(MOVIE), b.rmse))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_run_the_single_chain():
    sweeps = 3
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, sweeps, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=240) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    prob = _problem()
    ref = oracle.Oracle(prob, nthreads=2)
    rs, ra = ref.sweep(sweeps)
    for rank, ranges, U, V, hu, hv, rmse in res:
        # the ranks own disjoint ranges that tile each side
        for side, n in ((USER, prob.M), (MOVIE, prob.N)):
            assert ranges[side][0][0] == 0 and ranges[side][0][1] == ranges[side][1][0]
            assert ranges[side][1][1] == n
        np.testing.assert_array_equal(U, ref.get_factors(USER))
        np.testing.assert_array_equal(V, ref.get_factors(MOVIE))
        for got, want in zip(hu + hv, ref.get_hyper(USER) + ref.get_hyper(MOVIE)):
            np.testing.assert_array_equal(got, want)
        assert rmse == (rs, ra)
