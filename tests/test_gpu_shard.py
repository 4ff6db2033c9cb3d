"""Sharded sweeps of the GPU library: two processes, each with its own handle on the one
visible GPU, each updating a cost-balanced range of the rows of both sides and
exchanging the updated rows through gloo on host copies after every half-sweep
(bpmf_set_shard, bpmf_get_rows, bpmf_put_rows).  Their kernels never wait on each
other (the exchange is on the host).  After three sweeps both ranks hold the state of
one handle that ran the same three sweeps over all rows, bit for bit: factors,
hyper-parameters, sweep counter and RMSEs."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import workloads

pytestmark = pytest.mark.gpu


def _problem(K):
    # at K = 64 rows go to both the CUDA-core kernel and the tensor-core route; at K = 24
    # the long movie columns are split into segments on the CUDA-core kernel
    if K == 64:
        return workloads.random_small(1500, 400, 64, 60000, seed=83, n_test=200, long_rows=6,
                                      long_deg=300)
    return workloads.random_small(1200, 150, 24, 30000, seed=84, n_test=150, long_rows=4,
                                  long_deg=200)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, K, sweeps, q):
    import torch
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        import paper_1705_10633_gb300 as bp
        from paper_1705_10633_gb300.shard import HandleBackend, ShardedChain
        prob = _problem(K)
        kw = {"split_degree": 64} if K != 64 else {"long_min_degree": 48}
        h = bp.create_from_problem(prob, stream=bp.torch_stream(), **kw)
        try:
            b = HandleBackend(bp, h, prob.M, prob.N, prob.K, prob.degrees(), prob.col_degrees(),
                              device=False)
            chain = ShardedChain(b, rank, world)
            chain.sweep(sweeps)
            U, V, hyper, s = bp.bpmf_get_state(h, prob.M, prob.N, prob.K)
            rmse = bp.bpmf_sweep(h, 0)
            status = bp.bpmf_status(h)
            own = [bp.bpmf_info(h, side)["n_short"] + bp.bpmf_info(h, side)["n_long"]
                   for side in (0, 1)]
        finally:
            bp.bpmf_destroy(h)
        q.put((rank, U, V, hyper, s, rmse, status, own, chain.ranges))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("K", [64, 24])
def test_two_sharded_ranks_equal_one_handle(K):
    import torch
    import paper_1705_10633_gb300 as bp
    sweeps = 3
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, K, sweeps, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=600) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    torch.cuda.set_device(0)
    prob = _problem(K)
    kw = {"split_degree": 64} if K != 64 else {"long_min_degree": 48}
    h = bp.create_from_problem(prob, stream=bp.torch_stream(), **kw)
    try:
        rmse = bp.bpmf_sweep(h, sweeps)
        U, V, hyper, s = bp.bpmf_get_state(h, prob.M, prob.N, prob.K)
        if K == 64:
            assert bp.bpmf_info(h, 0)["n_long"] > 0 and bp.bpmf_info(h, 0)["n_short"] > 0
        else:
            assert bp.bpmf_info(h, 1)["n_split"] > 0
    finally:
        bp.bpmf_destroy(h)
    for rank, Ug, Vg, hg, sg, rg, status, own, ranges in res:
        assert status == 0 and sg == s == sweeps
        # each rank updated only its own rows
        for side in (0, 1):
            lo, hi = ranges[side][rank]
            assert own[side] == hi - lo and 0 < hi - lo < (prob.M if side == 0 else prob.N)
        np.testing.assert_array_equal(Ug, U)
        np.testing.assert_array_equal(Vg, V)
        np.testing.assert_array_equal(hg, hyper)
        assert rg == rmse
