"""Host-side logic of bench.py on CPU: world-size-2 gloo ranks agree on the
max-over-ranks time and the whole-job aggregate (each rank runs its own chain)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    r, w, local = bench.dist_env()
    bench.dist_init(w, "gloo")
    bench.barrier(w)
    my_ms = 100.0 + 50.0 * r
    mx = bench.reduce_over_ranks(my_ms, w, "max")
    tot = bench.reduce_over_ranks(1.0, w, "sum")
    value = bench.aggregate_rows_per_s(1000 * w, 10, mx)
    q.put((r, local, mx, tot, value))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_agree():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    for r, local, mx, tot, value in res:
        assert local == r
        assert mx == 150.0 and tot == 2.0
        assert value == pytest.approx(2000 * 10 / 0.150)


def test_single_rank_is_identity():
    assert bench.reduce_over_ranks(3.5, 1) == 3.5
    assert bench.aggregate_rows_per_s(500, 4, 2000.0) == 1000.0


def test_row_phase_work_figures():
    K = 64
    # per rating K(K+1) + 2K flops, per row K^3/3 + 6K^2
    assert bench.row_phase_flops(1, 0, K) == K * (K + 1) + 2 * K
    assert bench.row_phase_flops(0, 1, K) == pytest.approx(K**3 / 3 + 6 * K * K)
    assert bench.row_phase_bytes(1, 1, K) == (8 + 4 * K) + (8 + 4 * K)
