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


def _textbook_counts(K):
    """Multiply-adds of a loop-by-loop Cholesky and of two triangular solves."""
    chol = sum(j for j in range(K) for _ in range(j, K))  # row i >= j: j products
    solves = 2 * sum(range(K))
    return chol, solves


def test_row_work_figures_match_loop_counts():
    for K in (4, 16, 64):
        chol, solves = _textbook_counts(K)
        flops = 2 * (chol + solves)
        # the closed form drops O(K) terms only
        assert abs(bench.row_alu_flops(1, K) - flops) <= 4 * K
        assert bench.row_alu_flops(3, K) == pytest.approx(3 * bench.row_alu_flops(1, K))
    K = 64
    # one rating adds one outer product (K x K multiply-adds) and one scaled row (K)
    assert bench.row_gram_flops(1, K) == 2 * (K * K + K)
    # the symmetric count: the lower half of the outer product (K(K+1)/2 multiply-adds)
    assert bench.row_sym_gram_flops(1, K) == 2 * (K * (K + 1) / 2 + K)
    # the gathered 16-bit rows: FP16 hi and lo (2 B each per entry), or BF16 alone
    assert bench.gathered_bytes(1, K) == 2 * 2 * K
    assert bench.gathered_bytes(1, K, bf16=True) == 2 * K


def test_l2_note_states_how_inputs_stand_to_l2():
    # the ratings are held twice (row and column views), 8 B per rating each
    assert bench.l2_note(98_959_257).startswith("inputs larger than L2 (ratings CSR+CSC 1.58 GB)")
    assert bench.l2_note(20_000).startswith("inputs fit in L2")


def test_stratified_relabel_keeps_the_ratings_and_levels_the_blocks():
    """The oracle sampler's renumbering: the same (user, movie, rating) triples under a
    permutation of each side, columns ascending in every row, and blocks of 1/stride of
    a side with nearly equal rating counts (Zipf-like columns otherwise vary widely)."""
    import numpy as np
    import bench
    import workloads
    p = workloads.random_small(3000, 800, 16, 60000, seed=3, n_test=100, long_rows=5, long_deg=500)
    q = bench.stratified_relabel(p, 10)
    deg_u, deg_v = np.diff(p.csr_ptr), np.bincount(p.csr_col, minlength=p.N)
    rows_p = np.repeat(np.arange(p.M), deg_u)
    rows_q = np.repeat(np.arange(q.M), np.diff(q.csr_ptr))
    # recover the permutations from the degrees' new positions and compare triples
    trip_p = sorted(zip(deg_u[rows_p], deg_v[p.csr_col], p.csr_val.tolist()))
    dq_u, dq_v = np.diff(q.csr_ptr), np.bincount(q.csr_col, minlength=q.N)
    trip_q = sorted(zip(dq_u[rows_q], dq_v[q.csr_col], q.csr_val.tolist()))
    assert trip_p == trip_q and q.nnz == p.nnz
    for i in range(q.M):
        assert np.all(np.diff(q.csr_col[q.csr_ptr[i]:q.csr_ptr[i + 1]]) > 0)
    # round-robin by degree rank: blocks differ by at most one row's ratings
    blocks = [dq_v[b * 80:(b + 1) * 80].sum() for b in range(10)]
    assert max(blocks) - min(blocks) <= dq_v.max()
    ublocks = [dq_u[b * 300:(b + 1) * 300].sum() for b in range(10)]
    assert max(ublocks) - min(ublocks) <= dq_u.max()
    assert np.all((q.test_i >= 0) & (q.test_i < q.M)) and np.all((q.test_j >= 0) & (q.test_j < q.N))
