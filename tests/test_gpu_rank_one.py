"""The rank-one route for short rows on the CUDA-core kernel (Sec. 3.1: for items with
few ratings, update the Cholesky factor of the prior precision once per rating instead
of forming and factoring the Gram matrix).  The factor it reaches equals chol(Lambda_i)
up to rounding, so the same oracle applies: parity for every padded K with every row on
the route, with the route mixed with the Gram route and with empty rows; agreement with
the Gram route; bit-identical resume through bpmf_set_state (the stored prior's factor
is recomputed by the same FP64 routine); and bpmf_set_tuning moving rows between routes
(one more launch per half-sweep when the route has rows)."""
import numpy as np
import pytest

import workloads
from test_gpu_parity import ROW_TOL, assert_worst, rowwise_rel, step_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bp():
    import torch
    torch.cuda.set_device(0)
    import paper_1705_10633_gb300 as bp
    bp.lib()
    return bp


def _short(K, seed=41):
    # 600 x 300 with ~1,500 ratings: most rows have 1 to 4 ratings, some none
    return workloads.random_small(600, 300, K, 1500, seed=seed, n_test=100, empty_rows=20,
                                  empty_cols=10)


@pytest.mark.parametrize("K,r1", [(10, 1 << 20), (32, 1 << 20), (48, 1 << 20), (17, 3), (32, 2),
                                  (10, 1)])
def test_rank_one_parity(bp, K, r1):
    prob = _short(K)
    deg = np.diff(prob.csr_ptr)
    assert (deg == 0).sum() >= 20 and ((deg > 0) & (deg < 3)).sum() > 0
    assert_worst(step_parity(bp, prob, sweeps=2, rank_one_degree=r1))


def test_rank_one_with_long_rows_and_k64_cuda_core(bp):
    # every row with fewer than 40 ratings on the route, longer rows on the Gram route
    prob = workloads.random_small(300, 150, 64, 6000, seed=43, n_test=80, empty_rows=5,
                                  long_rows=4, long_deg=120)
    assert_worst(step_parity(bp, prob, flags=bp.BPMF_CUDA_CORE_GRAM, sweeps=2,
                             rank_one_degree=40))


def test_rank_one_agrees_with_gram_route(bp):
    import torch
    prob = _short(32, seed=44)
    out = []
    for r1 in (1 << 20, -1):
        h = bp.create_from_problem(prob, rank_one_degree=r1, flags=bp.BPMF_DEBUG_MEANS,
                                   stream=torch.cuda.Stream().cuda_stream)
        try:
            bp.bpmf_sweep(h, 1)
            out.append([bp.bpmf_debug_means(h, s, n, prob.K) for s, n in ((0, prob.M), (1, prob.N))])
        finally:
            bp.bpmf_destroy(h)
    for side in (0, 1):
        assert rowwise_rel(out[0][side], out[1][side]).max() <= 3 * ROW_TOL


def test_rank_one_resume_is_bit_identical(bp):
    import torch
    prob = _short(16, seed=45)
    mk = lambda: bp.create_from_problem(prob, burn_in=1, rank_one_degree=5,
                                        stream=torch.cuda.Stream().cuda_stream)
    a, b, c = mk(), mk(), mk()
    try:
        ra = bp.bpmf_sweep(a, 5)
        bp.bpmf_sweep(b, 2)
        bp.bpmf_sweep(c, 4)
        U, V, hyper, sweep = bp.bpmf_get_state(b, prob.M, prob.N, prob.K)
        ps, navg = bp.bpmf_get_accum(b, prob.T)
        bp.bpmf_set_state(c, U, V, hyper, sweep)
        bp.bpmf_set_accum(c, ps, navg)
        rc = bp.bpmf_sweep(c, 3)
        sa = bp.bpmf_get_state(a, prob.M, prob.N, prob.K)
        sc = bp.bpmf_get_state(c, prob.M, prob.N, prob.K)
        for x, y in zip(sa[:3], sc[:3]):
            np.testing.assert_array_equal(x, y)
        assert ra == rc
    finally:
        for h in (a, b, c):
            bp.bpmf_destroy(h)


def test_set_tuning_moves_rows_between_routes(bp):
    import torch
    prob = _short(24, seed=46)
    a = bp.create_from_problem(prob, rank_one_degree=-1, stream=torch.cuda.Stream().cuda_stream)
    b = bp.create_from_problem(prob, rank_one_degree=4, stream=torch.cuda.Stream().cuda_stream)
    try:
        n0 = bp.bpmf_launch_count(a)
        bp.bpmf_step(a, bp.BPMF_PHASE_ROWS_USER)
        one = bp.bpmf_launch_count(a) - n0
        bp.bpmf_set_tuning(a, 0, 0, 4)
        n0 = bp.bpmf_launch_count(a)
        bp.bpmf_step(a, bp.BPMF_PHASE_ROWS_USER)
        assert bp.bpmf_launch_count(a) - n0 == one + 1
        # a has now run one extra user half-sweep; compare from equal states
        U, V, hyper, sweep = bp.bpmf_get_state(b, prob.M, prob.N, prob.K)
        bp.bpmf_set_state(a, U, V, hyper, sweep)
        ra, rb = bp.bpmf_sweep(a, 3), bp.bpmf_sweep(b, 3)
        sa, sb = (bp.bpmf_get_state(x, prob.M, prob.N, prob.K) for x in (a, b))
        for x, y in zip(sa[:3], sb[:3]):
            np.testing.assert_array_equal(x, y)
    finally:
        bp.bpmf_destroy(a)
        bp.bpmf_destroy(b)
