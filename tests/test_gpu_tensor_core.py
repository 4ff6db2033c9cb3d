"""GPU parity of the tensor-core row kernel (K padded to 64, rows of the long bin).

The Gram of long rows runs on tcgen05 with an FP16 hi/lo split of the gathered
factors; the per-row tolerance stays the FP32 path's 1e-4 (norm-wise, against
the FP64 oracle from the same state).  Also: the full-size 480k x 18k workload
with 1e8 ratings in the launch configuration bench.py times, checked on
sampled rows, and the bounded-wait timeout path.
"""
import numpy as np
import pytest

import oracle
import workloads
from test_gpu_parity import ROW_TOL, assert_worst, full_size_sampled_rows, rowwise_rel, step_parity

pytestmark = pytest.mark.gpu

# CTAs per SM of the tensor-core Gram launch (its grid, and so the grids its balanced
# plans are made for)
GRAM_CTAS_PER_SM = 2


@pytest.fixture(scope="module")
def bp():
    import torch
    torch.cuda.set_device(0)
    import paper_1705_10633_gb300 as bp
    bp.lib()
    return bp


@pytest.mark.parametrize("K,long_min", [(64, 0), (50, 0), (64, 150)])
def test_long_rows_tensor_core_parity(bp, K, long_min):
    # degrees 60..400 on both sides: ragged against the 16-rating MMA step and the
    # 64-rating stage; with a threshold of 150 the rows below it stay on the warp
    # kernel (both kernels in one phase)
    prob = workloads.random_small(600, 300, K, 60000, seed=200 + K, n_test=400, long_rows=6,
                                  long_deg=290)
    for side in (0, 1):
        deg = np.diff(prob.csr_ptr) if side == 0 else prob.col_degrees()
        assert (deg >= 48).sum() > 0.5 * len(deg)
        if long_min:
            assert (deg < long_min).sum() > 0
    assert_worst(step_parity(bp, prob, sweeps=2, long_min_degree=long_min))


def test_long_rows_in_several_chunks_parity(bp):
    # 40 movies with ~3,000 ratings each: rows span 1-3 accumulation chunks of 1024
    # ratings, so the drain sums a row's Gram over several TMEM accumulators
    prob = workloads.random_small(8000, 40, 64, 150000, seed=31, n_test=300)
    deg = prob.col_degrees()
    assert deg.mean() >= 1024 and deg.max() > 2048
    assert_worst(step_parity(bp, prob, sweeps=2))


def test_balanced_row_plan_parity_and_identity(bp):
    """Tensor-core rows dealt to the CTAs of the Gram launch by the balanced plan (each row,
    longest first, to the CTA with the least work so far).  2,000 users with ~60 ratings and
    160 with ~1,060: round-robin would give a few CTAs two of the long rows, so the user
    side gets a plan for both launch grids; the movie side gets one exactly where
    bpmf_balance_rows finds round-robin uneven for that grid.  Parity with the oracle, and
    bpmf_sweep (one SM left to the hyper steps) bit-identical to phase-by-phase stepping
    (every SM): a row's result does not depend on which CTA takes it."""
    import torch
    prob = workloads.random_small(2000, 1200, 64, 120000, seed=77, n_test=300, long_rows=160,
                                  long_deg=1000)
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    a = bp.create_from_problem(prob, stream=sa.cuda_stream)
    b = bp.create_from_problem(prob, stream=sb.cuda_stream)
    try:
        nsm = torch.cuda.get_device_properties(0).multi_processor_count
        assert bp.bpmf_info(a, 0)["balanced"] == 3
        assert bp.bpmf_info(a, 0)["n_long"] > GRAM_CTAS_PER_SM * nsm
        # the movie side's long bin, longest first, against the two grids of a Gram launch
        vdeg = np.sort(prob.col_degrees())[::-1]
        vdeg = vdeg[:bp.bpmf_info(a, 1)["n_long"]].astype(np.int64)
        want = sum(bit for bit, g in ((1, GRAM_CTAS_PER_SM * nsm), (2, GRAM_CTAS_PER_SM * (nsm - 1)))
                   if bp.bpmf_balance_rows(vdeg, g) is not None)
        assert bp.bpmf_info(a, 1)["balanced"] == want
        ra = bp.bpmf_sweep(a, 2)
        seq = (bp.BPMF_PHASE_HYPER_MOVIE, bp.BPMF_PHASE_ROWS_MOVIE, bp.BPMF_PHASE_HYPER_USER,
               bp.BPMF_PHASE_ROWS_USER, bp.BPMF_PHASE_PREDICT, bp.BPMF_PHASE_ADVANCE)
        for _ in range(2):
            for ph in seq:
                bp.bpmf_step(b, ph)
        rb = bp.bpmf_sweep(b, 0)
        st_a = bp.bpmf_get_state(a, prob.M, prob.N, prob.K)
        st_b = bp.bpmf_get_state(b, prob.M, prob.N, prob.K)
        for x, y in zip(st_a[:3], st_b[:3]):
            np.testing.assert_array_equal(x, y)
        assert ra == rb
        assert bp.bpmf_status(a) == 0 and bp.bpmf_status(b) == 0
    finally:
        bp.bpmf_destroy(a)
        bp.bpmf_destroy(b)
    assert_worst(step_parity(bp, prob, sweeps=1))


# BF16 Gram: per-row means and samples within 1e-2 relative of the FP64 oracle (the
# rows enter the MMA rounded to 8 significant bits, 2^-9 relative per entry; the
# measured worst is printed).
BF16_ROW_TOL = 1e-2


def test_bf16_gram_parity(bp):
    prob = workloads.random_small(600, 300, 64, 60000, seed=264, n_test=400, long_rows=6,
                                  long_deg=290)
    w = step_parity(bp, prob, flags=bp.BPMF_BF16_GRAM, sweeps=2)
    print("bf16 worst:", {k: "%.2e" % v for k, v in w.items()})
    assert w["stats"] <= 1e-5 and w["hyper"] <= 1e-9 and w["rmse"] <= 1e-5, w
    assert w["x"] <= BF16_ROW_TOL and w["mean"] <= BF16_ROW_TOL, w
    assert w["x"] > 1e-5  # the BF16 path really ran (FP32-class errors would be ~1e-6)


def test_bf16_gram_rejected_without_tensor_cores(bp):
    prob = workloads.random_small(100, 60, 32, 2000, seed=3)
    with pytest.raises(bp.BpmfError) as ei:
        bp.create_from_problem(prob, flags=bp.BPMF_BF16_GRAM)
    assert ei.value.code == bp.BPMF_EINVAL


def test_tensor_core_and_cuda_core_paths_agree(bp):
    prob = workloads.random_small(500, 260, 64, 30000, seed=77, n_test=100)
    K = prob.K
    out = []
    for flags in (0, bp.BPMF_CUDA_CORE_GRAM):
        h = bp.create_from_problem(prob, flags=flags, stream=bp.torch_stream())
        try:
            assert (bp.bpmf_info(h, 1)["n_long"] > 0) or flags
            bp.bpmf_sweep(h, 2)
            out.append(bp.bpmf_get_state(h, prob.M, prob.N, K))
        finally:
            bp.bpmf_destroy(h)
    for side in (0, 1):
        assert rowwise_rel(out[0][side], out[1][side]).max() <= 3 * ROW_TOL


def test_wait_timeout_reports_status_and_context_survives(bp):
    prob = workloads.random_small(300, 200, 64, 20000, seed=5)
    p = bp.bpmf_default_params(alpha=prob.alpha, seed=prob.seed, flags=bp.BPMF_TEST_STALL,
                               wait_timeout_ms=100)
    h = bp.create_from_problem(prob, params=p, stream=bp.torch_stream())
    try:
        assert bp.bpmf_info(h, 1)["n_long"] > 0
        with pytest.raises(bp.BpmfError) as ei:
            bp.bpmf_sweep(h, 1)
        assert ei.value.code == bp.BPMF_ETIMEOUT
        assert bp.bpmf_status(h) == bp.BPMF_ETIMEOUT
    finally:
        bp.bpmf_destroy(h)
    h = bp.create_from_problem(prob, stream=bp.torch_stream())
    try:
        bp.bpmf_sweep(h, 1)
        assert bp.bpmf_status(h) == 0
    finally:
        bp.bpmf_destroy(h)


def test_full_size_config3_sampled_rows(bp, config3_problem):
    """One sweep of the 480,000 x 18,000, 1e8-rating, K = 64 workload (the bench
    configuration), each half-sweep checked on sampled rows against the oracle."""
    full_size_sampled_rows(bp, config3_problem)


def test_full_size_config3_sampled_rows_bf16(bp, config3_problem):
    """The same on the BF16 Gram, where rows of up to 2.7e5 ratings put the most BF16
    rounding into one precision matrix: sampled rows (the 8 longest among them) within
    the BF16 path's 1e-2 per row of the FP64 oracle."""
    full_size_sampled_rows(bp, config3_problem, flags=bp.BPMF_BF16_GRAM, tol=BF16_ROW_TOL)


def test_row_launch_timing(bp):
    # users below the tensor-core threshold on the CUDA-core kernel, the rest on the
    # tensor-core route (Gram kernel, then factorisation kernel): every part timed by
    # the library's events when on, -1 when off
    prob = workloads.random_small(400, 200, 64, 20000, seed=61)
    deg = np.diff(prob.csr_ptr)
    assert (deg < 48).sum() > 0 and (deg >= 48).sum() > 0
    h = bp.create_from_problem(prob, stream=bp.torch_stream(), long_min_degree=48)
    try:
        assert bp.bpmf_row_launch_ms(h) == (-1.0, -1.0, -1.0)
        bp.bpmf_set_row_timing(h, True)
        bp.bpmf_step(h, bp.BPMF_PHASE_ROWS_USER)
        cc, gram, chol = bp.bpmf_row_launch_ms(h)
        assert cc > 0 and gram > 0 and chol > 0
        bp.bpmf_sweep(h, 2)  # sweeps record nothing: the last timed phase stays
        assert bp.bpmf_row_launch_ms(h) == (cc, gram, chol)
        bp.bpmf_set_row_timing(h, False)
        assert bp.bpmf_row_launch_ms(h) == (-1.0, -1.0, -1.0)
        assert bp.bpmf_status(h) == 0
    finally:
        bp.bpmf_destroy(h)


def test_non_finite_factor_row_sets_not_pd_on_tensor_route(bp):
    """A non-finite row of the other side reaches the tensor-core route's Gram; the
    factorisation kernel then sees a pivot that is not positive and finite and raises
    the not-positive-definite status, without a fault; the context stays usable."""
    prob = workloads.random_small(300, 200, 64, 20000, seed=9)
    h = bp.create_from_problem(prob, stream=bp.torch_stream())
    try:
        assert bp.bpmf_info(h, 0)["n_long"] > 0
        U, V, hyper, s = bp.bpmf_get_state(h, prob.M, prob.N, prob.K)
        V[3, :] = np.inf
        bp.bpmf_set_state(h, U, V, hyper, s)
        bp.bpmf_step(h, bp.BPMF_PHASE_ROWS_USER)
        assert bp.bpmf_status(h) == bp.BPMF_ENOTPD
        h2 = bp.create_from_problem(prob, stream=bp.torch_stream())
        bp.bpmf_sweep(h2, 1)
        assert bp.bpmf_status(h2) == 0
        bp.bpmf_destroy(h2)
    finally:
        bp.bpmf_destroy(h)
