"""Tuning thresholds: a live handle re-binned by bpmf_set_tuning runs the same chain
as a handle created with those thresholds; parity with the oracle holds with rows
split between both routes; the autotuner leaves the chain state where it found it and
applies a candidate from its grid."""
import numpy as np
import pytest

import workloads
from test_gpu_parity import assert_worst, step_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bp():
    import torch
    torch.cuda.set_device(0)
    import paper_1705_10633_gb300 as bp
    bp.lib()
    return bp


def _prob():
    return workloads.random_small(700, 120, 64, 40000, seed=71, n_test=100, long_rows=4,
                                  long_deg=110)


def test_parity_with_mixed_kernels(bp):
    # rows below 60 ratings on the CUDA-core kernel, the rest (movies average ~270
    # ratings, the few long users ~110) on the tensor-core route
    assert_worst(step_parity(bp, _prob(), sweeps=2, long_min_degree=60))


def test_set_tuning_equals_creating_with_it(bp):
    import torch
    prob = _prob()
    a = bp.create_from_problem(prob, stream=torch.cuda.Stream().cuda_stream)
    b = bp.create_from_problem(prob, long_min_degree=60, stream=torch.cuda.Stream().cuda_stream)
    try:
        bp.bpmf_set_tuning(a, 60)
        assert bp.bpmf_info(a, 0)["n_short"] == bp.bpmf_info(b, 0)["n_short"] > 0
        ra, rb = bp.bpmf_sweep(a, 3), bp.bpmf_sweep(b, 3)
        sa, sb = (bp.bpmf_get_state(x, prob.M, prob.N, prob.K) for x in (a, b))
        for x, y in zip(sa[:3], sb[:3]):
            np.testing.assert_array_equal(x, y)
        assert ra == rb
    finally:
        bp.bpmf_destroy(a)
        bp.bpmf_destroy(b)


def test_autotune_restores_state_and_applies_a_grid_pair(bp):
    import torch

    from paper_1705_10633_gb300.autotune import autotune
    prob = _prob()
    st = torch.cuda.Stream()
    h = bp.create_from_problem(prob, stream=st.cuda_stream)
    try:
        bp.bpmf_sweep(h, 2)
        before = bp.bpmf_get_state(h, prob.M, prob.N, prob.K)
        best, times = autotune(h, prob.M, prob.N, prob.K, st.cuda_stream, long_min=(1, 24, 60))
        assert best in times and len(times) == 3 and all(t > 0 for t in times.values())
        assert best[1:] == (0, 0)
        after = bp.bpmf_get_state(h, prob.M, prob.N, prob.K)
        for x, y in zip(before, after):
            np.testing.assert_array_equal(x, y)
        bp.bpmf_sweep(h, 1)
        assert bp.bpmf_status(h) == 0
    finally:
        bp.bpmf_destroy(h)


def test_autotune_split_degree_below_k64(bp):
    import torch

    from paper_1705_10633_gb300.autotune import autotune
    prob = workloads.random_small(500, 100, 24, 20000, seed=72, n_test=50, long_rows=3,
                                  long_deg=90)
    st = torch.cuda.Stream()
    h = bp.create_from_problem(prob, stream=st.cuda_stream)
    try:
        bp.bpmf_sweep(h, 1)
        before = bp.bpmf_get_state(h, prob.M, prob.N, prob.K)
        best, times = autotune(h, prob.M, prob.N, prob.K, st.cuda_stream, split=(32, 1 << 30),
                               rank_one=(-1, 3))
        sp = min(((0, 32, 0), (0, 1 << 30, 0)), key=times.get)[1]
        assert sorted(times) == sorted([(0, 32, 0), (0, 1 << 30, 0), (0, sp, -1),
                                        (0, sp, 3)]) and best in times
        after = bp.bpmf_get_state(h, prob.M, prob.N, prob.K)
        for x, y in zip(before, after):
            np.testing.assert_array_equal(x, y)
        assert (bp.bpmf_info(h, 1)["n_split"] > 0) == (best[1] == 32)
        bp.bpmf_sweep(h, 1)
        assert bp.bpmf_status(h) == 0
    finally:
        bp.bpmf_destroy(h)


def test_autotune_cache_hit_applies_the_stored_tuning(bp, tmp_path):
    import torch

    from paper_1705_10633_gb300.autotune import TuningCache, autotune
    prob = workloads.random_small(500, 100, 24, 20000, seed=73, n_test=50, long_rows=3,
                                  long_deg=90)
    degs = (np.diff(prob.csr_ptr), prob.col_degrees())
    cache = TuningCache(str(tmp_path / "tuning.json"))
    st = torch.cuda.Stream()
    a = bp.create_from_problem(prob, stream=st.cuda_stream)
    b = bp.create_from_problem(prob, stream=st.cuda_stream)
    try:
        best, times = autotune(a, prob.M, prob.N, prob.K, st.cuda_stream, split=(32, 1 << 30),
                               rank_one=(-1,), cache=cache, degrees=degs)
        assert times and best in times
        hit, times2 = autotune(b, prob.M, prob.N, prob.K, st.cuda_stream, cache=TuningCache(
            str(tmp_path / "tuning.json")), degrees=degs)
        assert times2 == {} and hit == best
        for side in (0, 1):
            ia, ib = bp.bpmf_info(a, side), bp.bpmf_info(b, side)
            assert (ia["n_split"], ia["n_segments"]) == (ib["n_split"], ib["n_segments"])
    finally:
        bp.bpmf_destroy(a)
        bp.bpmf_destroy(b)
