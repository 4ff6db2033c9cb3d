"""Long rows split into segments on the CUDA-core kernel (Sec. 3.2: an item with many
ratings is cut into smaller tasks done in parallel).  Each segment's warp writes the
partial Gram rows and right-hand side of its ratings; the last warp of a row sums
them in segment order and samples the row.  Checked here: parity with the oracle
for every padded K, segment lengths down to one rating, the split inside the
tensor-core path's short bin, the number of rows and segments, bit-identical chains
across runs (the sum order does not depend on which warp finishes last) and across
bpmf_set_tuning versus creation, and agreement with the unsplit kernel."""
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


def _prob(K, seed=31):
    # 400 x 150 with ~12,000 ratings: rows ~30 ratings, columns ~80, six users with
    # 140 ratings each
    return workloads.random_small(400, 150, K, 12000, seed=seed, n_test=80, long_rows=6,
                                  long_deg=140)


def _expected_split(deg, split, lo=0, hi=None):
    """Rows with at least `split` ratings (within [lo, hi) of the kernel's bin) and their
    segments: ceil(d / (split // 2)) each."""
    sel = deg[(deg >= max(split, 2)) & (deg >= lo) & ((deg < hi) if hi else True)]
    seg = max(split // 2, 1)
    return len(sel), int(((sel + seg - 1) // seg).sum())


@pytest.mark.parametrize("K,split", [(10, 64), (32, 64), (48, 80), (32, 2), (17, 3)])
def test_split_rows_parity(bp, K, split):
    prob = _prob(K)
    flags = 0
    h = bp.create_from_problem(prob, split_degree=split, stream=bp.torch_stream())
    try:
        for side, deg in ((0, np.diff(prob.csr_ptr)), (1, prob.col_degrees())):
            info = bp.bpmf_info(h, side)
            assert (info["n_split"], info["n_segments"]) == _expected_split(deg, split)
            assert info["n_split"] > 0
    finally:
        bp.bpmf_destroy(h)
    assert_worst(step_parity(bp, prob, flags=flags, sweeps=2, split_degree=split))


def test_split_rows_cuda_core_gram_at_k64(bp):
    prob = _prob(64)
    assert_worst(step_parity(bp, prob, flags=bp.BPMF_CUDA_CORE_GRAM, sweeps=2, split_degree=50))


def test_split_inside_the_tensor_core_short_bin(bp):
    # rows below 120 ratings on the CUDA-core kernel, those from 40 up split; the rest
    # on the tensor-core kernel
    prob = _prob(64)
    h = bp.create_from_problem(prob, long_min_degree=120, split_degree=40, stream=bp.torch_stream())
    try:
        for side, deg in ((0, np.diff(prob.csr_ptr)), (1, prob.col_degrees())):
            info = bp.bpmf_info(h, side)
            assert (info["n_split"], info["n_segments"]) == _expected_split(deg, 40, hi=120)
            assert info["n_long"] == int((deg >= 120).sum())
    finally:
        bp.bpmf_destroy(h)
    assert_worst(step_parity(bp, prob, sweeps=2, long_min_degree=120, split_degree=40))


@pytest.mark.parametrize("K", [16, 40])
def test_split_chain_is_reproducible_and_set_tuning_equals_create(bp, K):
    import torch
    prob = _prob(K, seed=32)
    hs = [bp.create_from_problem(prob, split_degree=8, stream=torch.cuda.Stream().cuda_stream),
          bp.create_from_problem(prob, split_degree=8, stream=torch.cuda.Stream().cuda_stream),
          bp.create_from_problem(prob, stream=torch.cuda.Stream().cuda_stream)]
    try:
        bp.bpmf_set_tuning(hs[2], 0, 8)  # grows the segment arrays from none
        assert bp.bpmf_info(hs[2], 1)["n_segments"] == bp.bpmf_info(hs[0], 1)["n_segments"] > 0
        runs = [(bp.bpmf_sweep(h, 4), bp.bpmf_get_state(h, prob.M, prob.N, K)) for h in hs]
        for r, st in runs[1:]:
            assert r == runs[0][0]
            for x, y in zip(st[:3], runs[0][1][:3]):
                np.testing.assert_array_equal(x, y)
    finally:
        for h in hs:
            bp.bpmf_destroy(h)


def test_split_agrees_with_whole_rows(bp):
    import torch
    prob = _prob(32, seed=33)
    out = []
    for split in (16, 1 << 30):
        h = bp.create_from_problem(prob, split_degree=split, flags=bp.BPMF_DEBUG_MEANS,
                                   stream=torch.cuda.Stream().cuda_stream)
        try:
            assert (bp.bpmf_info(h, 1)["n_split"] > 0) == (split == 16)
            bp.bpmf_sweep(h, 1)
            out.append([bp.bpmf_debug_means(h, s, n, prob.K) for s, n in ((0, prob.M), (1, prob.N))])
        finally:
            bp.bpmf_destroy(h)
    for side in (0, 1):
        assert rowwise_rel(out[0][side], out[1][side]).max() <= 3 * ROW_TOL
