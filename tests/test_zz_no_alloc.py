"""The allocation-free row-statistics entry point against the handle's hyper step.

bpmf_row_stats_noalloc serves callers that cannot allocate device memory when
they need the reduction (a serving process whose pool already holds the whole
GPU, or a loop where cudaMalloc would synchronise the device).  It keeps its
scratch in a static device array shared by every call, so this test calls it
twice in a row and checks both results against bpmf_get_stats of a handle that
ran the same reduction (same rows, same shift).  This file is collected last.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


def test_row_stats_noalloc_matches_hyper_step_twice():
    import torch

    import paper_1705_10633_gb300 as bp

    torch.cuda.set_device(0)
    stream = bp.torch_stream()
    for K, M in ((64, 5000), (10, 3000)):
        prob = workloads.random_small(M, 400, K, 20 * M, seed=40 + K)
        h = bp.create_from_problem(prob, stream=stream)
        try:
            rng = np.random.default_rng(K)
            U = (rng.standard_normal((prob.M, K)) * 0.7 + 0.2).astype(np.float32)
            assert prob.M >= 256
            _, V, hyper, s = bp.bpmf_get_state(h, prob.M, prob.N, K)
            bp.bpmf_set_state(h, U, V, hyper, s)
            # the shift the hyper step uses: the FP64 mean of the first 256 rows, summed
            # row by row in order
            acc = np.zeros(K)
            for r in range(256):
                acc += U[r].astype(np.float64)
            shift = acc / 256.0
            bp.bpmf_step(h, bp.BPMF_PHASE_HYPER_USER)
            n, mean_ref, S_ref = bp.bpmf_get_stats(h, 0, K)
        finally:
            bp.bpmf_destroy(h)
        kp = (K + 15) // 16 * 16
        Xd = torch.zeros((prob.M, kp), dtype=torch.float32, device="cuda")
        Xd[:, :K] = torch.from_numpy(U).cuda()
        shift_d = torch.from_numpy(shift).cuda()
        for call in range(2):
            mean_d = torch.full((K,), float("nan"), dtype=torch.float64, device="cuda")
            S_d = torch.full((K, K), float("nan"), dtype=torch.float64, device="cuda")
            bp.bpmf_row_stats_noalloc(Xd.data_ptr(), prob.M, K, shift_d.data_ptr(), mean_d.data_ptr(),
                                      S_d.data_ptr(), stream)
            torch.cuda.synchronize()
            assert n == prob.M
            np.testing.assert_allclose(mean_d.cpu().numpy(), mean_ref, rtol=1e-10, atol=1e-12)
            np.testing.assert_allclose(S_d.cpu().numpy(), S_ref, rtol=1e-10, atol=1e-12)
    with pytest.raises(bp.BpmfError) as ei:
        bp.bpmf_row_stats_noalloc(Xd.data_ptr(), prob.M, 65, None, mean_d.data_ptr(),
                                  S_d.data_ptr(), stream)
    assert ei.value.code == bp.BPMF_EINVAL


def test_row_stats_noalloc_many_rows_without_shift_against_the_oracle():
    """A side larger than the reduction's block limit (the scratch holds 160 block
    partials; 400,000 rows would ask for more), summed without a shift (NULL): the
    mean and scatter match the FP64 oracle's row statistics within the FP32-chunk
    rounding of the device sums, and a second call gives the same bits."""
    import torch

    import paper_1705_10633_gb300 as bp

    torch.cuda.set_device(0)
    stream = bp.torch_stream()
    M, K = 400_000, 64
    rng = np.random.default_rng(5)
    U = (rng.standard_normal((M, K)) * 0.5 + 0.1).astype(np.float32)
    mean_ref, S_ref = oracle.row_stats(U.astype(np.float64))
    Xd = torch.from_numpy(U).cuda()
    outs = []
    for call in range(2):
        mean_d = torch.full((K,), float("nan"), dtype=torch.float64, device="cuda")
        S_d = torch.full((K, K), float("nan"), dtype=torch.float64, device="cuda")
        bp.bpmf_row_stats_noalloc(Xd.data_ptr(), M, K, None, mean_d.data_ptr(), S_d.data_ptr(),
                                  stream)
        torch.cuda.synchronize()
        outs.append((mean_d.cpu().numpy(), S_d.cpu().numpy()))
    mean, S = outs[0]
    # FP32 partial sums of ~1k rows: relative error well below 1e-5 of the scale
    assert np.abs(mean - mean_ref).max() <= 1e-5 * np.abs(mean_ref).max()
    assert np.abs(S - S_ref).max() <= 1e-5 * np.abs(S_ref).max()
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
