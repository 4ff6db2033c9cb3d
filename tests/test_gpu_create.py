"""bpmf_create's device-side input pass: the column indices of the row view are range
checked on the device (BPMF_EINVAL, nothing leaked), and the ratings' mean is an FP64
sum in a fixed order, equal to the exact mean within rounding and the same on every
run; a caller-supplied column view is checked for structure on the host and, entry by
entry, against the view the library builds from the rows; bpmf_device_bytes gives, before
any allocation, the bytes the handle then holds."""
import math

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bp():
    import torch
    torch.cuda.set_device(0)
    import paper_1705_10633_gb300 as bp
    bp.lib()
    return bp


@pytest.mark.parametrize("bad", [3, -1, 1 << 30])
def test_out_of_range_column_is_rejected(bp, bad):
    ptr = np.array([0, 2, 3], dtype=np.int64)
    col = np.array([0, bad, 1], dtype=np.int32)
    val = np.array([1.0, 2.0, 3.0], dtype=np.float32)
    with pytest.raises(bp.BpmfError) as ei:
        bp.bpmf_create(2, 3, 4, ptr, col, val, stream=bp.torch_stream())
    assert ei.value.code == bp.BPMF_EINVAL
    # with a caller-supplied column view the same input is refused too
    cp = np.array([0, 1, 2, 3], dtype=np.int64)
    cr = np.array([0, 1, 0], dtype=np.int32)
    with pytest.raises(bp.BpmfError) as ei:
        bp.bpmf_create(2, 3, 4, ptr, col, val, csc_ptr=cp, csc_row=cr, csc_val=val,
                       stream=bp.torch_stream())
    assert ei.value.code == bp.BPMF_EINVAL


def test_mean_is_exact_within_rounding_and_reproducible(bp):
    prob = workloads.random_small(3000, 700, 8, 200000, seed=91)
    # values far from zero with a wide spread, so the summation order matters in FP32
    val = (1e4 + np.random.default_rng(3).standard_normal(prob.nnz) * 1e3).astype(np.float32)
    exact = math.fsum(val.astype(np.float64)) / prob.nnz
    got = []
    for _ in range(3):
        h = bp.bpmf_create(prob.M, prob.N, prob.K, prob.csr_ptr, prob.csr_col, val,
                           stream=bp.torch_stream())
        try:
            got.append(bp.bpmf_info(h, 0)["rbar"])
        finally:
            bp.bpmf_destroy(h)
    assert got[0] == got[1] == got[2]
    assert abs(got[0] - exact) <= 1e-13 * abs(exact)


def test_caller_column_view_must_be_the_transpose(bp):
    """The column view a caller passes must hold the row view's ratings (rows ascending
    in each column): the true transpose gives the same chain as no column view; the same
    structure with its values permuted inside a column, or two row indices swapped, is
    refused with BPMF_EINVAL."""
    prob = workloads.random_small(300, 120, 16, 6000, seed=12, n_test=50)
    cptr, crow, cval = prob.csc()
    a = bp.create_from_problem(prob, stream=bp.torch_stream())
    b = bp.bpmf_create(prob.M, prob.N, prob.K, prob.csr_ptr, prob.csr_col, prob.csr_val,
                       csc_ptr=cptr, csc_row=crow, csc_val=cval,
                       test_i=prob.test_i, test_j=prob.test_j, test_r=prob.test_r,
                       params=bp.bpmf_default_params(alpha=prob.alpha, seed=prob.seed,
                                                     burn_in=prob.burn_in),
                       stream=bp.torch_stream())
    try:
        assert bp.bpmf_sweep(a, 2) == bp.bpmf_sweep(b, 2)
        sa = bp.bpmf_get_state(a, prob.M, prob.N, prob.K)
        sb = bp.bpmf_get_state(b, prob.M, prob.N, prob.K)
        for x, y in zip(sa[:3], sb[:3]):
            np.testing.assert_array_equal(x, y)
    finally:
        bp.bpmf_destroy(a)
        bp.bpmf_destroy(b)
    j = int(np.argmax(np.diff(cptr)))  # a column with several ratings
    lo, hi = int(cptr[j]), int(cptr[j + 1])
    assert hi - lo >= 2 and cval[lo] != cval[lo + 1]
    bad_val = cval.copy()
    bad_val[lo], bad_val[lo + 1] = cval[lo + 1], cval[lo]
    bad_row = crow.copy()
    bad_row[lo], bad_row[lo + 1] = crow[lo + 1], crow[lo]
    for r, v in ((crow, bad_val), (bad_row, cval)):
        with pytest.raises(bp.BpmfError) as ei:
            bp.bpmf_create(prob.M, prob.N, prob.K, prob.csr_ptr, prob.csr_col, prob.csr_val,
                           csc_ptr=cptr, csc_row=r, csc_val=v, stream=bp.torch_stream())
        assert ei.value.code == bp.BPMF_EINVAL


@pytest.mark.parametrize("K, flags, kw", [
    (16, 0, {}),
    (32, 0, {"split_degree": 64}),           # split rows: segment buffers
    (64, 0, {}),                             # tensor-core bins, plans and scratch
    (64, 0x4, {"long_min_degree": 16}),      # BPMF_DEBUG_MEANS, a larger long bin
    (64, 0x10, {}),                          # BPMF_CUDA_CORE_GRAM: no tensor-core buffers
])
def test_device_bytes_is_what_create_holds(bp, K, flags, kw):
    """bpmf_device_bytes, computed on the host before any allocation, equals the device
    bytes the handle holds after bpmf_create (the figure a server admits jobs by)."""
    import torch
    prob = workloads.random_small(2500, 700, K, 70000, seed=41 + K, n_test=300, empty_rows=3,
                                  long_rows=5, long_deg=600)
    params = bp.bpmf_default_params(alpha=float(prob.alpha), seed=3, flags=flags, **kw)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    want = bp.bpmf_device_bytes(prob.M, prob.N, prob.K, prob.csr_ptr, prob.csr_col,
                                len(prob.test_i), params=params, num_sms=sms)
    assert want == bp.bpmf_device_bytes(prob.M, prob.N, prob.K, prob.csr_ptr, prob.csr_col,
                                        len(prob.test_i), params=params)  # current device
    h = bp.bpmf_create(prob.M, prob.N, prob.K, prob.csr_ptr, prob.csr_col, prob.csr_val,
                       test_i=prob.test_i, test_j=prob.test_j, test_r=prob.test_r,
                       params=params, stream=bp.torch_stream())
    try:
        assert bp.bpmf_info(h, 0)["device_bytes"] == want
        if K == 64 and not flags & 0x10:
            assert bp.bpmf_info(h, 0)["n_long"] > 0
    finally:
        bp.bpmf_destroy(h)
