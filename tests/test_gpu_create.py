"""bpmf_create's device-side input pass: the column indices of the row view are range
checked on the device (BPMF_EINVAL, nothing leaked), and the ratings' mean is an FP64
sum in a fixed order, equal to the exact mean within rounding and the same on every
run; with a caller-supplied column view the host checks everything."""
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
    # with a caller-supplied column view the same input is refused on the host
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
