"""The C-ABI library builds for sm_103a, loads, and exports every entry point of
include/bpmf.h; argument validation happens on the host before any CUDA call.
No kernel runs here (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bpmf.h")


@pytest.fixture(scope="module")
def bp():
    from paper_1705_10633_gb300 import _build
    _build.build()
    import paper_1705_10633_gb300 as bp
    bp.lib()
    return bp


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(bpmf_\w+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("bpmf_create", "bpmf_sweep", "bpmf_predict", "bpmf_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(bp):
    L = C.CDLL(bp.LIB_PATH)
    for name in declared_functions():
        assert hasattr(L, name), name


def test_binding_has_the_same_names(bp):
    for name in declared_functions():
        assert hasattr(bp, name), name


def test_strerror(bp):
    assert bp.bpmf_strerror(0) == "ok"
    assert "invalid" in bp.bpmf_strerror(-1)
    assert bp.bpmf_strerror(12345) == "unknown error"


def test_destroy_null_is_ok(bp):
    assert bp.lib().bpmf_destroy(None) == 0


def _tiny():
    ptr = np.array([0, 2, 3], dtype=np.int64)
    col = np.array([0, 2, 1], dtype=np.int32)
    val = np.array([1.0, 2.0, 3.0], dtype=np.float32)
    return ptr, col, val


# Column indices of the row view are checked on the device (with the ratings' mean,
# in one pass over the uploaded arrays): see tests/test_gpu_create.py.
@pytest.mark.parametrize("case", ["bad_ptr0", "decreasing", "K0", "K65",
                                  "nu0", "alpha", "W0", "test_range", "order", "bf16"])
def test_create_rejects_malformed_input(bp, case):
    ptr, col, val = _tiny()
    M, N, K = 2, 3, 4
    kw = {}
    ti = tj = tr = None
    if case == "bad_ptr0":
        ptr = np.array([1, 2, 3], dtype=np.int64)
    elif case == "decreasing":
        ptr = np.array([0, 3, 2], dtype=np.int64)
    elif case == "col_range":
        col = np.array([0, 3, 1], dtype=np.int32)
    elif case == "neg_col":
        col = np.array([0, -1, 1], dtype=np.int32)
    elif case == "K0":
        K = 0
    elif case == "K65":
        K = 65
    elif case == "nu0":
        kw["nu0"] = K - 0.5
    elif case == "alpha":
        kw["alpha"] = 0.0
    elif case == "W0":
        kw["W0"] = -np.eye(K)
    elif case == "order":
        kw["order"] = 2
    elif case == "bf16":
        kw["flags"] = bp.BPMF_BF16_GRAM
    elif case == "test_range":
        ti, tj, tr = np.array([5], np.int32), np.array([0], np.int32), np.array([1.0], np.float32)
    p = bp.bpmf_default_params(**kw)
    with pytest.raises(bp.BpmfError) as ei:
        bp.bpmf_create(M, N, K, ptr, col, val, test_i=ti, test_j=tj, test_r=tr, params=p)
    assert ei.value.code == bp.BPMF_EINVAL


def test_create_without_gpu_reports_cuda_error(bp):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    ptr, col, val = _tiny()
    with pytest.raises(bp.BpmfError) as ei:
        bp.bpmf_create(2, 3, 4, ptr, col, val)
    assert ei.value.code == bp.BPMF_ECUDA


def test_product_code_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_1705_10633_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text.lower(), f


def test_set_tuning_and_batch_reject_null(bp):
    assert bp.lib().bpmf_set_tuning(None, 1, 1, 1) == bp.BPMF_EINVAL
    assert bp.lib().bpmf_set_row_timing(None, 1) == bp.BPMF_EINVAL
    arr = (__import__("ctypes").c_void_p * 1)(None)
    assert bp.lib().bpmf_sweep_batch(arr, 1, 1) == bp.BPMF_EINVAL
    assert bp.lib().bpmf_sweep_batch(arr, -1, 1) == bp.BPMF_EINVAL


def test_row_stats_noalloc_rejects_misaligned_pointers_on_the_host(bp):
    # checked before any CUDA call, so no device is needed: the pointers are never used
    base = 1 << 20
    for X, mean, S, shift in ((base + 4, base, base, 0), (base + 8, base, base, 0),
                              (base, base + 4, base, 0), (base, base, base + 2, 0),
                              (base, base, base, base + 4)):
        rc = bp.lib().bpmf_row_stats_noalloc(X, 100, 16, shift or None, mean, S, None)
        assert rc == bp.BPMF_EINVAL
    assert bp.lib().bpmf_row_stats_noalloc(base, 100, 65, None, base, base, None) == bp.BPMF_EINVAL
    assert bp.lib().bpmf_row_stats_noalloc(base, 0, 16, None, base, base, None) == bp.BPMF_EINVAL


def test_device_bytes_is_host_only_and_follows_the_buffers(bp):
    """bpmf_device_bytes runs without a GPU when the SM count is given, and moves with
    the buffers bpmf_create makes: the 16-bit factor copies and per-row scratch of the
    tensor-core route, the conditional means, the test set; bad input is refused on the
    host.  (That it equals what bpmf_create holds is checked on the GPU.)"""
    import workloads
    prob = workloads.random_small(2000, 600, 64, 50000, seed=7, n_test=200, long_rows=4,
                                  long_deg=500)

    def nbytes(K=64, n_test=200, **kw):
        return bp.bpmf_device_bytes(prob.M, prob.N, K, prob.csr_ptr, prob.csr_col, n_test,
                                    params=bp.bpmf_default_params(**kw), num_sms=152)

    base = nbytes()
    # rows with at least 16 ratings take the tensor-core route at K = 64: one 8,960-B
    # scratch slot per row of the larger long bin
    deg_u = np.diff(prob.csr_ptr)
    deg_v = np.bincount(prob.csr_col, minlength=prob.N)
    n_long = max(int((deg_u >= 16).sum()), int((deg_v >= 16).sum()))
    assert n_long > 0
    cuda_core = nbytes(flags=bp.BPMF_CUDA_CORE_GRAM)
    assert base - cuda_core >= n_long * 8960 + 2 * 2 * (prob.M + prob.N) * 64
    # the conditional means: one FP32 row per row of each side
    assert nbytes(flags=bp.BPMF_DEBUG_MEANS) - base >= 4 * 64 * (prob.M + prob.N)
    # K = 16 rows are a quarter of the K = 64 rows and take no tensor-core route
    assert nbytes(K=16) < cuda_core
    # each test point: index pair, rating and FP64 running sum
    assert nbytes(n_test=200 + 64 * 1024) - base >= 20 * 64 * 1024
    for bad in (dict(K=0), dict(K=65), dict(n_test=-1)):
        with pytest.raises(bp.BpmfError) as ei:
            nbytes(**bad)
        assert ei.value.code == bp.BPMF_EINVAL
    col = prob.csr_col.copy()
    col[5] = prob.N  # a column outside [0, N)
    with pytest.raises(bp.BpmfError) as ei:
        bp.bpmf_device_bytes(prob.M, prob.N, 64, prob.csr_ptr, col, 0, num_sms=152)
    assert ei.value.code == bp.BPMF_EINVAL


def test_batch_object_rejects_bad_arguments_on_the_host(bp):
    lib = bp.lib()
    out = C.c_void_p()
    arr = (C.c_void_p * 1)(None)
    assert lib.bpmf_batch_create(arr, 1, None, C.byref(out)) == bp.BPMF_EINVAL  # NULL handle
    assert lib.bpmf_batch_create(arr, 0, None, C.byref(out)) == bp.BPMF_EINVAL  # no chains
    assert lib.bpmf_batch_create(arr, 1, None, None) == bp.BPMF_EINVAL
    assert lib.bpmf_batch_sweep(None, 1) == bp.BPMF_EINVAL
    n = C.c_int64()
    assert lib.bpmf_batch_launch_count(None, C.byref(n)) == bp.BPMF_EINVAL
    assert lib.bpmf_batch_destroy(None) == bp.BPMF_OK
