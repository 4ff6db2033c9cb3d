"""GB300 BPMF Gibbs sampler: Python binding of the C ABI declared in ``include/bpmf.h``.

Every function here has the name of the C entry point it calls and only
marshals arguments (numpy arrays in, numpy arrays out); all of the sampler's
work runs in the sm_103a kernels of ``libbpmf.so``.  There is no CPU fallback:
importing the binding when the library has not been built raises.

PyTorch is optional plumbing: ``torch_stream()`` hands the current CUDA stream
to ``bpmf_create`` and ``torch_allocator()`` routes the library's device
allocations through PyTorch's caching allocator.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbpmf.so")

BPMF_OK, BPMF_EINVAL, BPMF_ENOMEM, BPMF_ECUDA = 0, -1, -2, -3
BPMF_ENOTPD, BPMF_ETIMEOUT, BPMF_ENAN, BPMF_EGAMMA = -4, -5, -6, -7

BPMF_BF16_GRAM = 0x1
BPMF_CLIP = 0x2
BPMF_DEBUG_MEANS = 0x4
BPMF_NO_CENTER = 0x8
BPMF_CUDA_CORE_GRAM = 0x10
BPMF_TEST_STALL = 0x100

BPMF_USER, BPMF_MOVIE = 0, 1
(BPMF_PHASE_HYPER_USER, BPMF_PHASE_HYPER_MOVIE, BPMF_PHASE_ROWS_USER, BPMF_PHASE_ROWS_MOVIE,
 BPMF_PHASE_PREDICT, BPMF_PHASE_ADVANCE) = range(6)

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class bpmf_params(C.Structure):
    _fields_ = [("alpha", C.c_double), ("beta0", C.c_double), ("nu0", C.c_double),
                ("mu0", C.POINTER(C.c_double)), ("W0", C.POINTER(C.c_double)),
                ("seed", C.c_uint64), ("job_id", C.c_uint32), ("burn_in", C.c_int32),
                ("order", C.c_int32), ("flags", C.c_uint32), ("clip_lo", C.c_double),
                ("clip_hi", C.c_double), ("long_min_degree", C.c_int32),
                ("wait_timeout_ms", C.c_int32), ("split_degree", C.c_int32),
                ("rank_one_degree", C.c_int32),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", C.c_void_p)]


class BpmfError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__("%s: %s (%d)" % (what, bpmf_strerror(code), code))


_lib = None


def lib():
    """Load ``libbpmf.so``; raises if it has not been built (no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libbpmf.so is not built; run `python -c 'import __graft_entry__ as g; "
                          "g.build()'`")
    L = C.CDLL(LIB_PATH)
    vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
    P = C.POINTER
    L.bpmf_default_params.argtypes = [P(bpmf_params)]
    L.bpmf_create.argtypes = [P(vp), i64, i64, i32, vp, vp, vp, vp, vp, vp, i64, vp, vp, vp,
                              P(bpmf_params), vp]
    L.bpmf_sweep.argtypes = [vp, i32, P(C.c_double), P(C.c_double)]
    L.bpmf_sweep_batch.argtypes = [P(vp), i32, i32]
    L.bpmf_step.argtypes = [vp, i32]
    L.bpmf_set_tuning.argtypes = [vp, i32, i32, i32]
    L.bpmf_predict.argtypes = [vp, i64, vp, vp, vp, i32]
    L.bpmf_get_state.argtypes = [vp, vp, vp, vp, P(C.c_uint64)]
    L.bpmf_set_state.argtypes = [vp, vp, vp, vp, C.c_uint64]
    L.bpmf_get_accum.argtypes = [vp, vp, P(i64)]
    L.bpmf_set_accum.argtypes = [vp, vp, i64]
    L.bpmf_get_stats.argtypes = [vp, i32, P(i64), vp, vp]
    L.bpmf_debug_means.argtypes = [vp, i32, vp]
    L.bpmf_status.argtypes = [vp]
    L.bpmf_info.argtypes = [vp, i32, P(i64), P(i64), P(i64), P(i64), P(C.c_double), P(i64),
                            P(i32)]
    L.bpmf_launch_count.argtypes = [vp, P(i64)]
    L.bpmf_balance_rows.argtypes = [i64, P(i64), i64, P(i32), P(i64), P(i32)]
    L.bpmf_bin_rows.argtypes = [i64, P(i64), i64, P(i32), P(i64)]
    L.bpmf_device_bytes.argtypes = [i64, i64, i32, vp, vp, i64, P(bpmf_params), i32, P(i64)]
    L.bpmf_batch_create.argtypes = [P(vp), i32, vp, P(vp)]
    L.bpmf_batch_sweep.argtypes = [vp, i32]
    L.bpmf_batch_launch_count.argtypes = [vp, P(i64)]
    L.bpmf_batch_destroy.argtypes = [vp]
    L.bpmf_set_row_timing.argtypes = [vp, i32]
    L.bpmf_row_launch_ms.argtypes = [vp, P(C.c_float), P(C.c_float), P(C.c_float)]
    L.bpmf_row_stats_noalloc.argtypes = [vp, i64, i32, vp, vp, vp, vp]
    L.bpmf_set_shard.argtypes = [vp, i32, i64, i64]
    L.bpmf_get_rows.argtypes = [vp, i32, i64, i64, vp, i32]
    L.bpmf_put_rows.argtypes = [vp, i32, i64, i64, vp, i32]
    L.bpmf_strerror.argtypes = [C.c_int]
    L.bpmf_strerror.restype = C.c_char_p
    L.bpmf_destroy.argtypes = [vp]
    _lib = L
    return L


def _ptr(a):
    return None if a is None else a.ctypes.data


def _check(rc, what):
    if rc != BPMF_OK:
        raise BpmfError(rc, what)


def bpmf_strerror(code):
    return lib().bpmf_strerror(int(code)).decode()


def bpmf_default_params(**kw):
    """bpmf_params filled with the library defaults, then with `kw` (mu0/W0 as arrays)."""
    p = bpmf_params()
    _check(lib().bpmf_default_params(C.byref(p)), "bpmf_default_params")
    keep = []
    for k, v in kw.items():
        if k in ("mu0", "W0"):
            if v is None:
                continue
            arr = np.ascontiguousarray(v, dtype=np.float64)
            keep.append(arr)
            setattr(p, k, arr.ctypes.data_as(C.POINTER(C.c_double)))
        elif k in ("alloc", "free"):
            setattr(p, k, v)
        else:
            setattr(p, k, v)
    p._keep = keep
    return p


def torch_stream():
    """The current PyTorch CUDA stream as a raw cudaStream_t (int)."""
    import torch
    return int(torch.cuda.current_stream().cuda_stream)


def torch_allocator(params):
    """Route the handle's device allocations through PyTorch's caching allocator."""
    import torch

    dev = torch.cuda.current_device()

    def _alloc(nbytes, stream, ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0))
        except Exception:  # out of memory -> NULL -> BPMF_ENOMEM
            return None

    def _free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    params.alloc = ALLOC_FN(_alloc)
    params.free = FREE_FN(_free)
    params._cb = (params.alloc, params.free)  # keep the thunks alive
    return params


def bpmf_create(M, N, K, csr_ptr, csr_col, csr_val, csc_ptr=None, csc_row=None, csc_val=None,
                test_i=None, test_j=None, test_r=None, params=None, stream=None):
    """Returns an opaque handle (int).  Host arrays are copied during the call."""
    L = lib()
    a = [np.ascontiguousarray(csr_ptr, dtype=np.int64), np.ascontiguousarray(csr_col, dtype=np.int32),
         np.ascontiguousarray(csr_val, dtype=np.float32)]
    csc = [None, None, None]
    if csc_ptr is not None:
        csc = [np.ascontiguousarray(csc_ptr, dtype=np.int64),
               np.ascontiguousarray(csc_row, dtype=np.int32),
               np.ascontiguousarray(csc_val, dtype=np.float32)]
    T = 0 if test_i is None else len(test_i)
    t = [None, None, None]
    if T:
        t = [np.ascontiguousarray(test_i, dtype=np.int32), np.ascontiguousarray(test_j, dtype=np.int32),
             np.ascontiguousarray(test_r, dtype=np.float32)]
    h = C.c_void_p()
    p = params if params is not None else bpmf_default_params()
    rc = L.bpmf_create(C.byref(h), int(M), int(N), int(K), *[_ptr(x) for x in a],
                       *[_ptr(x) for x in csc], int(T), *[_ptr(x) for x in t], C.byref(p),
                       None if stream is None else C.c_void_p(int(stream)))
    _check(rc, "bpmf_create")
    return h.value


def bpmf_sweep(h, n_sweeps=1, want_rmse=True):
    """Returns (rmse_sample, rmse_avg) of the last sweep, or None when not requested."""
    if want_rmse:
        rs, ra = C.c_double(), C.c_double()
        _check(lib().bpmf_sweep(h, int(n_sweeps), C.byref(rs), C.byref(ra)), "bpmf_sweep")
        return rs.value, ra.value
    _check(lib().bpmf_sweep(h, int(n_sweeps), None, None), "bpmf_sweep")
    return None


def bpmf_sweep_batch(handles, n_sweeps=1):
    """n_sweeps sweeps of every chain in `handles`, interleaved (chains on different
    streams run concurrently).  Does not wait."""
    arr = (C.c_void_p * len(handles))(*[int(h) if not isinstance(h, C.c_void_p) else h.value
                                         for h in handles])
    _check(lib().bpmf_sweep_batch(arr, len(handles), int(n_sweeps)), "bpmf_sweep_batch")


def bpmf_batch_create(handles, stream=None):
    """A batch over `handles` (borrowed): every step of a sweep runs for all of them in
    shared launches on `stream` (a cudaStream_t as int).  Returns an opaque handle."""
    arr = (C.c_void_p * len(handles))(*[int(h) if not isinstance(h, C.c_void_p) else h.value
                                         for h in handles])
    b = C.c_void_p()
    _check(lib().bpmf_batch_create(arr, len(handles), None if stream is None else C.c_void_p(int(stream)),
                                   C.byref(b)), "bpmf_batch_create")
    return b.value


def bpmf_batch_sweep(b, n_sweeps=1):
    """n_sweeps sweeps of every chain of the batch.  Does not wait."""
    _check(lib().bpmf_batch_sweep(b, int(n_sweeps)), "bpmf_batch_sweep")


def bpmf_batch_launch_count(b):
    n = C.c_int64()
    _check(lib().bpmf_batch_launch_count(b, C.byref(n)), "bpmf_batch_launch_count")
    return n.value


def bpmf_batch_destroy(b):
    _check(lib().bpmf_batch_destroy(b), "bpmf_batch_destroy")


def bpmf_set_tuning(h, long_min_degree=0, split_degree=0, rank_one_degree=0):
    """Re-bin and re-split a live handle's rows under new thresholds (0: library
    defaults; see bpmf_params for negative values)."""
    _check(lib().bpmf_set_tuning(h, int(long_min_degree), int(split_degree), int(rank_one_degree)),
           "bpmf_set_tuning")


def bpmf_step(h, phase):
    _check(lib().bpmf_step(h, int(phase)), "bpmf_step")


def bpmf_predict(h, i, j):
    i = np.ascontiguousarray(i, dtype=np.int32)
    j = np.ascontiguousarray(j, dtype=np.int32)
    out = np.empty(len(i), dtype=np.float32)
    _check(lib().bpmf_predict(h, len(i), _ptr(i), _ptr(j), _ptr(out), 0), "bpmf_predict")
    return out


def bpmf_predict_device(h, n, i_ptr, j_ptr, out_ptr):
    """Device-pointer form (where = 1): raw device addresses, ordered on the handle's stream."""
    _check(lib().bpmf_predict(h, int(n), i_ptr, j_ptr, out_ptr, 1), "bpmf_predict")


def bpmf_get_state(h, M, N, K):
    U = np.empty((M, K), dtype=np.float32)
    V = np.empty((N, K), dtype=np.float32)
    hyper = np.empty(2 * (K + K * K), dtype=np.float64)
    sweep = C.c_uint64()
    _check(lib().bpmf_get_state(h, _ptr(U), _ptr(V), _ptr(hyper), C.byref(sweep)), "bpmf_get_state")
    return U, V, hyper, sweep.value


def bpmf_set_state(h, U=None, V=None, hyper=None, sweep=0):
    U = None if U is None else np.ascontiguousarray(U, dtype=np.float32)
    V = None if V is None else np.ascontiguousarray(V, dtype=np.float32)
    hyper = None if hyper is None else np.ascontiguousarray(hyper, dtype=np.float64)
    _check(lib().bpmf_set_state(h, _ptr(U), _ptr(V), _ptr(hyper), int(sweep)), "bpmf_set_state")


def bpmf_get_accum(h, T):
    ps = np.empty(T, dtype=np.float64)
    n = C.c_int64()
    _check(lib().bpmf_get_accum(h, _ptr(ps) if T else None, C.byref(n)), "bpmf_get_accum")
    return ps, n.value


def bpmf_set_accum(h, psum, n_avg):
    psum = None if psum is None else np.ascontiguousarray(psum, dtype=np.float64)
    _check(lib().bpmf_set_accum(h, _ptr(psum), int(n_avg)), "bpmf_set_accum")


def bpmf_get_stats(h, side, K):
    mean = np.empty(K, dtype=np.float64)
    S = np.empty((K, K), dtype=np.float64)
    n = C.c_int64()
    _check(lib().bpmf_get_stats(h, int(side), C.byref(n), _ptr(mean), _ptr(S)), "bpmf_get_stats")
    return n.value, mean, S


def bpmf_debug_means(h, side, rows, K):
    out = np.empty((rows, K), dtype=np.float32)
    _check(lib().bpmf_debug_means(h, int(side), _ptr(out)), "bpmf_debug_means")
    return out


def bpmf_status(h):
    return lib().bpmf_status(h)


def bpmf_info(h, side):
    ns, nl, nsp, nsg, nb = (C.c_int64() for _ in range(5))
    rb = C.c_double()
    bal = C.c_int32()
    _check(lib().bpmf_info(h, int(side), C.byref(ns), C.byref(nl), C.byref(nsp), C.byref(nsg),
                           C.byref(rb), C.byref(nb), C.byref(bal)), "bpmf_info")
    return {"n_short": ns.value, "n_long": nl.value, "n_split": nsp.value,
            "n_segments": nsg.value, "rbar": rb.value, "device_bytes": nb.value,
            "balanced": bal.value}


def bpmf_device_bytes(M, N, K, csr_ptr, csr_col, n_test=0, params=None, num_sms=0):
    """Device bytes bpmf_create would hold for this problem (host only; num_sms <= 0:
    the current device's SM count)."""
    p = params if params is not None else bpmf_default_params()
    a = [np.ascontiguousarray(csr_ptr, dtype=np.int64), np.ascontiguousarray(csr_col, dtype=np.int32)]
    out = C.c_int64()
    _check(lib().bpmf_device_bytes(int(M), int(N), int(K), _ptr(a[0]), _ptr(a[1]), int(n_test),
                                   C.byref(p), int(num_sms), C.byref(out)), "bpmf_device_bytes")
    return out.value


def bpmf_bin_rows(ptr, long_min):
    """Degree bins of one side's rows (offsets `ptr`, rows + 1 entries): (order, n_short),
    the short bin then the long bin (rows of at least long_min ratings), each longest first.
    Host only."""
    p = np.ascontiguousarray(ptr, dtype=np.int64)
    rows = p.shape[0] - 1
    order = np.empty(max(rows, 1), dtype=np.int32)
    ns = C.c_int64()
    _check(lib().bpmf_bin_rows(rows, p.ctypes.data_as(C.POINTER(C.c_int64)), int(long_min),
                               order.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(ns)),
           "bpmf_bin_rows")
    return order[:rows], ns.value


def bpmf_balance_rows(degree, grid):
    """The balanced plan for rows of the given rating counts (longest first) over `grid`
    CTAs: (order, first) numpy arrays, or None when round-robin is kept.  Host only."""
    deg = np.ascontiguousarray(degree, dtype=np.int64)
    n = deg.shape[0]
    order = np.empty(max(n, 1), dtype=np.int32)
    first = np.empty(min(n, int(grid)) + 1 if n else 1, dtype=np.int64)
    planned = C.c_int32()
    _check(lib().bpmf_balance_rows(n, deg.ctypes.data_as(C.POINTER(C.c_int64)), int(grid),
                                   order.ctypes.data_as(C.POINTER(C.c_int32)),
                                   first.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(planned)),
           "bpmf_balance_rows")
    return (order[:n], first) if planned.value else None


def bpmf_set_row_timing(h, on=True):
    """Record CUDA events around the row kernels of phases run by bpmf_step."""
    _check(lib().bpmf_set_row_timing(h, 1 if on else 0), "bpmf_set_row_timing")


def bpmf_row_launch_ms(h):
    """(CUDA-core ms, Gram ms, factorisation ms) of the last timed row phase; -1 for a
    part that did not launch."""
    a, b, c = C.c_float(), C.c_float(), C.c_float()
    _check(lib().bpmf_row_launch_ms(h, C.byref(a), C.byref(b), C.byref(c)), "bpmf_row_launch_ms")
    return a.value, b.value, c.value


def bpmf_launch_count(h):
    n = C.c_int64()
    _check(lib().bpmf_launch_count(h, C.byref(n)), "bpmf_launch_count")
    return n.value


def bpmf_row_stats_noalloc(X_ptr, rows, K, shift_ptr, mean_ptr, S_ptr, stream=None):
    """Device pointers in and out (see include/bpmf.h); allocates nothing."""
    _check(lib().bpmf_row_stats_noalloc(X_ptr, int(rows), int(K), shift_ptr, mean_ptr, S_ptr,
                                        None if stream is None else C.c_void_p(int(stream))),
           "bpmf_row_stats_noalloc")


def bpmf_set_shard(h, side, row_begin, row_end):
    """Restrict the row phases of `side` to rows [row_begin, row_end)."""
    _check(lib().bpmf_set_shard(h, int(side), int(row_begin), int(row_end)), "bpmf_set_shard")


def bpmf_get_rows(h, side, row_begin, row_end, K, out_ptr=None):
    """Rows [row_begin, row_end) of U (side 0) or V (side 1): a new host array, or into the
    device buffer at out_ptr (K floats a row, ordered on the handle's stream)."""
    if out_ptr is not None:
        _check(lib().bpmf_get_rows(h, int(side), int(row_begin), int(row_end), out_ptr, 1),
               "bpmf_get_rows")
        return None
    out = np.empty((max(int(row_end) - int(row_begin), 0), int(K)), dtype=np.float32)
    _check(lib().bpmf_get_rows(h, int(side), int(row_begin), int(row_end), _ptr(out), 0),
           "bpmf_get_rows")
    return out


def bpmf_put_rows(h, side, row_begin, row_end, rows=None, in_ptr=None):
    """Overwrite rows [row_begin, row_end) of U or V from a host array (n x K) or from the
    device buffer at in_ptr."""
    if in_ptr is not None:
        _check(lib().bpmf_put_rows(h, int(side), int(row_begin), int(row_end), in_ptr, 1),
               "bpmf_put_rows")
        return
    rows = np.ascontiguousarray(rows, dtype=np.float32)
    _check(lib().bpmf_put_rows(h, int(side), int(row_begin), int(row_end), _ptr(rows), 0),
           "bpmf_put_rows")


def bpmf_destroy(h):
    if h:
        _check(lib().bpmf_destroy(h), "bpmf_destroy")


def create_from_problem(prob, flags=0, seed=None, burn_in=None, params=None, stream=None, **kw):
    """bpmf_create for a ``workloads.Problem`` (sizes, CSR, test set, alpha, seed, burn-in)."""
    if params is None:
        params = bpmf_default_params(alpha=float(prob.alpha), seed=int(prob.seed if seed is None else seed),
                                     burn_in=int(prob.burn_in if burn_in is None else burn_in),
                                     flags=int(flags), **kw)
    return bpmf_create(prob.M, prob.N, prob.K, prob.csr_ptr, prob.csr_col, prob.csr_val,
                       test_i=prob.test_i, test_j=prob.test_j, test_r=prob.test_r, params=params,
                       stream=stream)


EXPORTED = ["bpmf_default_params", "bpmf_create", "bpmf_sweep", "bpmf_sweep_batch",
            "bpmf_batch_create", "bpmf_batch_sweep", "bpmf_batch_launch_count", "bpmf_batch_destroy",
            "bpmf_set_tuning", "bpmf_step",
            "bpmf_predict",
            "bpmf_get_state", "bpmf_set_state", "bpmf_get_accum", "bpmf_set_accum",
            "bpmf_get_stats", "bpmf_debug_means", "bpmf_status", "bpmf_info", "bpmf_launch_count",
            "bpmf_set_row_timing", "bpmf_row_launch_ms", "bpmf_bin_rows", "bpmf_balance_rows",
            "bpmf_device_bytes",
            "bpmf_row_stats_noalloc", "bpmf_set_shard", "bpmf_get_rows", "bpmf_put_rows",
            "bpmf_strerror",
            "bpmf_destroy"]
