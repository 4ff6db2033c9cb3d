"""FP64 CPU oracle of the BPMF Gibbs sampler -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never links, calls
or reads it, and it shares no code with the CUDA path: the C source in
``bpmf_oracle.c`` has its own Philox4x32-10, Box-Muller, Marsaglia-Tsang gamma,
Bartlett-Wishart, Cholesky and triangular solves, all in double precision.

This module is argument marshalling over that C source (ctypes).  What each
routine computes, and which passage of the paper (arXiv:1705.10633, Alg. 1,
Sec. 2, Sec. 3.1) or of the cited BPMF paper it follows, is stated in the C
file.  Parity pins for every function live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bpmf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, EINVAL, ENOMEM, ENOTPD, EGAMMA = 0, -1, -2, -4, -7
FLAG_CLIP = 0x2
FLAG_NO_CENTER = 0x8

USER, MOVIE = 0, 1

TAG_INIT = (0, 1)
TAG_ROW = (2, 3)
TAG_HYPER_NORMAL = (4, 5)
TAG_GAMMA = (6, 7)


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to its source with plain gcc (-O2, IEEE math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def lib():
    global _lib
    if _lib is not None:
        return _lib
    L = C.CDLL(build())
    i64p, i32p, u32p = C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_uint32)
    f32p, f64p = C.POINTER(C.c_float), C.POINTER(C.c_double)
    L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
    L.orc_normal_stream.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int64,
                                    C.c_int64, f64p]
    L.orc_gamma.argtypes = [C.c_uint64, C.c_double, C.c_uint32, C.c_uint32, C.c_uint32, f64p,
                            C.POINTER(C.c_int)]
    L.orc_cholesky.argtypes = [C.c_int, f64p, f64p]
    L.orc_spd_inverse.argtypes = [C.c_int, f64p, f64p]
    L.orc_nw_draw.argtypes = [C.c_int, C.c_int64, f64p, f64p, C.c_double, C.c_double, f64p, f64p,
                              C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, f64p, f64p]
    L.orc_row_stats.argtypes = [C.c_int64, C.c_int, f64p, f64p, f64p]
    L.orc_row_conditional.argtypes = [C.c_int, f64p, f64p, C.c_double, C.c_int64, i32p, f64p,
                                      f64p, f64p, f64p, f64p, f64p]
    L.orc_create.restype = C.c_void_p
    L.orc_create.argtypes = [C.c_int64, C.c_int64, C.c_int32, i64p, i32p, f32p, C.c_int64, i32p,
                             i32p, f32p, C.c_double, C.c_double, C.c_double, f64p, f64p,
                             C.c_uint64, C.c_uint32, C.c_int32, C.c_int32, C.c_uint32, C.c_double,
                             C.c_double, C.c_int32]
    vp = C.c_void_p
    L.orc_destroy.argtypes = [vp]
    L.orc_rbar.argtypes = [vp]
    L.orc_rbar.restype = C.c_double
    L.orc_get_sweep.argtypes = [vp]
    L.orc_get_sweep.restype = C.c_uint32
    L.orc_get_navg.argtypes = [vp]
    L.orc_get_navg.restype = C.c_int64
    L.orc_set_counters.argtypes = [vp, C.c_uint32, C.c_int64]
    L.orc_hyper.argtypes = [vp, C.c_int]
    L.orc_nw_from_stats.argtypes = [vp, C.c_int, C.c_int64, f64p, f64p, C.c_uint32, f64p, f64p]
    L.orc_rows.argtypes = [vp, C.c_int]
    L.orc_rows_subset.argtypes = [vp, C.c_int, i64p, C.c_int64]
    L.orc_rows_range.argtypes = [vp, C.c_int, C.c_int64, C.c_int64]
    L.orc_predict.argtypes = [vp, f64p, f64p]
    L.orc_sweep.argtypes = [vp, C.c_int, f64p, f64p]
    for name in ("orc_get_factors", "orc_set_factors", "orc_get_means"):
        getattr(L, name).argtypes = [vp, C.c_int, f64p]
    L.orc_get_hyper.argtypes = [vp, C.c_int, f64p, f64p]
    L.orc_set_hyper.argtypes = [vp, C.c_int, f64p, f64p]
    L.orc_get_stats.argtypes = [vp, C.c_int, f64p, f64p]
    L.orc_get_psum.argtypes = [vp, f64p]
    L.orc_set_psum.argtypes = [vp, f64p]
    _lib = L
    return L


def _check(rc, what):
    if rc != OK:
        raise RuntimeError("oracle %s failed with code %d" % (what, rc))


# ----------------------------------------------------------------------------
# Pure functions
# ----------------------------------------------------------------------------
def philox(ctr, key):
    """Philox4x32-10 of one counter (4 x uint32) under one key (2 x uint32)."""
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def normal_stream(seed, c1, c2, c3, first, count):
    out = np.empty(int(count), dtype=np.float64)
    lib().orc_normal_stream(int(seed), int(c1), int(c2), int(c3), int(first), int(count), _dp(out))
    return out


def gamma(seed, shape, c1, c2, c3):
    """Returns (draw, attempts) of Gamma(shape, 1) by Marsaglia-Tsang."""
    out = C.c_double()
    att = C.c_int()
    _check(lib().orc_gamma(int(seed), float(shape), int(c1), int(c2), int(c3), C.byref(out),
                           C.byref(att)), "gamma")
    return out.value, att.value


def cholesky(A):
    A = np.ascontiguousarray(A, dtype=np.float64)
    K = A.shape[0]
    L = np.empty_like(A)
    _check(lib().orc_cholesky(K, _dp(A), _dp(L)), "cholesky")
    return L


def spd_inverse(A):
    A = np.ascontiguousarray(A, dtype=np.float64)
    out = np.empty_like(A)
    _check(lib().orc_spd_inverse(A.shape[0], _dp(A), _dp(out)), "spd_inverse")
    return out


def row_stats(X):
    X = np.ascontiguousarray(X, dtype=np.float64)
    n, K = X.shape
    xbar = np.empty(K)
    S = np.empty((K, K))
    lib().orc_row_stats(n, K, _dp(X), _dp(xbar), _dp(S))
    return xbar, S


def nw_draw(n, xbar, S, beta0, nu0, mu0, W0inv, seed, sweep, c3_normals, c3_gamma):
    xbar = np.ascontiguousarray(xbar, dtype=np.float64)
    S = np.ascontiguousarray(S, dtype=np.float64)
    mu0 = np.ascontiguousarray(mu0, dtype=np.float64)
    W0inv = np.ascontiguousarray(W0inv, dtype=np.float64)
    K = xbar.shape[0]
    Lam = np.empty((K, K))
    mu = np.empty(K)
    _check(lib().orc_nw_draw(K, int(n), _dp(xbar), _dp(S), float(beta0), float(nu0), _dp(mu0),
                             _dp(W0inv), int(seed), int(sweep), int(c3_normals), int(c3_gamma),
                             _dp(Lam), _dp(mu)), "nw_draw")
    return Lam, mu


def row_conditional(LamX, LamMu, alpha, idx, val, Y, z):
    """One row's conditional: returns (mean, sample) for given noise z."""
    LamX = np.ascontiguousarray(LamX, dtype=np.float64)
    LamMu = np.ascontiguousarray(LamMu, dtype=np.float64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    K = LamX.shape[0]
    mean = np.empty(K)
    x = np.empty(K)
    work = np.empty(3 * K * K + 3 * K)
    _check(lib().orc_row_conditional(K, _dp(LamX), _dp(LamMu), float(alpha), len(idx),
                                     idx.ctypes.data_as(C.POINTER(C.c_int32)), _dp(val), _dp(Y),
                                     _dp(z), _dp(mean), _dp(x), _dp(work)), "row_conditional")
    return mean, x


# ----------------------------------------------------------------------------
# Whole-sampler state
# ----------------------------------------------------------------------------
class Oracle:
    """FP64 Gibbs sampler over one rating problem (see ``workloads.Problem``)."""

    def __init__(self, prob, alpha=None, beta0=2.0, nu0=None, mu0=None, W0=None, seed=None,
                 job=0, burn_in=None, order=0, flags=0, clip=(1.0, 5.0), nthreads=None):
        self.M, self.N, self.K = int(prob.M), int(prob.N), int(prob.K)
        K = self.K
        self.alpha = float(prob.alpha if alpha is None else alpha)
        self.beta0 = float(beta0)
        self.nu0 = float(K if nu0 is None else nu0)
        self.seed = int(prob.seed if seed is None else seed)
        self.burn_in = int(prob.burn_in if burn_in is None else burn_in)
        self.mu0 = np.zeros(K) if mu0 is None else np.ascontiguousarray(mu0, dtype=np.float64)
        self.W0 = np.eye(K) if W0 is None else np.ascontiguousarray(W0, dtype=np.float64)
        self.W0inv = spd_inverse(self.W0)
        self.job = int(job)
        self.flags = int(flags)
        nthreads = nthreads or os.cpu_count() or 1
        self._keep = [np.ascontiguousarray(prob.csr_ptr, dtype=np.int64),
                      np.ascontiguousarray(prob.csr_col, dtype=np.int32),
                      np.ascontiguousarray(prob.csr_val, dtype=np.float32),
                      np.ascontiguousarray(prob.test_i, dtype=np.int32),
                      np.ascontiguousarray(prob.test_j, dtype=np.int32),
                      np.ascontiguousarray(prob.test_r, dtype=np.float32)]
        p, c, v, ti, tj, tr = self._keep
        self.T = len(ti)
        self.h = lib().orc_create(
            self.M, self.N, K, p.ctypes.data_as(C.POINTER(C.c_int64)),
            c.ctypes.data_as(C.POINTER(C.c_int32)), v.ctypes.data_as(C.POINTER(C.c_float)),
            self.T, ti.ctypes.data_as(C.POINTER(C.c_int32)),
            tj.ctypes.data_as(C.POINTER(C.c_int32)), tr.ctypes.data_as(C.POINTER(C.c_float)),
            self.alpha, self.beta0, self.nu0, _dp(self.mu0), _dp(self.W0), self.seed, self.job,
            self.burn_in, int(order), self.flags, float(clip[0]), float(clip[1]), int(nthreads))
        if not self.h:
            raise RuntimeError("oracle create failed")
        self._keep = None

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().orc_destroy(h)
            self.h = None

    def n_rows(self, side):
        return self.M if side == USER else self.N

    @property
    def rbar(self):
        return lib().orc_rbar(self.h)

    @property
    def sweep_index(self):
        return lib().orc_get_sweep(self.h)

    @property
    def n_avg(self):
        return lib().orc_get_navg(self.h)

    def set_counters(self, sweep, n_avg):
        lib().orc_set_counters(self.h, int(sweep), int(n_avg))

    def sweep(self, n=1):
        rs, ra = C.c_double(), C.c_double()
        _check(lib().orc_sweep(self.h, int(n), C.byref(rs), C.byref(ra)), "sweep")
        return rs.value, ra.value

    def hyper(self, side):
        _check(lib().orc_hyper(self.h, side), "hyper")

    def rows(self, side):
        _check(lib().orc_rows(self.h, side), "rows")

    def rows_subset(self, side, rows):
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        _check(lib().orc_rows_subset(self.h, side, rows.ctypes.data_as(C.POINTER(C.c_int64)),
                                     len(rows)), "rows_subset")

    def rows_range(self, side, begin, end):
        _check(lib().orc_rows_range(self.h, side, int(begin), int(end)), "rows_range")

    def predict(self):
        rs, ra = C.c_double(), C.c_double()
        _check(lib().orc_predict(self.h, C.byref(rs), C.byref(ra)), "predict")
        return rs.value, ra.value

    def get_factors(self, side):
        out = np.empty((self.n_rows(side), self.K))
        lib().orc_get_factors(self.h, side, _dp(out))
        return out

    def set_factors(self, side, X):
        X = np.ascontiguousarray(X, dtype=np.float64).reshape(self.n_rows(side), self.K)
        lib().orc_set_factors(self.h, side, _dp(X))

    def get_means(self, side):
        out = np.empty((self.n_rows(side), self.K))
        lib().orc_get_means(self.h, side, _dp(out))
        return out

    def get_hyper(self, side):
        mu, Lam = np.empty(self.K), np.empty((self.K, self.K))
        lib().orc_get_hyper(self.h, side, _dp(mu), _dp(Lam))
        return mu, Lam

    def set_hyper(self, side, mu, Lam):
        mu = np.ascontiguousarray(mu, dtype=np.float64)
        Lam = np.ascontiguousarray(Lam, dtype=np.float64)
        lib().orc_set_hyper(self.h, side, _dp(mu), _dp(Lam))

    def get_stats(self, side):
        xbar, S = np.empty(self.K), np.empty((self.K, self.K))
        lib().orc_get_stats(self.h, side, _dp(xbar), _dp(S))
        return xbar, S

    def nw_from_stats(self, side, n, xbar, S, sweep):
        xbar = np.ascontiguousarray(xbar, dtype=np.float64)
        S = np.ascontiguousarray(S, dtype=np.float64)
        Lam, mu = np.empty((self.K, self.K)), np.empty(self.K)
        _check(lib().orc_nw_from_stats(self.h, side, int(n), _dp(xbar), _dp(S), int(sweep),
                                       _dp(Lam), _dp(mu)), "nw_from_stats")
        return Lam, mu

    def get_psum(self):
        out = np.empty(self.T)
        lib().orc_get_psum(self.h, _dp(out))
        return out

    def set_psum(self, ps):
        ps = np.ascontiguousarray(ps, dtype=np.float64)
        lib().orc_set_psum(self.h, _dp(ps))
