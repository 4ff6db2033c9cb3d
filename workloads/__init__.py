"""Seeded synthetic rating problems for the BPMF Gibbs sampler.

This module holds input generators only: it draws rating matrices with the
shape, sparsity pattern, degree distribution and value distribution of the
workloads below, and none of the sampler's arithmetic.  Both the CUDA path's
tests and the FP64 oracle take their inputs from here.

The paper measures on ChEMBL (483,500 compounds x 5,775 targets, ~1.02M IC50
values) and MovieLens ml-20m (138,493 users x 27,278 movies, 20M ratings)
(Sec. 5.2).  Neither dataset is available here; the planted-factor problems
below stand in for them:

  config 1  1,000 x 500, 20,000 train + 2,000 test at uniform distinct
            positions, planted rank-10 factors, Gaussian noise sd 0.5, K = 10.
  config 2  200,000 x 5,000, 2,000,000 entries, row degrees Zipf(2.0)
            truncated to [1, 5000] and rescaled to the total, column weights
            Zipf(1.5) (heavy-tailed, ChEMBL-like), planted rank-32 signal +
            N(0,1) noise mapped to mean 6, sd 1.5, K = 32, 1% held out.
  config 3  480,000 x 18,000, 100,000,000 entries, row degrees log-normal
            (mu 4.5, sigma 1.2) rescaled to the total, column weights Zipf(1.2),
            integer ratings 1..5 = round(3 + planted rank-64 score + N(0,0.8^2)),
            K = 64, 1% held out (MovieLens-like, above ml-20m's size).

Planted factor entries have variance 1/sqrt(K), so the planted score u.v has
unit variance.  Positions inside a row are distinct; columns are drawn with
probability proportional to the column weights (Chung-Lu style).
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess

import numpy as np


@dataclasses.dataclass
class Problem:
    name: str
    M: int
    N: int
    K: int
    csr_ptr: np.ndarray  # int64, M + 1
    csr_col: np.ndarray  # int32, nnz, increasing inside each row
    csr_val: np.ndarray  # float32, nnz
    test_i: np.ndarray   # int32, T
    test_j: np.ndarray   # int32, T
    test_r: np.ndarray   # float32, T
    alpha: float
    seed: int
    burn_in: int
    sweeps: int
    noise_sd: float = float("nan")

    @property
    def nnz(self) -> int:
        return int(self.csr_ptr[-1])

    @property
    def T(self) -> int:
        return int(len(self.test_i))

    def degrees(self) -> np.ndarray:
        return np.diff(self.csr_ptr)

    def col_degrees(self) -> np.ndarray:
        return np.bincount(self.csr_col, minlength=self.N)

    def csc(self):
        """Column-major copy of the training entries (index transposition only)."""
        rows = np.repeat(np.arange(self.M, dtype=np.int32), self.degrees())
        order = np.argsort(self.csr_col, kind="stable")
        ptr = np.zeros(self.N + 1, dtype=np.int64)
        np.cumsum(np.bincount(self.csr_col, minlength=self.N), out=ptr[1:])
        return ptr, rows[order].astype(np.int32), self.csr_val[order].astype(np.float32)


def _planted(rng, n, K):
    return rng.standard_normal((n, K)) * (K ** -0.25)


def _dot_rows(U, V, rows, cols, chunk=1 << 20):
    out = np.empty(len(rows), dtype=np.float64)
    for a in range(0, len(rows), chunk):
        b = min(a + chunk, len(rows))
        out[a:b] = np.einsum("ij,ij->i", U[rows[a:b]], V[cols[a:b]])
    return out


def _csr_from_pairs(M, rows, cols, vals):
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    ptr = np.zeros(M + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=M), out=ptr[1:])
    return ptr, cols.astype(np.int32), vals.astype(np.float32)


def _cap_weights(w, total, max_col_deg, rounds=8):
    """Clip heavy-tailed column weights so that no column's expected degree
    total * w_j / sum(w) exceeds `max_col_deg`."""
    w = np.asarray(w, dtype=np.float64).copy()
    for _ in range(rounds):
        cap = max_col_deg * w.sum() / total
        if w.max() <= cap:
            break
        np.minimum(w, cap, out=w)
    return w


_HERE = os.path.dirname(os.path.abspath(__file__))
_GEN_SRC = os.path.join(_HERE, "_gen.c")
_GEN_LIB = os.path.join(_HERE, "libgen.so")
_gen = None


def build(force: bool = False) -> str:
    """Compile the C pattern generator next to its source (plain gcc)."""
    if force or not os.path.exists(_GEN_LIB) or \
            os.path.getmtime(_GEN_LIB) < os.path.getmtime(_GEN_SRC):
        tmp = _GEN_LIB + ".tmp%d" % os.getpid()
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", _GEN_SRC,
                        "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _GEN_LIB)
    return _GEN_LIB


def _genlib():
    global _gen
    if _gen is None:
        L = C.CDLL(build())
        L.gen_columns.argtypes = [C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_double, C.c_uint64, C.c_int, C.c_void_p]
        L.gen_planted_scores.argtypes = [C.c_int64, C.c_int64, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
        _gen = L
    return _gen


def _threads():
    return max(1, min(32, os.cpu_count() or 1))


def _pattern(seed, deg, weights, N, big_frac=0.1):
    """CSR pattern (ptr, col) with min(deg_i, N) distinct columns per row drawn
    with probability proportional to `weights`, columns increasing per row."""
    M = len(deg)
    deg = np.ascontiguousarray(np.minimum(deg, N), dtype=np.int64)
    w = np.ascontiguousarray(weights, dtype=np.float64)
    ptr = np.zeros(M + 1, dtype=np.int64)
    np.cumsum(deg, out=ptr[1:])
    col = np.empty(int(ptr[-1]), dtype=np.int32)
    rc = _genlib().gen_columns(M, N, deg.ctypes.data, ptr.ctypes.data, w.ctypes.data,
                               float(big_frac), int(seed) & ((1 << 64) - 1), _threads(),
                               col.ctypes.data)
    if rc != 0:
        raise MemoryError("pattern generator failed")
    return ptr, col


def _scores(ptr, col, U, V):
    U = np.ascontiguousarray(U, dtype=np.float64)
    V = np.ascontiguousarray(V, dtype=np.float64)
    out = np.empty(len(col), dtype=np.float64)
    _genlib().gen_planted_scores(len(ptr) - 1, U.shape[1], ptr.ctypes.data, col.ctypes.data,
                                 U.ctypes.data, V.ctypes.data, _threads(), out.ctypes.data)
    return out


def _split_csr(rng, M, ptr, col, val, frac, name, N, K, alpha, seed, burn_in, sweeps, noise):
    """Hold out a uniform `frac` of the entries; the rest stays in CSR order."""
    nnz = len(col)
    n_test = int(round(frac * nnz))
    test_idx = np.sort(rng.choice(nnz, size=n_test, replace=False))
    keep = np.ones(nnz, dtype=bool)
    keep[test_idx] = False
    rows_of = np.repeat(np.arange(M, dtype=np.int32), np.diff(ptr))
    new_ptr = np.zeros(M + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows_of[keep], minlength=M), out=new_ptr[1:])
    return Problem(name=name, M=M, N=N, K=K, csr_ptr=new_ptr, csr_col=col[keep],
                   csr_val=val[keep].astype(np.float32), test_i=rows_of[test_idx],
                   test_j=col[test_idx].astype(np.int32),
                   test_r=val[test_idx].astype(np.float32), alpha=float(alpha), seed=int(seed),
                   burn_in=int(burn_in), sweeps=int(sweeps), noise_sd=float(noise))


def _rescale_degrees(rng, d, total, lo, hi):
    d = d.astype(np.float64) * (total / d.sum())
    fl = np.floor(d)
    d = fl + (rng.random(len(d)) < (d - fl))
    return np.clip(d, lo, hi).astype(np.int64)


def _split_test(rng, rows, cols, vals, frac):
    n = len(rows)
    n_test = int(round(frac * n))
    perm = rng.permutation(n)
    te, tr = perm[:n_test], np.sort(perm[n_test:])
    return (rows[tr], cols[tr], vals[tr]), (rows[te], cols[te], vals[te])


def _assemble(name, M, N, K, train, test, alpha, seed, burn_in, sweeps, noise_sd):
    ptr, col, val = _csr_from_pairs(M, *train)
    return Problem(name=name, M=M, N=N, K=K, csr_ptr=ptr, csr_col=col, csr_val=val,
                   test_i=test[0].astype(np.int32), test_j=test[1].astype(np.int32),
                   test_r=test[2].astype(np.float32), alpha=float(alpha), seed=int(seed),
                   burn_in=int(burn_in), sweeps=int(sweeps), noise_sd=float(noise_sd))


def config1(seed: int = 0) -> Problem:
    """1,000 x 500, K = 10: 20,000 train + 2,000 test at distinct uniform positions."""
    M, N, K = 1000, 500, 10
    rng = np.random.default_rng(seed)
    pos = rng.choice(M * N, size=22000, replace=False)
    rows, cols = pos // N, pos % N
    U, V = _planted(rng, M, K), _planted(rng, N, K)
    vals = _dot_rows(U, V, rows, cols) + 0.5 * rng.standard_normal(len(rows))
    train = (rows[:20000], cols[:20000], vals[:20000])
    test = (rows[20000:], cols[20000:], vals[20000:])
    return _assemble("config1_1000x500_K10", M, N, K, train, test, alpha=4.0, seed=seed,
                     burn_in=50, sweeps=200, noise_sd=0.5)


def _truncated_zipf(rng, s, n, hi):
    out = rng.zipf(s, n)
    bad = out > hi
    while bad.any():
        out[bad] = rng.zipf(s, int(bad.sum()))
        bad = out > hi
    return out


def config2(seed: int = 1, scale: float = 1.0) -> Problem:
    """200,000 x 5,000, 2M entries, Zipf(2.0) rows / Zipf(1.5) columns, K = 32."""
    M, N, K = int(200_000 * scale), 5000, 32
    total = int(2_000_000 * scale)
    rng = np.random.default_rng(seed)
    deg = _truncated_zipf(rng, 2.0, M, 5000)
    deg = _rescale_degrees(rng, deg, total, 1, min(5000, N))
    w = _cap_weights(rng.zipf(1.5, N), total, 0.5 * M)
    ptr, col = _pattern(seed * 1000003 + 11, deg, w, N)
    U, V = _planted(rng, M, K), _planted(rng, N, K)
    s = _scores(ptr, col, U, V) + rng.standard_normal(len(col))
    vals = 6.0 + 1.5 * (s - s.mean()) / s.std()
    return _split_csr(rng, M, ptr, col, vals, 0.01, "config2_200kx5k_K32", N, K, 2.0, seed, 25,
                      100, 1.5 / np.sqrt(2.0))


def config3(seed: int = 2, scale: float = 1.0) -> Problem:
    """480,000 x 18,000, 1e8 entries, log-normal rows / Zipf(1.2) columns, ratings 1..5, K = 64."""
    M, N, K = int(480_000 * scale), 18_000, 64
    total = int(100_000_000 * scale)
    rng = np.random.default_rng(seed)
    deg = rng.lognormal(4.5, 1.2, M)
    deg = _rescale_degrees(rng, deg, total, 1, N)
    w = _cap_weights(rng.zipf(1.2, N), total, 0.5 * M)
    ptr, col = _pattern(seed * 1000003 + 13, deg, w, N)
    U, V = _planted(rng, M, K), _planted(rng, N, K)
    s = _scores(ptr, col, U, V)
    s += 0.8 * rng.standard_normal(len(col))
    vals = np.clip(np.rint(3.0 + s), 1.0, 5.0).astype(np.float32)
    del s
    return _split_csr(rng, M, ptr, col, vals, 0.01, "config3_480kx18k_K64", N, K, 2.0, seed, 12,
                      50, 0.8)


def planted_dense(M=300, N=200, K=4, density=0.4, sigma=0.5, seed=7, test_frac=0.1) -> Problem:
    """Small dense planted low-rank problem (for convergence to the noise floor)."""
    rng = np.random.default_rng(seed)
    n = int(density * M * N)
    pos = rng.choice(M * N, size=n, replace=False)
    rows, cols = pos // N, pos % N
    U, V = _planted(rng, M, K), _planted(rng, N, K)
    vals = _dot_rows(U, V, rows, cols) + sigma * rng.standard_normal(n)
    train, test = _split_test(rng, rows, cols, vals, test_frac)
    return _assemble("planted_%dx%d_K%d" % (M, N, K), M, N, K, train, test, alpha=1.0 / sigma**2,
                     seed=seed, burn_in=20, sweeps=80, noise_sd=sigma)


def random_small(M, N, K, nnz, seed, n_test=0, empty_rows=0, empty_cols=0, alpha=2.0,
                 long_rows=0, long_deg=0) -> Problem:
    """Uniform random sparse problem with optional empty rows/columns and a few long rows.

    Used for edge cases: degree-0 rows, ragged tails, rows longer than one tile.
    """
    rng = np.random.default_rng(seed)
    live_r = np.arange(empty_rows, M)
    live_c = np.arange(empty_cols, N)
    rr = rng.choice(live_r, size=nnz)
    cc = rng.choice(live_c, size=nnz)
    if long_rows:
        lr = rng.choice(live_r, size=long_rows, replace=False)
        d = min(long_deg, len(live_c))
        rr = np.concatenate([rr, np.repeat(lr, d)])
        cc = np.concatenate([cc] + [rng.choice(live_c, size=d, replace=False) for _ in lr])
    key = np.unique(rr.astype(np.int64) * N + cc)
    rows, cols = key // N, key % N
    U, V = _planted(rng, M, K), _planted(rng, N, K)
    vals = _dot_rows(U, V, rows, cols) + 0.3 * rng.standard_normal(len(rows))
    ti = rng.integers(0, M, n_test)
    tj = rng.integers(0, N, n_test)
    tv = _dot_rows(U, V, ti, tj) + 0.3 * rng.standard_normal(n_test)
    return _assemble("random_%dx%d_K%d" % (M, N, K), M, N, K, (rows, cols, vals), (ti, tj, tv),
                     alpha=alpha, seed=seed, burn_in=0, sweeps=4, noise_sd=0.3)


def fixed_degree(M: int, N: int, K: int, d: int, seed: int = 0) -> Problem:
    """Every row with exactly d ratings (columns (o_r + s k) mod N for k < d, with a random
    offset o_r per row and a stride s coprime to N, so they are distinct), planted values
    plus noise, no test set.  For per-row cost against degree (the paper's Fig. 3)."""
    if d > N:
        raise ValueError("degree above the column count")
    rng = np.random.default_rng(seed)
    s = 1 + 2 * int(rng.integers(0, N // 2))
    while np.gcd(s, N) != 1:
        s += 2
    off = rng.integers(0, N, M)
    cols = (off[:, None] + s * np.arange(d)[None, :]) % N
    rows = np.repeat(np.arange(M), d)
    U, V = _planted(rng, M, K), _planted(rng, N, K)
    vals = _dot_rows(U, V, rows, cols.ravel()) + 0.3 * rng.standard_normal(M * d)
    empty = np.zeros(0, np.int64)
    return _assemble("fixed_degree_%d_%dx%d_K%d" % (d, M, N, K), M, N, K,
                     (rows, cols.ravel(), vals), (empty, empty, np.zeros(0)), alpha=2.0,
                     seed=seed, burn_in=0, sweeps=1, noise_sd=0.3)


def config4(seed: int = 3, n_jobs: int = 256) -> list:
    """Many independent small jobs (batched form): per job M log-uniform in
    [1,000, 100,000], N log-uniform in [500, 10,000], density log-uniform in
    [0.1%, 2%], K drawn from {16, 32, 64}, planted Gaussian ratings (noise sd 0.3),
    1% of the ratings' count as test points.  Job j is seeded with 1000 seed + j."""
    rng = np.random.default_rng(seed)
    return [config4_job(rng, 1000 * seed + j) for j in range(n_jobs)]


def config4_job(rng, seed: int) -> Problem:
    """One job drawn from the distribution of config4: sizes, density and K from `rng`,
    the ratings from `seed`."""
    M = int(round(np.exp(rng.uniform(np.log(1e3), np.log(1e5)))))
    N = int(round(np.exp(rng.uniform(np.log(500.0), np.log(1e4)))))
    dens = float(np.exp(rng.uniform(np.log(1e-3), np.log(2e-2))))
    K = int(rng.choice([16, 32, 64]))
    nnz = max(1, int(dens * M * N))
    return random_small(M, N, K, nnz, seed=seed, n_test=max(1, nnz // 100))


def subsample_rows(prob: Problem, n_rows: int, seed: int = 123) -> Problem:
    """Stand-alone problem made of `n_rows` rows chosen by a seeded permutation.

    Each chosen row keeps all of its ratings; all N columns are kept (some may end
    up empty); test entries are those whose row was chosen.
    """
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.permutation(prob.M)[:n_rows])
    deg = prob.degrees()
    new_ptr = np.zeros(n_rows + 1, dtype=np.int64)
    np.cumsum(deg[pick], out=new_ptr[1:])
    starts = prob.csr_ptr[pick]
    idx = np.concatenate([np.arange(s, s + d) for s, d in zip(starts, deg[pick])]) \
        if n_rows else np.zeros(0, dtype=np.int64)
    remap = -np.ones(prob.M, dtype=np.int64)
    remap[pick] = np.arange(n_rows)
    keep = remap[prob.test_i] >= 0
    return Problem(name=prob.name + "_sub%d" % n_rows, M=n_rows, N=prob.N, K=prob.K,
                   csr_ptr=new_ptr, csr_col=prob.csr_col[idx].astype(np.int32),
                   csr_val=prob.csr_val[idx].astype(np.float32),
                   test_i=remap[prob.test_i[keep]].astype(np.int32),
                   test_j=prob.test_j[keep].astype(np.int32),
                   test_r=prob.test_r[keep].astype(np.float32), alpha=prob.alpha, seed=prob.seed,
                   burn_in=prob.burn_in, sweeps=prob.sweeps, noise_sd=prob.noise_sd)


CONFIGS = {1: config1, 2: config2, 3: config3}
