"""Autotuner for the row kernels' thresholds, on a job's own data.

The thresholds are the degree from which a row takes the tensor-core route
(below it, the CUDA-core warp-per-row kernel), the degree from which a CUDA-core
row is split into segments done by separate warps, and the degree below which a
CUDA-core row takes the rank-one route (Sec. 3.1; the GPU analogue of the paper's
measured crossover between its per-item methods, Sec. 3.2).  At K in 49..64 the
first is tuned (the CUDA-core kernel then holds few rows); below that the split
degree is tuned first and the rank-one degree second, at the best split.  Each candidate
is applied to the live handle (`bpmf_set_tuning` bins and splits the rows again),
the two row phases are run and timed with CUDA events on the handle's stream, and
the fastest candidate is kept.  The chain's factors, hyper-parameters and sweep
counter are saved first and restored after every trial, so tuning does not move
the chain (the row phases do not touch the running prediction sums).
"""
from __future__ import annotations

import json
import os

import numpy as np

LONG_MIN_CANDIDATES = (1, 16, 24, 48, 128)
SPLIT_CANDIDATES = (128, 512, 1024, 4096, 1 << 30)
RANK_ONE_CANDIDATES = (-1, 2, 4)


def tuning_key(K, deg_users, deg_movies, device):
    """Cache key of a job for its tuning: K padded to the kernels' width, the device name,
    and for each side the power-of-two buckets of its degree quantiles 0.5, 0.9 and 0.99,
    with the side's size to an order of magnitude -- jobs whose rows bin alike tune alike
    (a quantile on a bucket's edge can split resamples of one distribution)."""
    def shape(d):
        d = np.maximum(np.asarray(d, dtype=np.float64), 1.0)
        return [int(np.floor(np.log2(q))) for q in np.quantile(d, [0.5, 0.9, 0.99])]

    return json.dumps({"kp": (int(K) + 15) // 16 * 16, "device": str(device),
                       "users": shape(deg_users), "movies": shape(deg_movies),
                       "size": [len(str(len(deg_users))), len(str(len(deg_movies)))]},
                      sort_keys=True)


class TuningCache:
    """Tunings by `tuning_key`, kept in a JSON file (written on every store)."""

    def __init__(self, path):
        self.path = path
        self.entries = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.entries = {k: tuple(v) for k, v in json.load(f).items()}

    def get(self, key):
        return self.entries.get(key)

    def put(self, key, tuning):
        self.entries[key] = tuple(int(x) for x in tuning)
        if self.path:
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump({k: list(v) for k, v in self.entries.items()}, f, indent=1)
            os.replace(tmp, self.path)


def autotune(h, M, N, K, stream, long_min=LONG_MIN_CANDIDATES, split=SPLIT_CANDIDATES,
             rank_one=RANK_ONE_CANDIDATES, reps=2, cache=None, degrees=None):
    """Returns ((long_min_degree, split_degree, rank_one_degree),
    {tuple: ms for one pass of both row phases}).  `stream` is the raw cudaStream_t the
    handle was created with.  0 in a tuple is the library default.  With a `TuningCache`
    and the job's `degrees` (users', movies'), a cached tuning for the same key is applied
    without trials (the dict is then empty) and a new one is stored."""
    import torch

    import paper_1705_10633_gb300 as bp

    key = None
    if cache is not None and degrees is not None:
        key = tuning_key(K, degrees[0], degrees[1], torch.cuda.get_device_name())
        hit = cache.get(key)
        if hit is not None:
            bp.bpmf_set_tuning(h, *hit)
            return tuple(hit), {}

    st = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()
    U, V, hyper, sweep = bp.bpmf_get_state(h, M, N, K)
    rows = (bp.BPMF_PHASE_ROWS_MOVIE, bp.BPMF_PHASE_ROWS_USER)
    times = {}

    def trial(cand):
        bp.bpmf_set_tuning(h, *cand)
        for ph in rows:  # warm-up: launch shapes, caches
            bp.bpmf_step(h, ph)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            for ph in rows:
                bp.bpmf_step(h, ph)
        e1.record(st)
        e1.synchronize()
        times[cand] = e0.elapsed_time(e1) / reps
        bp.bpmf_set_state(h, U, V, hyper, sweep)

    try:
        if (K + 15) // 16 * 16 == 64:
            for lm in long_min:
                trial((lm, 0, 0))
        else:
            for sp in split:
                trial((0, sp, 0))
            sp = min(times, key=times.get)[1]
            for r1 in rank_one:
                if (0, sp, r1) not in times:
                    trial((0, sp, r1))
        best = min(times, key=times.get)
        bp.bpmf_set_tuning(h, *best)
    finally:
        bp.bpmf_set_state(h, U, V, hyper, sweep)
    if key is not None:
        cache.put(key, best)
    return best, times
