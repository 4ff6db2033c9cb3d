"""Sharded Gibbs sweeps: one process per GPU, each updating a slice of the rows.

The paper spreads the items over nodes by a per-item cost of a fixed part plus a part
per rating (Sec. 4.2) and, after each half-sweep, sends the updated items to the nodes
that need them (Sec. 4.3).  Here every rank owns one contiguous, cost-balanced range
of the rows of each side, updates only those in its row phases, and after each row
phase the ranks all-gather the updated ranges so that every rank again holds the
whole side.  The hyper step then runs on every rank over the whole side, and the
prediction step over every test point: both see the same data on every rank, so
they need no collective of their own.  A row's update depends only on the other
side, its side's hyper-parameters and (seed, sweep, row), so the sharded chain is,
bit for bit, the chain of one handle over all rows.

The exchange is the only collective: `torch.distributed.all_gather` of each rank's
range, padded to the longest range (NCCL on device buffers, or gloo on host copies).
The driver is written against a small backend interface so that the partition and
the exchange can be exercised without a GPU:

    backend.rows(side) -> int                    rows of U (0) or V (1)
    backend.degrees(side) -> array               ratings per row
    backend.set_shard(side, lo, hi)              restrict the row phase
    backend.hyper(side); backend.rows_phase(side); backend.predict(); backend.advance()
    backend.get_rows(side, lo, hi) -> tensor     n x K, on the exchange's device
    backend.put_rows(side, lo, hi, tensor)
"""
from __future__ import annotations

import numpy as np

USER, MOVIE = 0, 1
# the per-item cost of Sec. 4.2, c0 + c1 d, in 64-rating stages of the row kernels: a
# row costs its stages plus a fixed part for the factorisation and the solves
COST_FIXED = 2.0
COST_PER_RATING = 1.0 / 64.0


def cost_balanced_ranges(degrees, world, c0=COST_FIXED, c1=COST_PER_RATING):
    """Contiguous ranges [(lo, hi)] of the rows, one per rank, tiling [0, rows), each
    holding about 1 / world of the total cost c0 + c1 d: range r ends at the first row
    where the prefix cost reaches (r + 1) / world of the total."""
    d = np.asarray(degrees, dtype=np.float64)
    n = len(d)
    world = int(world)
    if world < 1:
        raise ValueError("world must be >= 1")
    cost = np.cumsum(c0 + c1 * d)
    total = cost[-1] if n else 0.0
    bounds = [0]
    for r in range(1, world):
        b = int(np.searchsorted(cost, total * r / world, side="left")) + 1 if n else 0
        bounds.append(min(max(b, bounds[-1]), n))
    bounds.append(n)
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


class ShardedChain:
    """Drives a backend through sharded sweeps (Alg. 1's order: movies first by default)."""

    def __init__(self, backend, rank, world, group=None, order=0):
        self.b = backend
        self.rank, self.world, self.group = int(rank), int(world), group
        self.order = order
        self.ranges = {s: cost_balanced_ranges(backend.degrees(s), world) for s in (USER, MOVIE)}
        for s in (USER, MOVIE):
            lo, hi = self.ranges[s][self.rank]
            backend.set_shard(s, lo, hi)

    def exchange(self, side):
        """All-gather the rows each rank updated, so every rank holds the whole side."""
        import torch
        import torch.distributed as dist
        lo, hi = self.ranges[side][self.rank]
        mine = self.b.get_rows(side, lo, hi)
        if self.world == 1:
            return
        width = max(h - l for l, h in self.ranges[side])
        padded = torch.zeros((width, mine.shape[1]), dtype=mine.dtype, device=mine.device)
        padded[: hi - lo] = mine
        parts = [torch.empty_like(padded) for _ in range(self.world)]
        dist.all_gather(parts, padded, group=self.group)
        for r, (l, h) in enumerate(self.ranges[side]):
            if r != self.rank and h > l:
                self.b.put_rows(side, l, h, parts[r][: h - l])

    def sweep(self, n=1):
        first = MOVIE if self.order == 0 else USER
        for _ in range(int(n)):
            for side in (first, 1 - first):
                self.b.hyper(side)
                self.b.rows_phase(side)
                self.exchange(side)
            self.b.predict()
            self.b.advance()


class HandleBackend:
    """A chain of the GPU library as a sharding backend.  device=True exchanges device
    buffers (for NCCL); device=False exchanges host copies (for gloo)."""

    def __init__(self, bp, h, M, N, K, degrees_u, degrees_v, device=True):
        self.bp, self.h, self.K = bp, h, int(K)
        self.n = {USER: int(M), MOVIE: int(N)}
        self.deg = {USER: np.asarray(degrees_u), MOVIE: np.asarray(degrees_v)}
        self.device = device

    def rows(self, side):
        return self.n[side]

    def degrees(self, side):
        return self.deg[side]

    def set_shard(self, side, lo, hi):
        self.bp.bpmf_set_shard(self.h, side, lo, hi)

    def hyper(self, side):
        self.bp.bpmf_step(self.h, self.bp.BPMF_PHASE_HYPER_USER if side == USER
                          else self.bp.BPMF_PHASE_HYPER_MOVIE)

    def rows_phase(self, side):
        self.bp.bpmf_step(self.h, self.bp.BPMF_PHASE_ROWS_USER if side == USER
                          else self.bp.BPMF_PHASE_ROWS_MOVIE)

    def predict(self):
        self.bp.bpmf_step(self.h, self.bp.BPMF_PHASE_PREDICT)

    def advance(self):
        self.bp.bpmf_step(self.h, self.bp.BPMF_PHASE_ADVANCE)

    def get_rows(self, side, lo, hi):
        import torch
        if self.device:
            # ordered on the handle's stream; the caller's collective runs on torch's
            # current stream, which the handle was created on
            out = torch.empty((hi - lo, self.K), dtype=torch.float32, device="cuda")
            if hi > lo:
                self.bp.bpmf_get_rows(self.h, side, lo, hi, self.K, out_ptr=out.data_ptr())
            return out
        return torch.from_numpy(self.bp.bpmf_get_rows(self.h, side, lo, hi, self.K))

    def put_rows(self, side, lo, hi, rows):
        if self.device:
            rows = rows.contiguous()
            self.bp.bpmf_put_rows(self.h, side, lo, hi, in_ptr=rows.data_ptr())
        else:
            self.bp.bpmf_put_rows(self.h, side, lo, hi, rows=rows.numpy())
