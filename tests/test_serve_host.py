"""Scheduling logic of the serving loop against a fake device backend (no GPU):
memory-budget admission in arrival order, continuous batching (jobs admitted as
others retire), every job swept exactly its number of sweeps, futures resolved."""
import threading
import time
from types import SimpleNamespace

import numpy as np
import pytest

from paper_1705_10633_gb300.serve import Job, Server, estimate_bytes, latency_percentiles


class FakeBackend:
    def __init__(self, delay=0.002):
        self.delay = delay
        self.lock = threading.Lock()
        self.swept = {}
        self.active = set()
        self.max_active = 0
        self.order = []
        self.created = 0

    def create(self, job):
        with self.lock:
            self.created += 1
            h = {"id": job.seed, "bytes": estimate_bytes(job.problem)}
            self.active.add(job.seed)
            self.max_active = max(self.max_active, len(self.active))
            self.order.append(job.seed)
            self.swept[job.seed] = 0
        return h

    def sweep_batch(self, handles, n):
        time.sleep(self.delay)
        with self.lock:
            for h in handles:
                self.swept[h["id"]] += n

    def mark(self, handle):
        return handle["id"]

    def wait(self, marks):
        pass

    def finish(self, handle, job):
        return np.full(len(job.query_i), float(job.seed), np.float32), 1.0, 0.5

    def bytes(self, handle):
        return handle["bytes"]

    def destroy(self, handle):
        with self.lock:
            self.active.discard(handle["id"])


def _job(seed, M=1000, N=500, K=16, nnz=20000, sweeps=7):
    prob = SimpleNamespace(M=M, N=N, K=K, nnz=nnz, test_i=np.zeros(10, np.int32))
    q = np.arange(5, dtype=np.int32)
    return Job(problem=prob, sweeps=sweeps, query_i=q, query_j=q, seed=seed)


def test_memory_budget_and_arrival_order():
    be = FakeBackend()
    one = estimate_bytes(_job(0).problem)
    srv = Server(memory_limit=2.5 * one, max_active=64, sweeps_per_round=3, backend=be)
    futs = [srv.submit(_job(s)) for s in range(1, 9)]
    res = [f.result(timeout=30) for f in futs]
    srv.close()
    assert be.max_active == 2                      # 2.5 jobs' worth of memory
    assert be.order == list(range(1, 9))           # admitted in arrival order
    assert all(be.swept[s] == 7 for s in range(1, 9))
    assert [float(r.predictions[0]) for r in res] == [float(s) for s in range(1, 9)]
    assert srv.memory_in_use == 0 and srv.peak_memory <= 2.5 * one
    # only the head of the queue is counted, once, while the budget holds it back
    assert 1 <= srv.memory_waits <= 6 and not srv._mem_blocked
    assert all(r.finished_at >= r.admitted_at >= r.submitted_at for r in res)
    lat = latency_percentiles(res)
    assert 0 <= lat["p50"] <= lat["p99"]


def test_slots_and_late_arrivals_are_admitted():
    be = FakeBackend(delay=0.005)
    srv = Server(memory_limit=1e12, max_active=3, sweeps_per_round=2, backend=be)
    first = [srv.submit(_job(s, sweeps=6)) for s in range(1, 5)]
    time.sleep(0.02)
    late = [srv.submit(_job(s, sweeps=2)) for s in range(5, 8)]
    for f in first + late:
        f.result(timeout=30)
    srv.close()
    assert be.max_active == 3
    assert all(be.swept[s] == (6 if s < 5 else 2) for s in range(1, 8))
    assert srv.rounds >= 4


def test_job_larger_than_budget_fails_alone():
    be = FakeBackend()
    srv = Server(memory_limit=8e6, backend=be)
    big = srv.submit(_job(1, M=100000, N=10000, nnz=10**7))
    small = srv.submit(_job(2, M=10, N=10, nnz=20))
    with pytest.raises(MemoryError):
        big.result(timeout=30)
    assert small.result(timeout=30).predictions[0] == 2.0
    srv.close()


def test_closed_server_rejects_jobs():
    srv = Server(backend=FakeBackend())
    srv.close()
    with pytest.raises(RuntimeError):
        srv.submit(_job(1))


def test_cancel_queued_and_running_jobs():
    import concurrent.futures as cf
    be = FakeBackend(delay=0.01)
    srv = Server(memory_limit=1e12, max_active=1, sweeps_per_round=1, backend=be)
    try:
        running = srv.submit(_job(1, sweeps=10_000))  # admitted, ~100 s of rounds
        queued = srv.submit(_job(2))                   # waits for the only slot
        deadline = time.time() + 5
        while be.created < 1 and time.time() < deadline:
            time.sleep(0.005)
        assert be.created == 1
        assert srv.cancel(queued) and queued.cancelled()
        assert srv.cancel(running)
        with pytest.raises(cf.CancelledError):
            running.result(timeout=5)
        later = srv.submit(_job(3, sweeps=3))
        assert later.result(timeout=5).predictions[0] == 3.0
        assert not srv.cancel(later)  # already finished
    finally:
        srv.close()
    assert be.order == [1, 3]          # the cancelled queued job was never created
    assert be.active == set() and srv.memory_in_use == 0
    assert be.swept[1] < 10_000
