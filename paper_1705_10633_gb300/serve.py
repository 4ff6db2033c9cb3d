"""Serving loop: continuous batching of independent BPMF jobs on one GPU.

A job is a ratings matrix, a number of Gibbs sweeps and a set of query points.
`Server.submit(job)` returns a future; a scheduler thread admits queued jobs in
arrival order while their device memory fits the budget and a slot is free,
keeps every admitted chain resident (U, V, hyper-parameters and counters live in
its handle), and runs rounds: each active job gets a few more sweeps, all of
them issued together with `bpmf_sweep_batch` (one stream per job, so their work
overlaps on the device; sweeps inside a round replay the handle's CUDA graph).
A job that has all its sweeps is answered (predictions of the current sample at
its query points, RMSEs), its handle destroyed and its memory returned; jobs
that arrive meanwhile are admitted at the next round boundary.

The device work goes through a backend object so that the scheduling logic can
run against a fake backend on a machine without a GPU.
"""
from __future__ import annotations

import concurrent.futures as cf
import threading
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Job:
    """One factorisation job.  `problem` carries M, N, K, the CSR arrays and the
    held-out test set (the fields of a workloads.Problem); queries are (i, j)
    index arrays; seed and flags are the chain's Philox seed and BPMF_* flags."""
    problem: object
    sweeps: int
    query_i: np.ndarray
    query_j: np.ndarray
    seed: int = 0
    flags: int = 0
    burn_in: int | None = None
    submitted_at: float = field(default=0.0)


@dataclass
class JobResult:
    predictions: np.ndarray
    rmse_sample: float
    rmse_avg: float
    submitted_at: float
    admitted_at: float
    finished_at: float

    @property
    def latency(self) -> float:
        return self.finished_at - self.submitted_at


def estimate_bytes(problem) -> int:
    """A rough figure of the device bytes a handle for `problem` needs: ratings twice
    (8-byte pointers, 4-byte index and value), FP32 factors and, at K = 64, their two
    16-bit copies, the test set and its running sums, plus 4 MB of small state.  For
    backends that cannot say better; the device backend asks the library
    (bpmf_device_bytes), which counts every allocation of bpmf_create."""
    kp = (problem.K + 15) // 16 * 16
    rows = problem.M + problem.N
    b = 16 * problem.nnz + 8 * (rows + 2)
    b += 4 * kp * rows * (2 if kp == 64 else 1)
    b += 20 * len(problem.test_i)
    return int(b + (4 << 20))


class DeviceBackend:
    """The library on the current CUDA device: one torch stream per job, device
    memory through PyTorch's caching allocator (no device-wide synchronisation
    when a job is admitted or retired)."""

    def __init__(self):
        import torch

        import paper_1705_10633_gb300 as bp
        self.torch, self.bp = torch, bp
        self.num_sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count

    def _params(self, job: Job):
        p = job.problem
        return self.bp.bpmf_default_params(alpha=p.alpha, seed=job.seed, flags=job.flags,
                                           burn_in=p.burn_in if job.burn_in is None else job.burn_in)

    def estimate(self, job: Job) -> int:
        """The device bytes bpmf_create will hold for this job (exact, host only)."""
        p = job.problem
        return self.bp.bpmf_device_bytes(p.M, p.N, p.K, p.csr_ptr, p.csr_col, len(p.test_i),
                                         params=self._params(job), num_sms=self.num_sms)

    def create(self, job: Job):
        bp, p = self.bp, job.problem
        stream = self.torch.cuda.Stream()
        params = self._params(job)
        keep = bp.torch_allocator(params)
        h = bp.bpmf_create(p.M, p.N, p.K, p.csr_ptr, p.csr_col, p.csr_val, test_i=p.test_i,
                           test_j=p.test_j, test_r=p.test_r, params=params,
                           stream=stream.cuda_stream)
        return {"h": h, "stream": stream, "keep": keep,
                "bytes": bp.bpmf_info(h, 0)["device_bytes"]}

    def sweep_batch(self, handles, n):
        self.bp.bpmf_sweep_batch([x["h"] for x in handles], n)

    def mark(self, handle):
        ev = self.torch.cuda.Event()
        ev.record(handle["stream"])
        return ev

    def wait(self, marks):
        for ev in marks:
            ev.synchronize()

    def finish(self, handle, job: Job):
        bp = self.bp
        rs, ra = bp.bpmf_sweep(handle["h"], 0)
        pred = bp.bpmf_predict(handle["h"], job.query_i, job.query_j)
        return pred, rs, ra

    def bytes(self, handle):
        return handle["bytes"]

    def destroy(self, handle):
        self.bp.bpmf_destroy(handle["h"])


class Server:
    """Continuous batching of jobs.  memory_limit: device bytes the admitted jobs may
    hold together; max_active: jobs resident at once; sweeps_per_round: sweeps each
    active job gets per round (the granularity at which new jobs are admitted)."""

    def __init__(self, memory_limit=150e9, max_active=64, sweeps_per_round=5, backend=None):
        self.memory_limit = float(memory_limit)
        self.max_active = int(max_active)
        self.sweeps_per_round = int(sweeps_per_round)
        self.backend = backend if backend is not None else DeviceBackend()
        self._pending = []  # (job, future, estimate) in arrival order
        self._active = []   # dicts: job, future, handle, left, bytes, admitted_at
        self._cancel = set()  # futures of admitted jobs to drop at the next round boundary
        self._cv = threading.Condition()
        self._closing = False
        self.memory_in_use = 0
        self.peak_memory = 0
        self.rounds = 0
        self.memory_waits = 0      # jobs that waited at the head of the queue for memory
        self._mem_blocked = set()  # their futures, until admitted
        self._thread = threading.Thread(target=self._run, name="bpmf-serve", daemon=True)
        self._thread.start()

    # ---- client side
    def submit(self, job: Job) -> cf.Future:
        fut = cf.Future()
        job.submitted_at = time.perf_counter()
        est = (self.backend.estimate(job) if hasattr(self.backend, "estimate")
               else estimate_bytes(job.problem))
        with self._cv:
            if self._closing:
                raise RuntimeError("server is closed")
            if est > self.memory_limit:
                fut.set_exception(MemoryError("job needs %d bytes, budget %d" % (est, self.memory_limit)))
                return fut
            self._pending.append((job, fut, est))
            self._cv.notify()
        return fut

    def cancel(self, fut) -> bool:
        """Cancel a submitted job: a queued job is dropped at once; an admitted one at the
        next round boundary (no sweep is interrupted), its handle destroyed and its memory
        returned.  The future then raises CancelledError.  False if it already finished."""
        with self._cv:
            if fut.done():
                return False
            for k, (job, f, est) in enumerate(self._pending):
                if f is fut:
                    del self._pending[k]
                    self._mem_blocked.discard(fut)
                    fut.cancel()
                    return True
            if any(a["fut"] is fut for a in self._active):
                self._cancel.add(fut)
                self._cv.notify()
                return True
        return False

    def close(self, wait=True):
        with self._cv:
            self._closing = True
            self._cv.notify()
        if wait:
            self._thread.join()

    # ---- scheduler
    def _admit(self):
        while self._pending and len(self._active) < self.max_active:
            job, fut, est = self._pending[0]
            if self.memory_in_use + est > self.memory_limit:
                if fut not in self._mem_blocked:
                    self._mem_blocked.add(fut)
                    self.memory_waits += 1
                break  # arrival order: a large job waits rather than being overtaken
            self._pending.pop(0)
            self._mem_blocked.discard(fut)
            self.memory_in_use += est
            try:
                handle = self.backend.create(job)
            except Exception as exc:  # the job fails alone
                self.memory_in_use -= est
                fut.set_exception(exc)
                continue
            real = self.backend.bytes(handle)
            self.memory_in_use += real - est
            self.peak_memory = max(self.peak_memory, self.memory_in_use)
            self._active.append({"job": job, "fut": fut, "handle": handle, "left": job.sweeps,
                                 "bytes": real, "admitted_at": time.perf_counter()})

    def _drop_cancelled(self):
        with self._cv:
            drop = [a for a in self._active if a["fut"] in self._cancel]
            self._cancel.clear()
        if not drop:
            return
        self._active = [a for a in self._active if all(a is not d for d in drop)]
        for a in drop:
            try:
                self.backend.destroy(a["handle"])
            finally:
                self.memory_in_use -= a["bytes"]
                a["fut"].cancel()

    def _round(self):
        self._drop_cancelled()
        if not self._active:
            return
        groups = {}
        for a in self._active:
            n = min(self.sweeps_per_round, a["left"])
            if n > 0:
                groups.setdefault(n, []).append(a)
        for n, group in groups.items():
            self.backend.sweep_batch([a["handle"] for a in group], n)
            for a in group:
                a["left"] -= n
        self.backend.wait([self.backend.mark(a["handle"]) for a in self._active])
        self.rounds += 1
        done = [a for a in self._active if a["left"] == 0]
        self._active = [a for a in self._active if a["left"] > 0]
        for a in done:
            try:
                pred, rs, ra = self.backend.finish(a["handle"], a["job"])
                res = JobResult(pred, rs, ra, a["job"].submitted_at, a["admitted_at"],
                                time.perf_counter())
                a["fut"].set_result(res)
            except Exception as exc:
                a["fut"].set_exception(exc)
            finally:
                self.backend.destroy(a["handle"])
                self.memory_in_use -= a["bytes"]

    def _run(self):
        while True:
            with self._cv:
                while not self._pending and not self._active and not self._closing:
                    self._cv.wait()
                if self._closing and not self._pending and not self._active:
                    return
                self._admit()
            if self._active:
                try:
                    self._round()
                except Exception as exc:  # a device error ends the jobs in flight, not the server
                    failed, self._active = self._active, []
                    for a in failed:
                        if not a["fut"].done():
                            a["fut"].set_exception(exc)
                        try:
                            self.backend.destroy(a["handle"])
                        finally:
                            self.memory_in_use -= a["bytes"]


def latency_percentiles(results, qs=(50, 99)):
    lat = np.array([r.latency for r in results])
    return {"p%d" % q: float(np.percentile(lat, q)) for q in qs}


def queue_wait_percentiles(results, qs=(50, 99)):
    """Percentiles of the time each job spent queued before admission."""
    w = np.array([r.admitted_at - r.submitted_at for r in results])
    return {"p%d" % q: float(np.percentile(w, q)) for q in qs}
