#!/usr/bin/env python
"""Throughput of the GB300 BPMF Gibbs sampler: latent rows sampled per second.

One step = one full Gibbs sweep of Alg. 1 (hyper(V), every movie, hyper(U),
every user, test predictions + RMSE) over the 480,000 x 18,000 rating matrix
with 1e8 ratings at K = 64 (synthetic, seeded; ``workloads.config3``).
value = (M + N) x sweeps / device time of the slowest rank.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Under torchrun (N > 1) the ranks run one chain together: each rank updates a cost-
balanced range of the rows of both sides and the ranks all-gather the updated rows
after every half-sweep (NCCL), so the total work is fixed and scaling is strong.
``--impl reference`` times the FP64 CPU oracle on bounded blocks of the same
workload on the host cores (rank 0 only) and prints the same metric.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "latent rows sampled/s (Gibbs sweep, K=%d)"
# the cpu_baseline leg: this many oracle steps of the reference arm's kind (about 10 s of
# 16 host cores on the 480k x 18k workload)
CPU_BASELINE_STEPS = 2
UNIT = "rows/s"


# ----------------------------------------------------------------------------
# distributed plumbing (host only)
# ----------------------------------------------------------------------------
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def dist_init(world, backend):
    if world <= 1:
        return
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group(backend=backend)


def barrier(world, device=None):
    if world > 1:
        import torch.distributed as dist
        if device is not None and dist.get_backend() == "nccl":
            dist.barrier(device_ids=[device])
        else:
            dist.barrier()


def reduce_over_ranks(x, world, op="max", device=None):
    """Max (or sum) of a float over all ranks; identity for one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64,
                     device=device if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def aggregate_rows_per_s(rows_per_rank, sweeps, max_ms):
    """Whole-job throughput: units of all ranks over the slowest rank's time."""
    return rows_per_rank * sweeps / (max_ms / 1e3)


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = str(index)
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.index, "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm, mx, reasons = [], [], set()
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 8:
                    continue
                try:
                    sm.append(float(f[0]))
                    mx.append(float(f[1]))
                except ValueError:
                    continue
                for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                    "sw_power_cap"), f[4:8]):
                    if v.lower() == "active":
                        reasons.add(name)
            os.unlink(self.path)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------
# algorithmic work per phase
# ----------------------------------------------------------------------------
def row_alu_flops(rows, K):
    """CUDA-core work per row: Cholesky K^3/3, forward and back substitution K^2
    each, the prior terms and noise add (O(K), ignored)."""
    return rows * (K**3 / 3.0 + 2.0 * K * K)


def row_gram_flops(nnz, K):
    """Tensor-core work per rating: the full K x K Gram tile 2K^2 (the symmetric
    half is K(K+1)) and the right-hand side 2K."""
    return nnz * (2.0 * K * K + 2.0 * K)


def row_sym_gram_flops(nnz, K):
    """The same on the symmetric half: K(K+1) + 2K per rating."""
    return nnz * (K * (K + 1.0) + 2.0 * K)


def gathered_bytes(nnz, K, bf16=False):
    """Factor-row bytes the Gram kernel gathers per rating: the other side's FP16 hi
    and lo rows (2 x 2K B), or the BF16 row alone (2K B)."""
    return nnz * (2 if bf16 else 4) * K


# DRAM bytes (read + write) per launch, per workload, phase and kernel, from one ncu
# capture of the current kernels (two metrics, one pass, full size): the commit that
# changes a kernel sets its entry to None until it is captured again.  480k x 18k,
# K = 64, rows of 16 ratings or more on the tensor-core route: the movie Gram launch
# reads 1.09 GB (the column view's index and value stream, 0.79 GB, and user rows that
# miss L2) and writes 78.9 MB; the user Gram launch reads 0.91 GB and writes its 451,177
# Gram slots (3.98 GB), which the user factorisation launch reads back (4.05 GB) before
# writing the new rows (0.23 GB).
TRAFFIC = {"config3_480kx18k_K64": {"rows_movie/rows_gram_kernel": 1.170e9,
                                    "rows_movie/rows_chol_kernel": 142.6e6,
                                    "rows_user/rows_gram_kernel": 4.889e9,
                                    "rows_user/rows_chol_kernel": 4.271e9}}


def l2_note(nnz):
    """How the timed sweeps stand to the 129 MB L2: the ratings are held twice (CSR and
    CSC), 8 B per rating each."""
    gb = nnz * 16 / 1e9
    if gb * 1e3 > 129:
        return "inputs larger than L2 (ratings CSR+CSC %.2f GB), no flush needed" % gb
    return ("inputs fit in L2 (ratings CSR+CSC %.3f GB); sweeps run back to back in one "
            "bpmf_sweep call without a flush, as a chain's sweeps do" % gb)


def finite_or_none(x):
    """JSON has no NaN: an RMSE that is not defined yet (before burn-in) prints as null."""
    return x if x is not None and math.isfinite(x) else None


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ----------------------------------------------------------------------------
# CPU oracle timing (baseline and reference arm)
# ----------------------------------------------------------------------------
def stratified_relabel(prob, stride):
    """The same ratings with users and movies renumbered so that every contiguous block of
    1/stride of a side holds the same mix of degrees: each side's rows in degree order
    are dealt round-robin to the blocks (block b gets ranks b, b + stride, ...) and each
    block's rows are numbered consecutively, in a seeded random order.  Degrees, and so the oracle's work per row,
    are unchanged; only which rows share a block changes (a heavy-tailed side, such as
    Zipf-popular movies, otherwise gives blocks of very different cost)."""
    rng = np.random.default_rng(12345)

    def new_ids(deg):
        n = len(deg)
        ranked = np.argsort(-np.asarray(deg), kind="stable")
        # each block shuffled: the oracle's threads split a block into contiguous ranges,
        # which must not be ordered by degree either
        order = np.concatenate([rng.permutation(ranked[b::stride]) for b in range(stride)])
        ids = np.empty(n, dtype=np.int64)
        ids[order] = np.arange(n)
        return order, ids
    deg_u = np.diff(prob.csr_ptr)
    deg_v = np.bincount(prob.csr_col, minlength=prob.N)
    order_u, _ = new_ids(deg_u)
    _, ids_v = new_ids(deg_v)
    rows = np.repeat(np.arange(prob.M, dtype=np.int64), deg_u)
    new_u = np.empty(prob.M, dtype=np.int64)
    new_u[order_u] = np.arange(prob.M)
    r = new_u[rows]
    c = ids_v[prob.csr_col]
    key = np.lexsort((c, r))  # rows in their new order, columns ascending in each
    ptr = np.zeros(prob.M + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=prob.M), out=ptr[1:])
    import workloads
    return workloads.Problem(name=prob.name, M=prob.M, N=prob.N, K=prob.K, csr_ptr=ptr,
                             csr_col=c[key].astype(np.int32), csr_val=prob.csr_val[key],
                             test_i=new_u[prob.test_i].astype(np.int32),
                             test_j=ids_v[prob.test_j].astype(np.int32), test_r=prob.test_r,
                             alpha=prob.alpha, seed=prob.seed, burn_in=prob.burn_in,
                             sweeps=prob.sweeps, noise_sd=prob.noise_sd)


class OracleSampler:
    """Bounded steps of the FP64 oracle on the bench's own workload, on the host cores.

    The workload's rows are first renumbered so that every block of 1/stride of a side
    holds the same mix of degrees (stratified_relabel).  Step q takes block q mod `stride`
    of each side: rows [b n / stride, (b + 1) n / stride), which the oracle's threads
    split into contiguous ranges as they split a whole side; `stride` consecutive steps
    cover one full sweep's rows once.  A step runs the row statistics of its rows and
    their row updates (the oracle's whole per-row work of a sweep) and is timed end to
    end: rows/s = rows updated / seconds, measured, not extrapolated."""

    def __init__(self, prob, frac, nthreads=None):
        import oracle
        self.cores = nthreads or os.cpu_count() or 1
        self.stride = max(1, int(round(1.0 / frac)))
        prob = stratified_relabel(prob, self.stride)
        self.orc = oracle.Oracle(prob, nthreads=self.cores)
        self.sides = [(oracle.MOVIE, prob.N), (oracle.USER, prob.M)]

    def step(self, q):
        import oracle
        b = q % self.stride
        rows_done, secs = 0, 0.0
        for side, n in self.sides:
            lo, hi = b * n // self.stride, (b + 1) * n // self.stride
            X = self.orc.get_factors(side)[lo:hi]
            t0 = time.perf_counter()
            oracle.row_stats(X)
            self.orc.rows_range(side, lo, hi)
            secs += time.perf_counter() - t0
            rows_done += hi - lo
        return rows_done, secs

    def describe(self, steps):
        return ("%d step(s), each 1/%d of both sides (a block of %d movies and %d users with "
                "the sides' mix of degrees; row statistics and row updates), timed, not "
                "extrapolated; %d steps cover one sweep" % (
                    steps, self.stride, self.sides[0][1] // self.stride,
                    self.sides[1][1] // self.stride, self.stride))


# ----------------------------------------------------------------------------
# arms
# ----------------------------------------------------------------------------
def make_problem(args, rank):
    import workloads
    gen = workloads.CONFIGS[args.config]
    kw = {"seed": {1: 0, 2: 1, 3: 2}[args.config] + 1000 * rank}
    if args.config != 1:
        kw["scale"] = args.scale
    return gen(**kw)


def run_native(args):
    import torch

    import paper_1705_10633_gb300 as bp

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist_init(world, "nccl")
    dev = torch.device("cuda", local)
    prob = make_problem(args, rank)
    K = prob.K
    flags = bp.BPMF_BF16_GRAM if args.bf16 else 0
    stream = torch.cuda.Stream(device=dev)
    params = bp.bpmf_default_params(alpha=prob.alpha, seed=prob.seed, burn_in=prob.burn_in,
                                    flags=flags)
    h = bp.bpmf_create(prob.M, prob.N, K, prob.csr_ptr, prob.csr_col, prob.csr_val,
                       test_i=prob.test_i, test_j=prob.test_j, test_r=prob.test_r, params=params,
                       stream=stream.cuda_stream)
    phases = [bp.BPMF_PHASE_HYPER_MOVIE, bp.BPMF_PHASE_ROWS_MOVIE, bp.BPMF_PHASE_HYPER_USER,
              bp.BPMF_PHASE_ROWS_USER, bp.BPMF_PHASE_PREDICT, bp.BPMF_PHASE_ADVANCE]
    names = ["hyper_movie", "rows_movie", "hyper_user", "rows_user", "predict", "advance"]
    tuning = None
    try:
        if args.autotune:
            from paper_1705_10633_gb300.autotune import TuningCache, autotune
            cache = TuningCache(args.tuning_cache) if args.tuning_cache else None
            best, times = autotune(h, prob.M, prob.N, K, stream.cuda_stream, cache=cache,
                                   degrees=(np.diff(prob.csr_ptr), prob.col_degrees()))
            tuning = {"long_min_degree": best[0], "split_degree": best[1],
                      "rank_one_degree": best[2],
                      "trials_ms": {"%d/%d/%d" % k: round(v, 3) for k, v in sorted(times.items())}}
        for _ in range(args.warmup):
            bp.bpmf_sweep(h, 1, want_rmse=False)
        torch.cuda.synchronize(dev)
        barrier(world, local)
        torch.cuda.synchronize(dev)
        n0 = bp.bpmf_launch_count(h)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        clocks = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
        clocks.start()
        # timed region: one bpmf_sweep call of K sweeps (hyper steps overlapped with
        # row phases on the library's second stream)
        t0.record(stream)
        bp.bpmf_sweep(h, args.steps, want_rmse=False)
        t1.record(stream)
        torch.cuda.synchronize(dev)
        clk = clocks.stop()
        barrier(world, local)
        torch.cuda.synchronize(dev)
        launches = bp.bpmf_launch_count(h) - n0
        status = bp.bpmf_status(h)
        if status != 0:
            raise bp.BpmfError(status, "timed sweeps")
        rs, ra = bp.bpmf_sweep(h, 0)
        total_ms = t0.elapsed_time(t1)
        # phase breakdown (not part of the headline): phase-by-phase sweeps with
        # CUDA events on the same stream, for the roofline of the dominant launch
        nph = max(2, min(5, args.steps))
        ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(len(phases))] for _ in range(nph)]
        # the library's own events around each row phase's CUDA-core and tensor-core
        # launches (on the handle's stream)
        bp.bpmf_set_row_timing(h, True)
        launch_ms = {"rows_movie": [], "rows_user": []}
        with torch.cuda.stream(stream):
            for s_ in range(nph):
                for p_, ph in enumerate(phases):
                    ev[s_][p_][0].record(stream)
                    bp.bpmf_step(h, ph)
                    ev[s_][p_][1].record(stream)
                    if names[p_] in launch_ms:  # waits for the phase (after its end event)
                        launch_ms[names[p_]].append(bp.bpmf_row_launch_ms(h))
        torch.cuda.synchronize(dev)
        bp.bpmf_set_row_timing(h, False)
        phase_ms = {n: sum(ev[s_][p_][0].elapsed_time(ev[s_][p_][1]) for s_ in range(nph))
                    / nph for p_, n in enumerate(names)}
        phase_sweep_ms = sum(phase_ms.values())
        info_u = bp.bpmf_info(h, 0)
        info_v = bp.bpmf_info(h, 1)
        if args.log_jsonl and rank == 0:
            # per-sweep log after the measurement: one bpmf_sweep call per record, its RMSEs
            # read back (wall clock, so each record includes the read)
            done = args.warmup + args.steps + nph  # sweeps run so far on this handle
            with open(args.log_jsonl, "a") as f:
                for k in range(args.steps):
                    t_a = time.perf_counter()
                    r_s, r_a = bp.bpmf_sweep(h, 1)
                    t_ms = (time.perf_counter() - t_a) * 1e3
                    f.write(json.dumps({"job": prob.name, "sweep": done + k + 1,
                                        "rmse_sample": finite_or_none(r_s),
                        "rmse_avg": finite_or_none(r_a), "t_ms": round(t_ms, 4),
                        "rows_per_s": round((prob.M + prob.N) / (t_ms / 1e3), 1)}) + "\n")
    finally:
        bp.bpmf_destroy(h)

    max_ms = reduce_over_ranks(total_ms, world, "max", dev)
    value = aggregate_rows_per_s((prob.M + prob.N) * world, args.steps, max_ms)
    ms_per_step = max_ms / args.steps

    # The dominant kernel: the longest launch of the slower row phase -- on the tensor-core
    # route (K pads to 64) the Gram kernel (tcgen05) or the factorisation kernel (FP32
    # CUDA cores), else the CUDA-core kernel, whose FP32 work includes the Gram.
    nnz = prob.nnz
    tc_path = (K + 15) // 16 * 16 == 64
    dom = max(("rows_movie", "rows_user"), key=lambda n: phase_ms[n])
    peaks = load_peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = n_sm * 128 * 2 * sm_max * 1e6 / 1e12  # FP32 FMA lanes x 2 flops x clock
    tc_peak = peaks.get("bf16_tflops_sustained", 1700.0)
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    fp32_src = "FP32 CUDA-core peak derived from %d SMs x 128 lanes x 2 x %.0f MHz" % (n_sm, sm_max)
    tc_src = "measured sustained bf16 (FP16 runs at the bf16 rate)"
    traffic_of = TRAFFIC.get(prob.name, {})

    def split_bins(phase):
        # the phase's rows by route: the short bin (n_short smallest degrees) on the
        # CUDA-core kernel, the rest on the tensor-core route when K pads to 64
        info_d = info_u if phase == "rows_user" else info_v
        deg = np.sort(np.diff(prob.csr_ptr) if phase == "rows_user" else prob.col_degrees())
        n_s = int(info_d["n_short"])
        r_s = int(deg[:n_s].sum())
        rows_all = prob.M if phase == "rows_user" else prob.N
        return n_s, r_s, rows_all - n_s, nnz - r_s

    def mean_ms(phase, k):
        vals = [v[k] for v in launch_ms[phase] if v[k] >= 0]
        return float(np.mean(vals)) if vals else None

    def launch_entry(phase, kern):
        """Achieved rate of one launch of `phase` against its own roof."""
        n_s, r_s, n_l, r_l = split_bins(phase)
        if kern == "rows_gram_kernel":
            t = mean_ms(phase, 1)
            if t is None:
                return None
            t /= 1e3
            fl = row_gram_flops(r_l, K)
            e = {"kernel": "rows_gram_kernel (%s: %d rows, %d ratings)" % (phase, n_l, r_l),
                 "bound": "tensor", "launch_ms": round(t * 1e3, 4),
                 "achieved": round(fl / t / 1e12, 2), "peak": tc_peak, "unit": "TFLOP/s",
                 "frac": round(fl / t / 1e12 / tc_peak, 4), "peak_source": tc_src,
                 "algorithmic": "2K^2 + 2K flop per rating (the full K x K Gram tile and the "
                                "right-hand side); %d ratings" % r_l,
                 "symmetric": {"achieved": round(row_sym_gram_flops(r_l, K) / t / 1e12, 2),
                               "frac": round(row_sym_gram_flops(r_l, K) / t / 1e12 / tc_peak, 4),
                               "note": "K(K+1) + 2K flop per rating, the Gram's lower half"},
                 "gathered_l2_tbs": round(gathered_bytes(r_l, K, args.bf16) / t / 1e12, 3),
                 "gathered_note": "the other side's 16-bit factor rows gathered per rating "
                                  "(%d B), served mostly from L2; not an HBM rate"
                                  % ((2 if args.bf16 else 4) * K)}
        elif kern == "rows_chol_kernel":
            t = mean_ms(phase, 2)
            if t is None:
                return None
            t /= 1e3
            fl = row_alu_flops(n_l, K)
            e = {"kernel": "rows_chol_kernel (%s: %d rows)" % (phase, n_l), "bound": "alu",
                 "launch_ms": round(t * 1e3, 4), "achieved": round(fl / t / 1e12, 3),
                 "peak": round(fp32_peak, 2), "unit": "TFLOP/s",
                 "frac": round(fl / t / 1e12 / fp32_peak, 4), "peak_source": fp32_src,
                 "algorithmic": "K^3/3 + 2K^2 flop per row (Cholesky, two triangular solves)"}
        else:
            t = mean_ms(phase, 0)
            if t is None:
                return None
            t /= 1e3
            n_r, r_r = (n_s, r_s) if tc_path else (n_s + n_l, r_s + r_l)
            fl = row_alu_flops(n_r, K) + row_gram_flops(r_r, K)
            e = {"kernel": "rows_warp_kernel (%s: %d rows, %d ratings)" % (phase, n_r, r_r),
                 "bound": "alu", "launch_ms": round(t * 1e3, 4),
                 "achieved": round(fl / t / 1e12, 3), "peak": round(fp32_peak, 2),
                 "unit": "TFLOP/s", "frac": round(fl / t / 1e12 / fp32_peak, 4),
                 "peak_source": fp32_src,
                 "algorithmic": "Gram 2K^2 + 2K flop per rating and K^3/3 + 2K^2 per row"}
        tr = traffic_of.get("%s/%s" % (phase, kern))
        e["traffic"] = tr
        if tr:
            e["dram"] = {"achieved_gbs": round(tr / t / 1e9, 1), "peak_gbs": hbm_peak,
                         "frac": round(tr / t / 1e9 / hbm_peak, 4),
                         "note": "ncu DRAM bytes of one launch over its time, of measured HBM copy"}
        return e

    per_launch = {}
    for phase in ("rows_movie", "rows_user"):
        for kern in (("rows_warp_kernel", "rows_gram_kernel", "rows_chol_kernel") if tc_path
                     else ("rows_warp_kernel",)):
            ent = launch_entry(phase, kern)
            if ent is not None:
                per_launch["%s/%s" % (phase, kern)] = ent
    dom_key = max((k for k in per_launch if k.startswith(dom)),
                  key=lambda k: per_launch[k]["launch_ms"])
    roofline = dict(per_launch[dom_key])
    roofline["launches"] = {k: {kk: v[kk] for kk in ("launch_ms", "bound", "achieved", "unit",
                                                     "frac", "traffic")}
                            for k, v in per_launch.items() if k != dom_key}
    roofline["phase_ms"] = {k: round(v, 4) for k, v in phase_ms.items()}
    roofline["phase_note"] = ("phases timed one by one (hyper steps not overlapped, all SMs to "
                              "the row kernels, row phases also recording their launch events); "
                              "%.2f ms per sweep that way" % phase_sweep_ms)

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, prob, bp, torch, dev, stream, world, local)

    out = {"metric": METRIC % K, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "bf16-gram/f32" if args.bf16 else "f32", "data": "synthetic",
           "config": {"workload": prob.name, "M": prob.M, "N": prob.N, "K": K, "nnz": nnz,
                      "test": prob.T, "sweeps_per_s": round(1e3 / ms_per_step, 3),
                      "l2": l2_note(nnz),
                      "bins": {"users": [info_u["n_short"], info_u["n_long"]],
                               "movies": [info_v["n_short"], info_v["n_long"]],
                               "split_rows_segments": [[info_u["n_split"], info_u["n_segments"]],
                                                       [info_v["n_split"], info_v["n_segments"]]],
                               "balanced_plan": [info_u["balanced"], info_v["balanced"]]},
                      "tuning": tuning, "parallelism": "replicas x%d" % world, "rmse_sample": finite_or_none(rs), "rmse_avg": finite_or_none(ra)},
           "roofline": roofline, "clocks": clk, "gpu_launches": int(launches), "e2e": e2e}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sampler = OracleSampler(prob, args.cpu_frac)
        rows_t, secs_t = 0, 0.0
        for s in range(CPU_BASELINE_STEPS):
            rows, secs = sampler.step(s)
            rows_t += rows
            secs_t += secs
        out["cpu_baseline"] = {"value": round(rows_t / secs_t, 2), "unit": UNIT,
                               "cores": sampler.cores, "kind": "oracle",
                               "sample": sampler.describe(CPU_BASELINE_STEPS)}
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_sharded(args):
    """N > 1 ranks, one chain: each rank updates a cost-balanced range of the rows of
    both sides and the ranks all-gather the updated rows after every half-sweep
    (paper_1705_10633_gb300.shard); every rank holds the whole problem.  The total work
    is one chain whatever N: strong scaling.  value = (M + N) x sweeps / the slowest
    rank's time."""
    import torch
    import torch.distributed as dist

    import paper_1705_10633_gb300 as bp
    from paper_1705_10633_gb300.shard import HandleBackend, ShardedChain

    rank, world, local = dist_env()
    device_x = args.exchange == "device"
    torch.cuda.set_device(local if device_x else local % max(1, torch.cuda.device_count()))
    dist_init(world, "nccl" if device_x else "gloo")
    dev = torch.device("cuda", torch.cuda.current_device())
    prob = make_problem(args, 0)  # one chain: every rank builds the same problem
    K = prob.K
    flags = bp.BPMF_BF16_GRAM if args.bf16 else 0
    params = bp.bpmf_default_params(alpha=prob.alpha, seed=prob.seed, burn_in=prob.burn_in,
                                    flags=flags)

    def sync():
        torch.cuda.synchronize(dev)
        barrier(world, dev.index if device_x else None)
        torch.cuda.synchronize(dev)

    # the handle's stream is torch's current stream, so the collectives (ordered on the
    # current stream) and the handle's copies and kernels follow one order
    t_e0 = time.perf_counter()
    h = bp.bpmf_create(prob.M, prob.N, K, prob.csr_ptr, prob.csr_col, prob.csr_val,
                       test_i=prob.test_i, test_j=prob.test_j, test_r=prob.test_r, params=params,
                       stream=bp.torch_stream())
    try:
        chain = ShardedChain(HandleBackend(bp, h, prob.M, prob.N, K, prob.degrees(),
                                           prob.col_degrees(), device=device_x), rank, world)
        chain.sweep(args.warmup)
        sync()
        n0 = bp.bpmf_launch_count(h)
        clocks = ClockSampler(dev.index)
        clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        chain.sweep(args.steps)
        e1.record()
        sync()
        clk = clocks.stop()
        total_ms = e0.elapsed_time(e1)
        launches = bp.bpmf_launch_count(h) - n0
        rs, ra = bp.bpmf_sweep(h, 0)  # the RMSE read back ends the end-to-end region
        t_e1 = time.perf_counter()
        assert bp.bpmf_status(h) == 0
    finally:
        bp.bpmf_destroy(h)
    max_ms = reduce_over_ranks(total_ms, world, "max", dev.index if device_x else None)
    value = (prob.M + prob.N) * args.steps / (max_ms / 1e3)
    e2e_s = reduce_over_ranks(t_e1 - t_e0, world, "max", dev.index if device_x else None)
    out = {"metric": METRIC % K, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(max_ms / args.steps, 4), "higher_is_better": True,
           "scaling": "strong", "vs_baseline": None,
           "dtype": "bf16-gram/f32" if args.bf16 else "f32", "data": "synthetic",
           "config": {"workload": prob.name, "M": prob.M, "N": prob.N, "K": K, "nnz": prob.nnz,
                      "test": prob.T, "l2": l2_note(prob.nnz),
                      "parallelism": "sharded rows x%d (%s all-gather after each half-sweep)"
                                     % (world, "NCCL" if device_x else "gloo host"),
                      "ranges": {"users": chain.ranges[0], "movies": chain.ranges[1]},
                      "rmse_sample": finite_or_none(rs), "rmse_avg": finite_or_none(ra)},
           "clocks": clk, "gpu_launches": int(launches),
           "e2e": {"value": round((prob.M + prob.N) * (args.warmup + args.steps) / e2e_s, 1),
                   "unit": UNIT,
                   "h2d_bytes_per_step": int(8 * (prob.M + 1) + 8 * prob.nnz + 12 * prob.T)
                                         // (args.warmup + args.steps),
                   "d2h_bytes_per_step": 16 // (args.warmup + args.steps),
                   "note": "wall clock of bpmf_create from host arrays, the warm-up and timed "
                           "sweeps with their exchanges, and the RMSE read back; slowest rank"}}
    if rank == 0:
        print(json.dumps(out), flush=True)
    dist.destroy_process_group()


def run_e2e(args, prob, bp, torch, dev, stream, world, local):
    """Whole job through the public C ABI from host buffers: create (host -> device
    copies of the ratings and test set, column view, bins, initial draw), then
    `steps` sweeps each returning its RMSE to the host."""
    h2d = (prob.csr_ptr.nbytes + prob.csr_col.nbytes + prob.csr_val.nbytes + prob.test_i.nbytes
           + prob.test_j.nbytes + prob.test_r.nbytes)
    # the job's host buffers live in pinned memory (filled before the timed region)
    ptr, col, val, ti, tj, tr = (torch.from_numpy(x).pin_memory().numpy() for x in
                                 (prob.csr_ptr, prob.csr_col, prob.csr_val, prob.test_i,
                                  prob.test_j, prob.test_r))
    barrier(world, local)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    params = bp.bpmf_default_params(alpha=prob.alpha, seed=prob.seed, burn_in=prob.burn_in,
                                    flags=bp.BPMF_BF16_GRAM if args.bf16 else 0)
    h = bp.bpmf_create(prob.M, prob.N, prob.K, ptr, col, val, test_i=ti, test_j=tj, test_r=tr,
                       params=params, stream=stream.cuda_stream)
    try:
        for _ in range(args.steps):
            bp.bpmf_sweep(h, 1)  # RMSE of the step read back to the host
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
    finally:
        bp.bpmf_destroy(h)
    ms = reduce_over_ranks((t1 - t0) * 1e3, world, "max", dev)
    return {"value": round(aggregate_rows_per_s((prob.M + prob.N) * world, args.steps, ms), 1),
            "unit": UNIT, "h2d_bytes_per_step": int(h2d / args.steps),
            "d2h_bytes_per_step": 16,
            "note": "wall clock of bpmf_create from pinned host arrays + %d x bpmf_sweep with "
                    "RMSE read back" % args.steps}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    prob = make_problem(args, 0)
    sampler = OracleSampler(prob, args.ref_frac)
    walls, rows_t, secs_t = [], 0, 0.0
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        rows, secs = sampler.step(s)
        t1 = time.perf_counter()
        if s >= args.warmup:
            walls.append(t1 - t0)
            rows_t += rows
            secs_t += secs
    value = rows_t / secs_t
    cores, desc = sampler.cores, sampler.describe(args.steps)
    out = {"metric": METRIC % prob.K, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(1e3 * float(np.mean(walls)), 2), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": prob.name, "M": prob.M, "N": prob.N, "K": prob.K,
                      "nnz": prob.nnz},
           "cpu_baseline": {"value": round(value, 2), "unit": UNIT, "cores": cores,
                            "kind": "oracle", "sample": desc},
           "e2e": {"value": round(value, 2), "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_batched(args):
    """Many independent jobs (the batched form): the same jobs and sweeps run one at a
    time on one stream (plain per-job form), together with bpmf_sweep_batch (one
    stream per job), and in shared launches with bpmf_batch_sweep (the headline).
    Device-bound regions between synchronisations are timed with the host clock
    (nothing else runs on the GPU).  Prints one JSON line."""
    import torch

    import paper_1705_10633_gb300 as bp
    import workloads

    torch.cuda.set_device(0)
    jobs = workloads.config4(n_jobs=args.jobs)
    rows = sum(j.M + j.N for j in jobs)
    nnz = sum(j.nnz for j in jobs)

    def make(prob, stream):
        flags = bp.BPMF_BF16_GRAM if (args.bf16 and prob.K == 64) else 0
        p = bp.bpmf_default_params(alpha=prob.alpha, seed=prob.seed, burn_in=prob.burn_in,
                                   flags=flags)
        return bp.bpmf_create(prob.M, prob.N, prob.K, prob.csr_ptr, prob.csr_col, prob.csr_val,
                              test_i=prob.test_i, test_j=prob.test_j, test_r=prob.test_r,
                              params=p, stream=stream)

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    out = {}
    one = torch.cuda.Stream()
    hs = [make(prob, one.cuda_stream) for prob in jobs]
    try:
        for h in hs:
            bp.bpmf_sweep(h, args.warmup, want_rmse=False)
        t_plain = timed(lambda: [bp.bpmf_sweep(h, args.steps, want_rmse=False) for h in hs])
        plain_rmse = [bp.bpmf_sweep(h, 0) for h in hs]
    finally:
        for h in hs:
            bp.bpmf_destroy(h)
    streams = [torch.cuda.Stream() for _ in jobs]
    hs = [make(prob, st.cuda_stream) for prob, st in zip(jobs, streams)]
    try:
        bp.bpmf_sweep_batch(hs, args.warmup)
        n0 = sum(bp.bpmf_launch_count(h) for h in hs)
        t_batch = timed(lambda: bp.bpmf_sweep_batch(hs, args.steps))
        launches = sum(bp.bpmf_launch_count(h) for h in hs) - n0
        batch_rmse = [bp.bpmf_sweep(h, 0) for h in hs]
        status = [bp.bpmf_status(h) for h in hs]
    finally:
        for h in hs:
            bp.bpmf_destroy(h)
    # the shared-launch form: every step for all jobs in one launch per kernel variant
    streams = [torch.cuda.Stream() for _ in jobs]
    bst = torch.cuda.Stream()
    hs = [make(prob, st.cuda_stream) for prob, st in zip(jobs, streams)]
    b = None
    try:
        b = bp.bpmf_batch_create(hs, stream=bst.cuda_stream)
        bp.bpmf_batch_sweep(b, args.warmup)
        n0 = bp.bpmf_batch_launch_count(b)
        t_shared = timed(lambda: bp.bpmf_batch_sweep(b, args.steps))
        launches_shared = bp.bpmf_batch_launch_count(b) - n0
        shared_rmse = [bp.bpmf_sweep(h, 0) for h in hs]
        status += [bp.bpmf_status(h) for h in hs]
    finally:
        if b is not None:
            bp.bpmf_batch_destroy(b)
        for h in hs:
            bp.bpmf_destroy(h)
    same = all(x == y == z for x, y, z in zip(plain_rmse, batch_rmse, shared_rmse))
    value = rows * args.steps / t_shared
    out = {"metric": "latent rows sampled/s (batched independent jobs)", "value": round(value, 1),
           "unit": "rows/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(1e3 * t_shared / args.steps, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "bf16-gram/f32" if args.bf16 else "f32", "data": "synthetic",
           "config": {"workload": "config4_%djobs" % len(jobs), "jobs": len(jobs), "rows": rows,
                      "nnz": nnz, "K": {str(k): sum(1 for j in jobs if j.K == k)
                                        for k in (16, 32, 64)},
                      "form": "bpmf_batch_sweep: shared launches over a table of jobs, heaviest "
                              "first, one CUDA graph per sweep"},
           "streams": {"value": round(rows * args.steps / t_batch, 1), "unit": "rows/s",
                       "ms_per_step": round(1e3 * t_batch / args.steps, 3),
                       "gpu_launches": int(launches),
                       "note": "bpmf_sweep_batch: each job's captured sweep on its own streams"},
           "plain": {"value": round(rows * args.steps / t_plain, 1), "unit": "rows/s",
                     "ms_per_step": round(1e3 * t_plain / args.steps, 3),
                     "note": "same jobs one at a time on one stream"},
           "shared_over_streams": round(t_batch / t_shared, 3),
           "shared_over_plain": round(t_plain / t_shared, 3),
           "sweeps_per_s": {"shared": round(len(jobs) * args.steps / t_shared, 1),
                            "streams": round(len(jobs) * args.steps / t_batch, 1),
                            "plain": round(len(jobs) * args.steps / t_plain, 1)},
           "same_rmse_all_forms": same, "status_ok": all(x == 0 for x in status),
           "gpu_launches": int(launches_shared)}
    print(json.dumps(out), flush=True)


def run_serving(args):
    """Serving loop (continuous batching): jobs arrive as a Poisson process (rate
    args.rate per second for args.duration seconds), each a fresh problem drawn from
    config 4's distribution with its own chain seed, asking for args.job_sweeps sweeps
    and predictions at 1,000 query points.  The same arrival sequence is served three
    ways: up to args.slots jobs resident under a 150 GB budget (memory never binds),
    the same slots under a budget that binds (args.mem_budget_gb, by default a quarter
    of the first run's peak, at least the largest job), and one job at a time.  Prints
    one JSON line with latency and queue-wait percentiles, aggregate rows/s, peak
    device memory and how many jobs waited for memory, for each form side by side."""
    import torch

    import paper_1705_10633_gb300 as bp
    import workloads
    from paper_1705_10633_gb300.serve import Job, Server, latency_percentiles, queue_wait_percentiles

    torch.cuda.set_device(0)
    rng = np.random.default_rng(17)
    t, arrivals = 0.0, []
    while True:
        t += rng.exponential(1.0 / args.rate)
        if t > args.duration:
            break
        prob = workloads.config4_job(rng, 5000 + len(arrivals))
        qi = rng.integers(0, prob.M, 1000).astype(np.int32)
        qj = rng.integers(0, prob.N, 1000).astype(np.int32)
        arrivals.append((t, prob, qi, qj, int(rng.integers(1 << 30))))
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    largest = max(bp.bpmf_device_bytes(a[1].M, a[1].N, a[1].K, a[1].csr_ptr, a[1].csr_col,
                                       len(a[1].test_i), num_sms=sms) for a in arrivals)

    def serve(slots, budget):
        srv = Server(memory_limit=budget, max_active=slots, sweeps_per_round=5)
        futs, t0 = [], time.perf_counter()
        for at, prob, qi, qj, seed in arrivals:
            delay = t0 + at - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            futs.append(srv.submit(Job(problem=prob, sweeps=args.job_sweeps, query_i=qi,
                                       query_j=qj, seed=seed)))
        res = [f.result() for f in futs]
        srv.close()
        span = max(r.finished_at for r in res) - min(r.submitted_at for r in res)
        rows = sum((a[1].M + a[1].N) * args.job_sweeps for a in arrivals)
        lat, wait = latency_percentiles(res), queue_wait_percentiles(res)
        return {"p50_s": round(lat["p50"], 4), "p99_s": round(lat["p99"], 4),
                "queue_wait_p50_s": round(wait["p50"], 4),
                "queue_wait_p99_s": round(wait["p99"], 4),
                "rows_per_s": round(rows / span, 1), "jobs_per_s": round(len(res) / span, 2),
                "makespan_s": round(span, 3), "rounds": srv.rounds,
                "memory_budget_gb": round(budget / 1e9, 3),
                "peak_memory_gb": round(srv.peak_memory / 1e9, 3),
                "jobs_waited_for_memory": srv.memory_waits}, res

    batched, rb = serve(args.slots, 150e9)
    budget = (args.mem_budget_gb * 1e9 if args.mem_budget_gb
              else max(largest, 0.25 * batched["peak_memory_gb"] * 1e9))
    bound, rm = serve(args.slots, budget)
    alone, ra = serve(1, 150e9)
    same = all(np.array_equal(x.predictions, y.predictions) and
               np.array_equal(x.predictions, z.predictions) for x, y, z in zip(rb, ra, rm))
    out = {"metric": "serving job latency p50/p99 (s) and aggregate rows/s",
           "value": batched["p99_s"], "unit": "s (p99 job latency)", "n_gpus": 1,
           "higher_is_better": False, "data": "synthetic",
           "config": {"workload": "config5_poisson", "rate_jobs_per_s": args.rate,
                      "duration_s": args.duration, "jobs": len(arrivals),
                      "sweeps_per_job": args.job_sweeps, "queries_per_job": 1000,
                      "jobs_from": "each a fresh draw from config 4's distribution",
                      "rows_per_job_mean": round(float(np.mean([a[1].M + a[1].N
                                                                for a in arrivals])), 1),
                      "ratings_per_job_mean": round(float(np.mean([a[1].nnz
                                                                   for a in arrivals])), 1),
                      "largest_job_gb": round(largest / 1e9, 3), "slots": args.slots,
                      "sweeps_per_round": 5},
           "batched": batched, "batched_memory_bound": bound, "one_at_a_time": alone,
           "p99_ratio_alone_over_batched": round(alone["p99_s"] / batched["p99_s"], 3),
           "rows_per_s_ratio": round(batched["rows_per_s"] / alone["rows_per_s"], 3),
           "same_predictions_in_all_three": same}
    print(json.dumps(out), flush=True)


def run_fig3(args):
    """Per-row cost against degree for each route of the row update, the GPU analogue of
    the paper's Fig. 3 (time to update one item against its number of ratings for the
    rank-one, sequential-Cholesky and parallel-Cholesky methods, Sec. 3.2).  For each
    degree d and route: microseconds per row of a user phase over many rows of degree d
    (throughput), and the phase time for a single row (latency of one item)."""
    import torch

    import paper_1705_10633_gb300 as bp
    import workloads
    torch.cuda.set_device(0)
    degrees = [1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096]
    no = 1 << 30
    routes = {
        32: {"gram": dict(rank_one_degree=-1, split_degree=no),
             "rank_one": lambda d: dict(rank_one_degree=d + 1, split_degree=no),
             "split": lambda d: dict(rank_one_degree=-1, split_degree=max(2, d // 4))},
        64: {"gram_cuda_core": dict(flags=bp.BPMF_CUDA_CORE_GRAM, rank_one_degree=-1,
                                    split_degree=no),
             "rank_one": lambda d: dict(flags=bp.BPMF_CUDA_CORE_GRAM, rank_one_degree=d + 1,
                                        split_degree=no),
             "split_cuda_core": lambda d: dict(flags=bp.BPMF_CUDA_CORE_GRAM, rank_one_degree=-1,
                                               split_degree=max(2, d // 4)),
             "tensor_core": dict(rank_one_degree=-1, split_degree=no)},
    }

    def phase_ms(prob, kw):
        st = torch.cuda.Stream()
        params = bp.bpmf_default_params(alpha=prob.alpha, seed=1, **kw)
        h = bp.bpmf_create(prob.M, prob.N, prob.K, prob.csr_ptr, prob.csr_col, prob.csr_val,
                           params=params, stream=st.cuda_stream)
        try:
            bp.bpmf_step(h, bp.BPMF_PHASE_ROWS_USER)
            ts = []
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                bp.bpmf_step(h, bp.BPMF_PHASE_ROWS_USER)
                e1.record(st)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            if bp.bpmf_status(h) != 0:
                raise bp.BpmfError(bp.bpmf_status(h), "fig3")
            return float(np.median(ts))
        finally:
            bp.bpmf_destroy(h)

    table = {}
    for K, rs in routes.items():
        table[K] = {name: {} for name in rs}
        for d in degrees:
            M = int(max(256, min(20000, 4_000_000 // d)))
            N = max(2 * d, 2000)
            many = workloads.fixed_degree(M, N, K, d, seed=d)
            one = workloads.fixed_degree(1, N, K, d, seed=d)
            for name, kw in rs.items():
                kw = kw(d) if callable(kw) else kw
                t_many = phase_ms(many, kw)
                t_one = phase_ms(one, kw)
                table[K][name][d] = [round(1e3 * t_many / M, 4), round(1e3 * t_one, 2)]
    out = {"metric": "row update time against degree (us per row over many rows; us for one row)",
           "data": "synthetic, every row of the phase with the same degree",
           "degrees": degrees, "table": {str(k): v for k, v in table.items()}}
    print(json.dumps(out), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--config", type=int, choices=[1, 2, 3, 4, 5], default=3,
                    help="4: batched independent jobs (bpmf_sweep_batch against one at a time); "
                         "5: serving loop with Poisson arrivals")
    ap.add_argument("--jobs", type=int, default=256, help="config 4: number of jobs")
    ap.add_argument("--rate", type=float, default=50.0, help="config 5: arrivals per second")
    ap.add_argument("--duration", type=float, default=4.0, help="config 5: arrival window (s)")
    ap.add_argument("--job-sweeps", type=int, default=100, help="config 5: sweeps per job")
    ap.add_argument("--slots", type=int, default=64, help="config 5: jobs resident at once")
    ap.add_argument("--mem-budget-gb", type=float, default=None,
                    help="config 5: device memory budget of the memory-bound run")
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--bf16", action="store_true",
                    help="BF16-input tensor-core Gram (lower precision; not the headline)")
    ap.add_argument("--autotune", action="store_true",
                    help="tune the row kernels' thresholds on the workload before timing")
    ap.add_argument("--tuning-cache", default=None,
                    help="with --autotune: JSON file of tunings by workload shape (reused on a hit)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-frac", type=float, default=0.1,
                    help="fraction of each side's rows in one oracle step (cpu_baseline leg)")
    ap.add_argument("--ref-frac", type=float, default=0.1,
                    help="the same for --impl reference (one oracle step per bench step)")
    ap.add_argument("--log-jsonl", default=None,
                    help="append one JSON record per sweep (sweep, RMSEs, time) after the run")
    ap.add_argument("--exchange", choices=["device", "host"], default="device",
                    help="N > 1: all-gather device rows over NCCL (one GPU per rank), or host "
                         "copies over gloo (ranks may then share a GPU)")
    ap.add_argument("--fig3", action="store_true",
                    help="row update time against degree for every route (the paper's Fig. 3)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference" and args.config in (4, 5):
        print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the "
                          "single-job configs 1-3; configs 4 and 5 compare batched and "
                          "one-at-a-time forms of this library"}), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    elif args.fig3:
        run_fig3(args)
    elif args.config == 4:
        run_batched(args)
    elif args.config == 5:
        run_serving(args)
    elif dist_env()[1] > 1:
        run_sharded(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
