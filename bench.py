#!/usr/bin/env python
"""Throughput of the fused all-pairs Lipschitz envelope evaluation on a B300.

Default workload (monotone_d4): N = 100,000 data points, Q = 1,000,000 queries in [0,1]^4,
increasing in x1 and x2.  One step = the whole hot path over that batch, once per norm
(L1, L2, Linf):
  fit   (lip_clear + lip_add: copy and scan-layout transform, Sec. 5 add())
  eval  (lip_eval: scan kernel + split merge with FP64 re-evaluation, Eq. (upperlower), (eq:g))
  M_est (lip_estimate_M: all-pairs Lipschitz constant, Sec. 5)
Metric: query x datapoint pairs evaluated per second (G pairs/s) = 3 Q N / step time.

Other workloads (--workload): plain_d2 (d=2, FP32 and FP64), cluster_d16 (d=16 Gaussian
mixture, N = Q = 1e6, plain FP32 L2), grad_d8 (d=8, forward + backward), batch_4096
(4096 independent sets in one persistent launch replayed from a CUDA graph).

Timing: CUDA events per step on the launching stream.  Where the inputs fit in L2
(126 MB), L2 is flushed before every timed step by writing a 256 MB buffer (outside the
timed interval).  N > 1 (torchrun), monotone_d4: the queries are sharded over the GPUs
(weak scaling: rank r evaluates its own block of 1e6 queries of an N x 1e6 query set,
the data replicated on every GPU, no exchange in the evaluation), and the estimate's pair
triangle is shared out block-cyclically with one all_gather of the ranks' 4-number
results per norm; value = all ranks' query x data pairs / the slowest rank's time.
Other workloads run one copy per GPU.

--impl reference times the FP64 CPU oracle (the checker, as it stands) on the host
cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2606_04670_b300 import workloads as W  # noqa: E402

METRIC = "G pairs/s (query x datapoint) fused eval"
UNIT = "G pairs/s"
NORMS = (W.NORM_L1, W.NORM_L2, W.NORM_LINF)
NNAME = {1: "L1", 2: "L2", 3: "Linf"}
FP32_LANES_PER_SM = 128
WORKLOADS = ("monotone_d4", "plain_d2", "cluster_d16", "cluster_d16_tc", "cluster_d16_bf16", "cluster_d16_fp16",
             "grad_d8", "batch_4096", "local_d4", "smooth_d4")
SMOOTH_ITERS = 10
LOCAL_KNOTS, LOCAL_SAMPLE, LOCAL_SEED = 16, 32768, 0
# special-function (MUFU) results per SM per clock
MUFU_PER_SM = 16
# TF32 dense peak: the measured BF16 peak times the nominal TF32 / BF16 ratio (1.1 / 2.25)
TF32_OVER_BF16 = 1.1 / 2.25
# FP32 lane operations per pair of the tensor-core epilogue (TMEM load share, clamp, the
# square root's share, two FMAs, two extrema, the candidate test)
TC_I_EPI = 6
# dram__bytes_read.sum + dram__bytes_write.sum per launch of each workload's dominant
# kernel at the full workload size (one-pass ncu captures of the timed step's launch).  An
# entry is removed whenever its kernel changes, until it is captured again.
KERNEL_DRAM_BYTES = {
    ("monotone_d4", 2): 19.136000e6 + 11.619840e6,     # scan_exact_kernel<L2, C=2, U=2, R=4>
    ("monotone_d4", 1, "pruned"): 23.162e6 + 0.374e6,  # scan_pruned_kernel<L1, C=2, U=2, R=4>
    ("monotone_d4", 2, "pruned"): 24.757e6 + 1.910e6,  # scan_pruned_kernel<L2, C=2, U=2, R=4>
    ("monotone_d4", 3, "pruned"): 24.953e6 + 2.098e6,  # scan_pruned_kernel<Linf, C=2, U=2, R=4>
    ("grad_d8", 2): 16.66e6 + 13.47e6,                 # scan_exact_kernel<L2, C=4, U=4, R=2>
    ("cluster_d16", 2): 618.02e6 + 185.20e6,           # scan_exact_kernel<L2, C=0, U=16, R=2>
    ("cluster_d16", 2, "pruned"): 659.572e6 + 34.959e6,  # scan_pruned_kernel<L2, C=0, U=16, R=1>
    ("cluster_d16_tc", 2): 7185.37e6 + 1213.84e6,      # tc_scan_kernel<K=16, 4 parts, TF32> (persistent, soft lockstep)
    ("cluster_d16_bf16", 2): 5275.18e6 + 1081.80e6,    # tc_scan_kernel<K=16, 4 parts, BF16> (persistent, soft lockstep)
    ("cluster_d16_fp16", 2): 3413.92e6 + 943.47e6,     # tc_scan_kernel<K=16, 4 parts, FP16> (persistent, soft lockstep)
    ("local_d4", 2): 32.64e6 + 1.43e6,                 # loc_scan_kernel<L2, 4, bucket, G=2>
    ("smooth_d4", 2): 4.54e6 + 40.80e6,                # smooth_pass_kernel<L2, 4> (share q, 64 splits)
    ("batch_4096", 0): 4817.68e6 + 1598.16e6,          # batch_scan_kernel
}


def traffic_for(args, name, norm, pruned=False):
    """The stored DRAM bytes of a workload's dominant kernel, at the full workload size only."""
    key = (name, norm, "pruned") if pruned else (name, norm)
    return None if getattr(args, "queries", 0) else KERNEL_DRAM_BYTES.get(key)


def i_pair(norm: int, d: int, c: int) -> int:
    """Algorithmic FP32 lane operations per pair: minimal scalar instruction counts with
    |.| and negation as free operand modifiers, plus 4 for the two bounds and extrema:
    2(d-c) for the free coordinates, k c + 2 for the c constrained ones (k = 4 L1,
    5 L2, 3 Linf)."""
    k = {W.NORM_L1: 4, W.NORM_L2: 5, W.NORM_LINF: 3}[norm]
    return 2 * (d - c) + (k * c + 2 if c else 0) + 4


def mufu_per_pair(norm: int, c: int) -> int:
    return 0 if norm != W.NORM_L2 else (2 if c else 1)


def fma_lanes_per_pair(norm: int, d: int, c: int) -> int:
    """Algorithmic lane operations per pair on the FP32 FMA pipe (adds, multiplies and FMAs;
    minimum, maximum and the positive / negative parts run on the ALU pipe, square roots on
    MUFU): the d coordinate differences, then L2: one square-accumulate per free coordinate
    and two per constrained one (the upper and the lower part); L1: one add per coordinate;
    Linf: none (maxima only); plus the two bound values y + M d_up and y - M d_lo."""
    if norm == W.NORM_L2:
        return d + (d - c) + 2 * c + 2
    if norm == W.NORM_L1:
        return d + d + 2
    return d + 2


def tc_roofline(ctx, prec, d, pairs, ms, alu, traffic):
    """Roofline of the tensor-core scan.  The algorithmic tensor work of a pair is the
    augmented product of the method, [-2q, 1, |q|^2 hi, |q|^2 lo] . [x, |x|^2 hi, |x|^2 lo, 1]:
    2 K flops with K = d + 3 padded to the MMA's K step (8 for TF32, 16 for the 16-bit kinds;
    24 and 32 at d = 16), against the measured dense BF16 peak (FP16's rate is BF16's;
    TF32 takes 1.1 / 2.25 of it).  The MMA work the kernel actually issues (the split
    products and the norm block) and the epilogue's ALU roof are reported beside it."""
    fmt = {"tc_tf32": "TF32", "tc_bf16": "BF16", "tc_fp16": "FP16"}[prec]
    f16 = fmt != "TF32"
    step = 16 if f16 else 8
    k_alg = step * ((d + 3 + step - 1) // step)
    # issued: the piece products over K = d padded, plus the norm block's 32 bytes of K
    kk = 16 * ((d + 15) // 16) if f16 else 8 * ((d + 7) // 8)
    npass = 6 if fmt == "BF16" else 3
    fpp_issued = 2 * (npass * kk + (16 if f16 else 8))
    pairs_s = pairs / (ms / 1e3)
    ratio = 1.0 if f16 else TF32_OVER_BF16
    peak = float(ctx.peaks.get("bf16_tflops", 1800.0)) * ratio * 1e12
    sus = float(ctx.peaks.get("bf16_tflops_sustained", 1400.0)) * ratio * 1e12
    ach = 2.0 * k_alg * pairs_s
    # epilogue: about I_EPI FP32 lane operations per pair on the SMs' 128 lanes per clock
    epi_peak = ctx.sms * FP32_LANES_PER_SM * ctx.sm_max * 1e6 / TC_I_EPI
    return {"bound": "tensor", "kernel": f"tc_scan_kernel<K={kk}, {fmt}>",
            "achieved": ach / 1e12, "peak": peak / 1e12, "unit": f"TFLOP/s ({fmt})", "frac": ach / peak,
            "traffic": traffic, "traffic_unit": "bytes per launch (ncu dram read + write)",
            "flops_per_pair": 2 * k_alg, "k_algorithmic": k_alg,
            "peak_source": ("measured bf16 dense peak of MEASURED_PEAKS.json (fp16 dense rate = bf16)" if f16 else
                            "measured bf16 dense peak of MEASURED_PEAKS.json x 1.1/2.25 (nominal TF32/BF16)"),
            "frac_of_sustained": ach / sus,
            "issued_mma": {"flops_per_pair": fpp_issued, "achieved": fpp_issued * pairs_s / 1e12,
                           "frac": fpp_issued * pairs_s / peak, "frac_of_sustained": fpp_issued * pairs_s / sus},
            "epilogue": {"i_epi": TC_I_EPI, "roof_pairs_per_s": epi_peak, "frac": pairs_s / epi_peak},
            "alu_view": {k: alu[k] for k in ("achieved", "peak", "frac", "fma_lanes_per_pair")}}


def parse():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=WORKLOADS, default="monotone_d4")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the CPU-baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--scan-variant", type=int, default=-1,
                    help="FP32 handles: lip_set_tuning variant (0-7) instead of the autotuned one")
    ap.add_argument("--tc-variant", type=int, default=-1,
                    help="tensor-core handles: lip_set_tuning variant (0-5; -1 keeps the default 0)")
    ap.add_argument("--tc-window-mb", type=int, default=0,
                    help="tensor-core handles: lockstep window in MB (lip_set_tc_window; 0 = default)")
    ap.add_argument("--serial-problems", action="store_true",
                    help="run a step's problems one after another on one stream (default: one stream each)")
    ap.add_argument("--no-tc-vs-plain", action="store_true",
                    help="monotone_d4: skip the tensor-core vs plain comparison on cluster_d16 (after the timed steps)")
    ap.add_argument("--sets", type=int, default=0, help="batch_4096: use only the first N sets (profiling)")
    ap.add_argument("--queries", type=int, default=0,
                    help="use only the first N queries of a single-set workload (small profiling cases)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# ------------------------------------------------------------------ clocks

def out_dir():
    """Where the bench writes its side files (clock samples, the autotune cache it collects):
    $LIPFIT_BENCH_OUT, else bench_out/ at the repository root."""
    return os.environ.get("LIPFIT_BENCH_OUT") or os.path.join(ROOT, "bench_out")


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(out_dir(), f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ multi-rank aggregation

def aggregate(pairs_local: float, ms_local: float, device=None):
    """Whole-job throughput: all ranks' pairs over the slowest rank's time (G pairs/s).

    Single process: pairs / time.  Under torch.distributed the pairs are summed and the
    time is the maximum over ranks (one all_reduce each, on `device`)."""
    import torch
    import torch.distributed as tdist
    if tdist.is_available() and tdist.is_initialized() and tdist.get_world_size() > 1:
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        p = torch.tensor([pairs_local], dtype=torch.float64, device=device)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        tdist.all_reduce(p, op=tdist.ReduceOp.SUM)
        ms_local, pairs_local = float(t.item()), float(p.item())
    return pairs_local / (ms_local / 1e3) / 1e9, ms_local


# ------------------------------------------------------------------ CPU oracle timing

def oracle_rate(problems, seconds: float, rng_seed=5):
    """Pairs/s of the FP64 oracle over random queries of the given problems (one oracle
    call per problem), sized from a 64-query probe to take about `seconds`."""
    import oracle
    o = oracle.default()
    rng = np.random.default_rng(rng_seed)
    p0 = problems[0]
    probe = p0.Q[rng.choice(p0.nq, min(64, p0.nq), replace=False)]
    t0 = time.perf_counter()
    o.evaluate(p0.X, p0.y, probe, p0.M, p0.norm, mon=p0.mon, w=p0.w)
    per_pair = max(time.perf_counter() - t0, 1e-4) / (len(probe) * p0.N)
    budget_pairs = seconds / per_pair
    pairs, dt = 0, 0.0
    for p in problems:
        nq = int(max(16, min(p.nq, budget_pairs / len(problems) / p.N)))
        Qs = p.Q[rng.choice(p.nq, nq, replace=False)]
        t0 = time.perf_counter()
        o.evaluate(p.X, p.y, Qs, p.M, p.norm, mon=p.mon, w=p.w)
        dt += time.perf_counter() - t0
        pairs += nq * p.N
    return {"value": pairs / dt / 1e9, "unit": UNIT, "cores": oracle.default_threads(), "kind": "oracle",
            "sample": f"{pairs:.3g} pairs: random queries x all data points of {len(problems)} problem(s) "
                      f"(FP64, {oracle.default_threads()} threads, {dt:.1f} s)"}, dt


def oracle_local_rate(p, seconds: float, n_sub: int = 20_000, rng_seed=5):
    """Pairs/s of the FP64 oracle's local evaluation (Sec. 4.3) over random queries against
    the first n_sub data points, with the oracle's own table for those points (built
    before the timed part; its rate is reported in the sample text)."""
    import oracle
    o = oracle.default()
    X, y = p.X[:n_sub].astype(np.float64), p.y[:n_sub].astype(np.float64)
    t0 = time.perf_counter()
    T, _, _ = o.local_knots(X, LOCAL_KNOTS, LOCAL_SAMPLE, LOCAL_SEED, p.norm, w=p.w)
    tab = o.local_table(X, y, T, p.norm, w=p.w)
    t_tab = time.perf_counter() - t0
    rng = np.random.default_rng(rng_seed)
    probe = p.Q[rng.choice(p.nq, 64, replace=False)]
    t0 = time.perf_counter()
    o.evaluate_local(X, y, probe, T, tab, p.norm, w=p.w)
    per_pair = max(time.perf_counter() - t0, 1e-4) / (64 * len(y))
    nq = int(max(64, min(p.nq, seconds / per_pair / len(y))))
    Qs = p.Q[rng.choice(p.nq, nq, replace=False)]
    t0 = time.perf_counter()
    o.evaluate_local(X, y, Qs, T, tab, p.norm, w=p.w)
    dt = time.perf_counter() - t0
    pairs = nq * len(y)
    return {"value": pairs / dt / 1e9, "unit": UNIT, "cores": oracle.default_threads(), "kind": "oracle",
            "sample": f"{pairs:.3g} pairs: {nq} random queries x the first {len(y)} data points, local constants "
                      f"from the oracle's table of those points ({len(y)}^2 pairs in {t_tab:.1f} s, untimed); "
                      f"FP64, {oracle.default_threads()} threads, {dt:.1f} s"}, dt


def reference_problems(workload):
    if workload == "monotone_d4":
        base = W.monotone_d4(norm=W.NORM_L2)
        return [base.with_norm(n) for n in NORMS]
    if workload == "plain_d2":
        return [W.plain_d2(dtype=np.float64)]
    if workload in ("cluster_d16", "cluster_d16_tc", "cluster_d16_bf16", "cluster_d16_fp16"):
        return [W.cluster_d16(n_query=20_000)]
    if workload == "grad_d8":
        return [W.grad_d8()]
    plan = W.batch_plan()
    rng = np.random.default_rng(3)
    out = []
    for k in rng.choice(len(plan), 48, replace=False):
        bs = plan[k]
        X, y, Q, f = W.batch_set_data(bs)
        out.append(W.Problem("batch", X, y, Q, bs.M, bs.norm, bs.mon, None, f))
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    per_step = max(2.0, min(8.0, 60.0 / max(1, args.steps + args.warmup)))
    if args.workload == "local_d4":
        problems = W.local_d4()
        rate = lambda sec: oracle_local_rate(problems, sec)  # noqa: E731
    elif args.workload == "smooth_d4":
        problems = W.smooth_d4()
        rate = lambda sec: oracle_smooth_rate(problems, sec)  # noqa: E731
    else:
        problems = reference_problems(args.workload)
        rate = lambda sec: oracle_rate(problems, sec)  # noqa: E731
    for _ in range(args.warmup):
        rate(per_step / 4)
    rates, times, base = [], [], None
    for _ in range(args.steps):
        base, dt = rate(per_step)
        rates.append(base["value"])
        times.append(dt)
    value = statistics.mean(rates)
    base = dict(base, value=value)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": f"synthetic (seeded, {args.workload} workload)", "config": {"workload": args.workload},
            "cpu_baseline": base,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm helpers

class Ctx:
    def __init__(self, args):
        import torch
        self.args = args
        self.rank, self.world, self.local = dist_env()
        self.torch = torch
        props = torch.cuda.get_device_properties(self.local)
        self.sms = props.multi_processor_count
        try:
            self.peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except Exception:
            self.peaks = {}
        self.sm_max = float(self.peaks.get("sm_max_mhz", 2032.0))
        self.flush_buf = torch.empty(64 << 20, dtype=torch.float32, device="cuda")    # 256 MB > L2

    def flush(self):
        self.flush_buf.fill_(1.0)

    def timed(self, step, steps, flush=True):
        """Per-step CUDA-event times of `steps` calls of step(), with clocks sampled during
        the timed region and the library's kernel launches counted."""
        from paper_2606_04670_b300 import lipfit as L
        torch = self.torch
        torch.cuda.synchronize()
        if self.world > 1:
            torch.distributed.barrier()
        sampler = ClockSampler(self.local)
        sampler.start()
        launches0 = L.lip_kernel_launches()
        ms = []
        for _ in range(steps):
            if flush:
                self.flush()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            step()
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        torch.cuda.synchronize()
        if self.world > 1:
            torch.distributed.barrier()
        return ms, sampler.stop(), L.lip_kernel_launches() - launches0

    def roofline(self, kernel, pairs_per_launch, ms_per_launch, ipair, mufu, clocks, traffic=None, fma=None):
        """Roofline of an all-pairs ALU kernel.  Two pipes can bind: the FP32 FMA pipe (fma
        algorithmic lane operations per pair against SMs x 128 lanes x clock) and the
        special-function pipe MUFU (mufu square roots per pair against SMs x 16 x clock).
        frac is the larger of the two fractions and `pipe` names it.  The survey's scalar
        count of all FP32 lane operations per pair (ipair, FMA and ALU pipes together)
        is kept as `lane_ops_view`; packed f32x2 and three-input min / max instructions let
        that count exceed 1.0 of the FMA pipe's lane peak, so it is not the fraction."""
        pairs_s = pairs_per_launch / (ms_per_launch / 1e3)
        lane_peak = self.sms * FP32_LANES_PER_SM * self.sm_max * 1e6
        src = f"(max SM clock{' of MEASURED_PEAKS.json' if self.peaks else ', nominal'})"
        fma = ipair if fma is None else fma
        fma_ach = pairs_s * fma
        r = {"bound": "alu", "kernel": kernel, "pipe": "fma", "achieved": fma_ach / 1e12, "peak": lane_peak / 1e12,
             "unit": "T lane ops/s (FP32 FMA pipe)", "frac": fma_ach / lane_peak, "traffic": traffic,
             "traffic_unit": "bytes per launch (ncu dram read + write)",
             "peak_source": f"{self.sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {self.sm_max:.0f} MHz {src}",
             "fma_lanes_per_pair": fma, "mufu_per_pair": mufu,
             "fma_pipe": {"achieved": fma_ach / 1e12, "peak": lane_peak / 1e12, "frac": fma_ach / lane_peak},
             "lane_ops_view": {"i_pair": ipair, "achieved": pairs_s * ipair / 1e12, "peak": lane_peak / 1e12,
                               "frac": pairs_s * ipair / lane_peak}}
        if mufu:
            m = self.mufu_bound(pairs_s, mufu)
            r["mufu"] = m
            if m["frac"] > r["frac"]:
                r.update(pipe="mufu", achieved=m["achieved"], peak=m["peak"], unit=m["unit"], frac=m["frac"],
                         peak_source=m["peak_source"])
        if clocks and clocks.get("sm_mhz"):
            r["frac_at_measured_clock"] = r["frac"] * self.sm_max / clocks["sm_mhz"]
        return r

    def mufu_bound(self, pairs_per_s, mufu_per_pair):
        """The special-function (MUFU) pipe as a second bound: square roots per second against
        148 SMs x 16 per clock x the maximum SM clock (a throughput kernel measured 15.0
        sqrt.approx, and as many rsqrt.approx, per SM per clock on the B300s)."""
        peak = self.sms * MUFU_PER_SM * self.sm_max * 1e6
        ach = pairs_per_s * mufu_per_pair
        return {"achieved": ach / 1e12, "peak": peak / 1e12, "unit": "T square roots/s (MUFU)", "frac": ach / peak,
                "per_pair": mufu_per_pair,
                "peak_source": f"{self.sms} SMs x {MUFU_PER_SM} MUFU results x {self.sm_max:.0f} MHz (max SM clock)"}

    def line(self, value, ms_total, steps, dtype, config, roof, cpu, e2e, clocks, launches, detail):
        if self.world == 1:
            par = "single GPU"
        elif config["workload"] == "monotone_d4":
            par = (f"queries sharded over {self.world} GPUs (data replicated; M_est pair tiles block-cyclic, "
                   f"one all_gather per norm)")
        else:
            par = f"replicas{self.world}"
        return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": self.world, "steps": steps,
                "warmup": max(3, self.args.warmup), "ms_per_step": ms_total / steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": dtype,
                "data": f"synthetic (seeded, {config['workload']} workload)",
                "config": dict(config, parallelism=par), "roofline": roof,
                "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": launches, "detail": detail}


def _tune_cache():
    """The autotune cache: the one collected in the output folder (out_dir()) by earlier
    runs, else the committed default.  Saved back to the output folder (copy it to the
    default to keep it)."""
    from paper_2606_04670_b300 import autotune as AT
    local = os.path.join(out_dir(), "autotune_cache.json")
    cache = AT.load_cache(local) if os.path.exists(local) else AT.load_cache()
    return cache, (lambda: AT.save_cache(cache, local))


def _cpu(ctx, problems):
    if ctx.rank != 0 or ctx.args.no_cpu_baseline:
        return None
    return oracle_rate(problems, ctx.args.cpu_seconds)[0]


# ------------------------------------------------------------------ workloads

def wl_single(ctx, name, problems, precisions=("fp32",), with_est=True, with_bwd=False, flush=True):
    """fit + eval (+ M_est) (+ backward) of each problem per step."""
    from paper_2606_04670_b300 import lipfit as L
    from paper_2606_04670_b300 import shard as S
    torch, args = ctx.torch, ctx.args
    if args.queries > 0:
        problems = [p.sub_queries(args.queries) for p in problems]
    runs = []
    for p in problems:
        for prec in precisions:
            dt = torch.float64 if prec == "fp64" else torch.float32
            X = torch.as_tensor(p.X).to("cuda", dt)
            y = torch.as_tensor(p.y).to("cuda", dt)
            Q = torch.as_tensor(p.Q).to("cuda", dt)
            m = L.LipFit(M=p.M, norm=p.norm, mon=p.mon, w=p.w, capacity=p.N, d=p.d, precision=prec)
            if prec.startswith("tc_"):
                if args.tc_variant >= 0:
                    m.set_tuning(0, 0, args.tc_variant)
                m.set_tc_window(args.tc_window_mb << 20)
            elif prec == "fp32" and args.scan_variant >= 0:
                m.set_tuning(0, 0, args.scan_variant)
            ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            m.set_timing_events(*ev)
            runs.append(dict(p=p, prec=prec, X=X, y=y, Q=Q, m=m, ev=ev, scan=[], bwd=[],
                             bev=(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)),
                             gb=torch.ones(p.nq, device="cuda", dtype=dt)))
    tuning = {}
    if not args.no_autotune:
        from paper_2606_04670_b300 import autotune as AT
        cache, save = _tune_cache()
        for r in runs:
            if r["prec"].startswith("tc_") or (r["prec"] == "fp32" and args.scan_variant >= 0):
                continue               # the launch shape knobs belong to the plain scan (or are set)
            r["m"].clear()
            r["m"].add(r["X"], r["y"])
            tuning[f"{NNAME[r['p'].norm]}/{r['prec']}"] = AT.tune_eval(r["m"], r["Q"], cache=cache)
        save()
    est = {}
    # One stream per problem on one GPU: the problems of a step are independent, so their
    # kernels run side by side (one scan's last wave overlaps the next problem's start, and
    # the small latency-bound kernels overlap the others' scans); the estimates are queued
    # with lip_estimate_M_async and read once everything is queued.
    side = [torch.cuda.Stream() for _ in runs] if len(runs) > 1 and ctx.world == 1 and not args.serial_problems \
        else None

    def step(record=False, serial=False):
        main = torch.cuda.current_stream()
        streams = None if serial else side
        for k, r in enumerate(runs):
            s = streams[k] if streams else main
            if streams:
                s.wait_stream(main)
            with torch.cuda.stream(s):
                m = r["m"]
                m.clear()
                m.add_async(r["X"], r["y"])       # the finiteness check reported by check() below
                out = m.eval(r["Q"], need=("g", "lo", "hi", "idx_up", "idx_lo"))
                if with_bwd:
                    r["bev"][0].record()
                    m.backward(r["Q"], out["idx_up"], out["idx_lo"], r["gb"])
                    r["bev"][1].record()
                if with_est:
                    if ctx.world > 1:
                        # the pair triangle shared out over the GPUs, one all_gather per norm
                        est[k] = S.estimate_M_sharded(S.DeviceShard(m, 0), device="cuda")[0]
                    else:
                        m.lipschitz_constant_async()
        if with_est and ctx.world == 1:
            for k, r in enumerate(runs):
                est[k] = r["m"].lipschitz_constant_result()[0]
        if streams:
            for s in streams:
                main.wait_stream(s)
        for r in runs:
            r["m"].check()
        if record:
            torch.cuda.synchronize()
            for r in runs:
                r["scan"].append(r["ev"][0].elapsed_time(r["ev"][1]))
                if with_bwd:
                    r["bwd"].append(r["bev"][0].elapsed_time(r["bev"][1]))

    for _ in range(max(3, args.warmup)):
        step()
    ms, clocks, launches = ctx.timed(lambda: step(True), args.steps, flush=flush)
    concurrent_scan_ms = {}
    if side:
        # The scans' own durations for the roofline come from steps with the problems one
        # after another on one stream (the same kernels, nothing beside them); those of
        # the timed steps, shared with the other problems' kernels, are reported as well.
        concurrent_scan_ms = {f"{NNAME[r['p'].norm]}/{r['prec']}": statistics.mean(r["scan"]) for r in runs}
        for r in runs:
            r["scan"].clear()
            r["bwd"].clear()
        for _ in range(max(3, min(args.steps, 5))):
            if flush:
                ctx.flush()
            step(True, serial=True)
    pairs_step = sum(r["p"].nq * r["p"].N for r in runs)
    value, total = aggregate(pairs_step * args.steps, sum(ms), device="cuda")
    # dominant kernel: the scan with the largest average time
    avg = [statistics.mean(r["scan"]) for r in runs]
    kdom = int(np.argmax(avg))
    rd = runs[kdom]
    p = rd["p"]
    c = 0 if p.mon is None else int((np.asarray(p.mon) != 0).sum())
    ip = i_pair(p.norm, p.d, c)
    exact = rd["prec"] in ("fp32", "fp64") and (p.d <= 10 or c == 0)
    kern = (f"scan_{'exact' if exact else 'generic'}_kernel<{NNAME[p.norm]}, C={c}, U={p.d - c}, "
            f"R={rd['m'].tuning()['queries_per_thread']}> {rd['prec']}")
    if rd["prec"] == "fp64":
        kern = "FP32 screen " + kern.replace(" fp64", "") + " + screen64_kernel (FP64 candidates)"
    # the pruned scan (variants 6, 7) evaluates only the (32-query row, 32-point chunk) pairs
    # its bound test keeps: its roofline counts the pairs it evaluated, the whole pair space
    # stays in value
    tun_dom = rd["m"].tuning()
    evaluated, wtotal = rd["m"].last_scan_work() if rd["prec"] == "fp32" else (-1, -1)
    share = evaluated / wtotal if wtotal > 0 and evaluated >= 0 else 1.0
    if wtotal > 0:
        kern = (f"scan_pruned_kernel<{NNAME[p.norm]}, C={c}, U={p.d - c}, R={tun_dom['queries_per_thread']}> fp32 "
                f"(variant {tun_dom['variant']})")
    roof = ctx.roofline(kern, p.nq * p.N * share, avg[kdom], ip, mufu_per_pair(p.norm, c), clocks,
                        traffic_for(args, name, p.norm, pruned=wtotal > 0) if rd["prec"] == "fp32" else None,
                        fma=fma_lanes_per_pair(p.norm, p.d, c))
    if wtotal > 0:
        roof["pruned"] = {"evaluated_row_chunks": evaluated, "row_chunks": wtotal, "evaluated_share": share,
                          "pairs_per_s_whole_space": p.nq * p.N / (avg[kdom] / 1e3),
                          "note": "achieved counts the pairs of the evaluated (row, chunk) blocks (share x Q x N); "
                                  "the per-chunk bound tests are not counted"}
    if rd["prec"] in ("tc_tf32", "tc_bf16", "tc_fp16"):
        roof = tc_roofline(ctx, rd["prec"], p.d, p.nq * p.N, avg[kdom], roof, traffic_for(args, name, p.norm))

    e2e = None
    if not args.no_e2e:
        hostruns = []
        for r in runs:
            ndt = np.float64 if r["prec"] == "fp64" else np.float32
            hX, hy, hQ = (torch.as_tensor(np.ascontiguousarray(a, dtype=ndt)).pin_memory()
                          for a in (r["p"].X, r["p"].y, r["p"].Q))
            hdt = torch.float64 if r["prec"] == "fp64" else torch.float32
            outs = {k: torch.empty(r["p"].nq, dtype=hdt).pin_memory() for k in ("g", "lo", "hi")}
            outs.update({k: torch.empty(r["p"].nq, dtype=torch.int32).pin_memory() for k in ("idx_up", "idx_lo")})
            hostruns.append((r, hX, hy, hQ, outs))
            r["m"].set_timing_events(None, None)

        def step_host():
            # every problem's fit, evaluation and estimate queued first, each on its own
            # stream as in the device step (lip_eval_host_async: the copies of one overlap
            # the kernels of another), then the estimates' results, then lip_check, which
            # also waits for the host-path copies
            main = torch.cuda.current_stream()
            for k, (r, hX, hy, hQ, outs) in enumerate(hostruns):
                s = side[k] if side else main
                if side:
                    s.wait_stream(main)
                with torch.cuda.stream(s):
                    m = r["m"]
                    m.clear()
                    m.add_host_async(hX, hy)
                    m.eval_host(hQ, outs, wait=False)
                    if with_est and ctx.world == 1:
                        m.lipschitz_constant_async()
            if with_est:
                for r, *_ in hostruns:
                    if ctx.world > 1:
                        S.estimate_M_sharded(S.DeviceShard(r["m"], 0), device="cuda")
                    else:
                        r["m"].lipschitz_constant_result()
            if side:
                for s in side:
                    main.wait_stream(s)
            for r, *_ in hostruns:
                r["m"].check()

        step_host()
        torch.cuda.synchronize()
        e2e_ms = []
        for _ in range(args.steps):
            if flush:
                ctx.flush()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            step_host()
            torch.cuda.synchronize()
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
        ev_, tot = aggregate(pairs_step * args.steps, sum(e2e_ms), device="cuda")
        h2d = sum(hX.numel() * hX.element_size() + hy.numel() * hy.element_size() + hQ.numel() * hQ.element_size()
                  for _, hX, hy, hQ, _ in hostruns)
        d2h = sum(sum(t.numel() * t.element_size() for t in o.values()) + (24 if with_est else 0)
                  for *_, o in hostruns)
        e2e = {"value": ev_, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": tot / args.steps}
        if with_bwd:
            e2e["note"] = "host path covers fit + eval (+ M_est); the backward pass is device-only"

    cpu = _cpu(ctx, [r["p"] for r in runs])
    tun = rd["m"].tuning()
    key = lambda r: f"{NNAME[r['p'].norm]}/{r['prec']}"  # noqa: E731
    detail = {"scan_ms": {key(r): statistics.mean(r["scan"]) for r in runs},
              "problems_concurrent": bool(side),
              "scan_ms_concurrent": concurrent_scan_ms,
              "scan_gpairs_per_s": {key(r): r["p"].nq * r["p"].N / (statistics.mean(r["scan"]) / 1e3) / 1e9
                                    for r in runs},
              "splits": tun["last_splits"], "tile_groups": tun["tile_groups"],
              "queries_per_thread": tun["queries_per_thread"], "sms": ctx.sms, "autotune": tuning,
              "tc_fallback_queries": {key(r): r["m"].last_fallback() for r in runs if r["prec"].startswith("tc_")},
              "tc_variant": {key(r): r["m"].tuning()["variant"] for r in runs if r["prec"].startswith("tc_")},
              "tc_window_mb": args.tc_window_mb or 32}
    if with_bwd:
        # backward (one launch): per query it reads q, both indices and grad_g, gathers the
        # two chosen data rows, writes grad_q and adds to grad_y (two atomic read-modify-
        # writes); the binding zeroes grad_y [N] first
        bb = {}
        for r in runs:
            pp = r["p"]
            es = 8 if r["prec"] == "fp64" else 4
            byts = pp.nq * (pp.d * es + 8 + es + 2 * pp.d * es + pp.d * es + 4 * es) + pp.N * es
            ms_b = statistics.mean(r["bwd"])
            bb[key(r)] = {"ms": ms_b, "algorithmic_bytes": byts, "gb_per_s": byts / (ms_b / 1e3) / 1e9,
                          "hbm_peak_gb_per_s": float(ctx.peaks.get("hbm_gbs", 6518.0)),
                          "frac_of_hbm": byts / (ms_b / 1e3) / 1e9 / float(ctx.peaks.get("hbm_gbs", 6518.0))}
        detail["backward"] = bb
    if with_est:
        detail["M_est"] = {key(r): est[k] for k, r in enumerate(runs)}
        detail["M_true"] = {key(r): r["p"].M for r in runs}
        # the pruned estimate's screen: tile pairs entered, (warp, chunk) pairs evaluated, total
        detail["estimate_work"] = {key(r): r["m"].last_estimate_work() for r in runs}
    # the pruned scan's evaluated share of its (row, chunk) pairs and the share of the data
    # tiles its blocks copied, per norm
    shares, tiles, raw = {}, {}, {}
    for r in runs:
        if r["prec"] == "fp32":
            st = r["m"].last_scan_stats()
            if st[1] > 0:
                shares[key(r)] = st[0] / st[1]
                tiles[key(r)] = st[2] / st[3]
                raw[key(r)] = st
    detail["pruned_scan_share"] = shares
    detail["pruned_tiles_copied_share"] = tiles
    # [evaluated (row, chunk), all (row, chunk), tiles copied, blocks x tiles, (warp, chunk) past the warp-box test]
    detail["pruned_scan_stats"] = raw
    for r in runs:
        r["m"].close()
    if name == "monotone_d4" and not args.no_tc_vs_plain and ctx.world == 1:
        detail["tc_vs_plain"] = tc_vs_plain(ctx)
    p0 = problems[0]
    config = {"workload": name, "d": p0.d, "N": p0.N, "Q": p0.nq,
              "mon": None if p0.mon is None else [int(v) for v in p0.mon],
              "norms": [NNAME[p.norm] for p in problems], "precisions": list(precisions),
              "step": "per problem: fit + eval" + (" + M_est" if with_est else "") + (" + backward" if with_bwd else "")
                      + ("; the problems side by side, one stream each" if side else ""),
              "l2": "flushed before every timed step (256 MB write)" if flush else "inputs larger than L2"}
    return ctx.line(value, total, args.steps, "f64" if precisions == ("fp64",) else "f32", config, roof, cpu, e2e,
                    clocks, launches, detail)


TC_FORMS = ("fp32", "tc_tf32", "tc_bf16", "tc_fp16")
# the comparison's forms: the plain FP32 scan (default launch), the pruned FP32 scan
# (variant 7) and the three tensor-core forms
CMP_FORMS = ("fp32", "fp32_pruned", "tc_tf32", "tc_bf16", "tc_fp16")


def tc_vs_plain(ctx, n_oracle=192, reps=3):
    """The tensor-core L2 forms against the plain FP32 scan (its default launch and the pruned
    scan) on the precision workload at full
    size (cluster_d16: d = 16, N = Q = 1e6, 32-cluster Gaussian mixture), measured in this
    process: per form the whole lip_eval call and its scan kernel alone (CUDA events, best of
    `reps` after a warm-up), the queries the tensor-core form sent to the plain fallback, and
    the clocks.  Accuracy: the FP64 oracle, timed on the host cores as this comparison's CPU
    baseline, evaluates n_oracle random queries against all 1e6 points; every form's g, lo,
    hi are compared with it (max error over M * diam, the tolerance 1e-5) and its indices
    wherever the oracle's gap exceeds the tolerance."""
    from paper_2606_04670_b300 import lipfit as L
    torch = ctx.torch
    p = W.cluster_d16()
    X, y, Q = (torch.as_tensor(a).cuda() for a in (p.X, p.y, p.Q))
    rng = np.random.default_rng(11)
    sample = np.sort(rng.choice(p.nq, n_oracle, replace=False))
    lo_c = np.minimum(p.X.min(0), p.Q.min(0)).astype(np.float64)
    hi_c = np.maximum(p.X.max(0), p.Q.max(0)).astype(np.float64)
    scale = p.M * float(np.sqrt(((hi_c - lo_c) ** 2).sum()))
    tol = 1e-5 * scale
    sampler = ClockSampler(ctx.local)
    sampler.start()
    forms = {}
    outs = {}
    for prec in CMP_FORMS:
        m = L.LipFit(X, y, p.M, norm=p.norm, precision="fp32" if prec == "fp32_pruned" else prec)
        if prec == "fp32_pruned":
            m.set_tuning(0, 0, 7)
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r = m.eval(Q)                      # warm-up (tensor-core tiles built here)
        m.set_timing_events(*ev)
        t_eval, t_scan = [], []
        for _ in range(reps):
            torch.cuda.synchronize()
            a.record()
            r = m.eval(Q)
            b.record()
            torch.cuda.synchronize()
            t_eval.append(a.elapsed_time(b))
            t_scan.append(ev[0].elapsed_time(ev[1]))
        m.check()
        outs[prec] = {k: v[torch.as_tensor(sample).cuda()].cpu().numpy() for k, v in r.items()}
        forms[prec] = {"eval_ms": min(t_eval), "scan_ms": min(t_scan),
                       "gpairs_per_s": p.nq * p.N / (min(t_eval) / 1e3) / 1e9,
                       "scan_gpairs_per_s": p.nq * p.N / (min(t_scan) / 1e3) / 1e9}
        if prec.startswith("tc_"):
            forms[prec]["fallback_queries"] = m.last_fallback()
        m.close()
        del r
    clocks = sampler.stop()
    # the FP64 oracle on the sample: this comparison's CPU baseline and its accuracy reference
    import oracle
    o = oracle.default()
    t0 = time.perf_counter()
    ref = o.evaluate(p.X, p.y, p.Q[sample], p.M, p.norm)
    dt = time.perf_counter() - t0
    for prec in CMP_FORMS:
        g = outs[prec]
        err = {k: float(np.max(np.abs(g[k].astype(np.float64) - ref[k]))) for k in ("g", "lo", "hi")}
        mism = 0
        for k, gk in (("idx_up", "gap_up"), ("idx_lo", "gap_lo")):
            mism += int(np.sum((ref[gk] > tol) & (g[k].astype(np.int64) != ref[k])))
        forms[prec].update(max_abs_err=err, max_err_over_M_diam=max(err.values()) / scale,
                           index_mismatches_above_gap=mism, within_tol=bool(max(err.values()) <= tol and mism == 0))
    base = forms["fp32"]["eval_ms"]
    return {"workload": "cluster_d16", "d": p.d, "N": p.N, "Q": p.nq, "norm": "L2", "M": p.M,
            "tolerance": "1e-5 * M * diam", "tol_abs": tol, "oracle_queries": n_oracle,
            "forms": forms, "speedup_vs_fp32": {k: base / v["eval_ms"] for k, v in forms.items()},
            "clocks": clocks,
            "cpu_baseline": {"value": n_oracle * p.N / dt / 1e9, "unit": UNIT, "cores": oracle.default_threads(),
                             "kind": "oracle", "sample": f"{n_oracle} random queries x all {p.N} data points "
                                                         f"(FP64, {dt:.1f} s)"}}


def wl_batch(ctx):
    from paper_2606_04670_b300 import lipfit as L
    torch, args = ctx.torch, ctx.args
    plan = W.batch_plan()
    if args.sets > 0:
        plan = plan[:args.sets]
    sets_np = [W.batch_set_data(bs) for bs in plan]
    qoff = np.concatenate([[0], np.cumsum([bs.nq * bs.d for bs in plan])])
    noff = np.concatenate([[0], np.cumsum([bs.nq for bs in plan])])
    hQ = torch.empty(int(qoff[-1]), dtype=torch.float32).pin_memory()
    for k, (X, y, Q, f) in enumerate(sets_np):
        hQ[int(qoff[k]):int(qoff[k + 1])] = torch.from_numpy(Q.reshape(-1))
    dQ = hQ.to("cuda")
    tq = int(noff[-1])
    dout = {k: torch.empty(tq, device="cuda") for k in ("g", "lo", "hi")}
    dout.update({k: torch.empty(tq, device="cuda", dtype=torch.int32) for k in ("idx_up", "idx_lo")})
    sets, outs = [], []
    for k, bs in enumerate(plan):
        X, y, Q, f = sets_np[k]
        sets.append(dict(X=torch.as_tensor(X), y=torch.as_tensor(y),
                         Q=dQ[int(qoff[k]):int(qoff[k + 1])].view(bs.nq, bs.d), M=bs.M, norm=bs.norm, mon=bs.mon))
        outs.append({key: v[int(noff[k]):int(noff[k + 1])] for key, v in dout.items()})
    tuning = None
    opts = {}
    if not args.no_autotune:
        from paper_2606_04670_b300 import autotune as AT
        cache, save = _tune_cache()
        tuning = AT.tune_batch(sets, cache=cache, outputs=outs)
        save()
        opts = {k: tuning[k] for k in ("tile_groups", "items_per_block", "waves")}
    b = L.LipBatch(sets, outputs=outs, **opts)
    info = b.info()
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    for _ in range(max(3, args.warmup)):
        b.eval()
    torch.cuda.synchronize()
    b.check()
    stream = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        b.eval()
    graph.replay()
    torch.cuda.synchronize()
    # the persistent scan kernel alone (events recorded by the library around it)
    b.set_timing_events(*ev)
    scan_ms = []
    for _ in range(2):
        b.eval()
        torch.cuda.synchronize()
        scan_ms.append(ev[0].elapsed_time(ev[1]))
    b.set_timing_events(None, None)
    ms, clocks, _ = ctx.timed(graph.replay, args.steps, flush=False)
    launches = 2 * args.steps      # each replay runs the persistent scan and the batched merge
    value, total = aggregate(info["total_pairs"] * args.steps, sum(ms), device="cuda")
    ops = fma = mufu = 0.0
    for bs in plan:
        c = int((bs.mon != 0).sum())
        ops += bs.nq * bs.N * i_pair(bs.norm, bs.d, c)
        fma += bs.nq * bs.N * fma_lanes_per_pair(bs.norm, bs.d, c)
        mufu += bs.nq * bs.N * mufu_per_pair(bs.norm, c)
    tp = info["total_pairs"]
    roof = ctx.roofline("batch_scan_kernel (persistent, 4096 sets)", tp, min(scan_ms), ops / tp, mufu / tp, clocks,
                        traffic_for(args, "batch_4096", 0), fma=fma / tp)
    e2e = None
    if not args.no_e2e:
        hout = {k: torch.empty(tq, dtype=v.dtype).pin_memory() for k, v in dout.items()}
        e2e_ms = []
        for _ in range(args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dQ.copy_(hQ, non_blocking=True)
            graph.replay()
            for k in hout:
                hout[k].copy_(dout[k], non_blocking=True)
            torch.cuda.synchronize()
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
        ev_, tot = aggregate(info["total_pairs"] * args.steps, sum(e2e_ms), device="cuda")
        e2e = {"value": ev_, "unit": UNIT, "h2d_bytes_per_step": hQ.numel() * 4,
               "d2h_bytes_per_step": sum(t.numel() * t.element_size() for t in hout.values()),
               "ms_per_step": tot / args.steps,
               "note": "per step: all sets' queries host->device, graph replay, all outputs device->host"}
    cpu = None
    if ctx.rank == 0 and not args.no_cpu_baseline:
        cpu = oracle_rate(reference_problems("batch_4096"), args.cpu_seconds)[0]
    b.close()
    config = {"workload": "batch_4096" if len(plan) == 4096 else f"batch_4096 (first {len(plan)} sets)", "sets": len(plan), "N": "log-uniform [64, 65536]", "d": "uniform {2..10}",
              "Q": "log-uniform [1e3, 1e5] per set", "total_pairs": info["total_pairs"],
              "total_queries": info["total_queries"], "norms": ["L1", "L2"],
              "step": "one CUDA-graph replay: persistent scan over the work list + batched merge",
              "l2": "inputs larger than L2 (about 3 GB of data, layout and queries)"}
    detail = {"scan_ms": min(scan_ms), "items": info["items"], "grid": info["grid"], "sms": ctx.sms,
              "autotune": tuning}
    return ctx.line(value, total, args.steps, "f32", config, roof, cpu, e2e, clocks, launches, detail)


def wl_local(ctx, name="local_d4"):
    """Local Lipschitz constants (Sec. 4.3): per step, fit + compute_local_lipschitz (knot
    sample, exact table: one N^2 screening scan with candidate lists) + the local evaluation of
    every query."""
    from paper_2606_04670_b300 import lipfit as L
    torch, args = ctx.torch, ctx.args
    p = W.local_d4()
    if args.queries > 0:
        p = p.sub_queries(args.queries)
    X, y, Q = (torch.as_tensor(a).cuda() for a in (p.X, p.y, p.Q))
    m = L.LipFit(M=p.M, norm=p.norm, capacity=p.N, d=p.d)
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    tev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    m.set_timing_events(*ev)
    scan, table = [], []

    def step(record=False):
        m.clear()
        m.add(X, y)
        tev[0].record()
        m.compute_local_lipschitz(LOCAL_KNOTS, LOCAL_SAMPLE, LOCAL_SEED)
        tev[1].record()
        m.eval_local(Q)
        if record:
            torch.cuda.synchronize()
            scan.append(ev[0].elapsed_time(ev[1]))
            table.append(tev[0].elapsed_time(tev[1]))

    for _ in range(max(3, args.warmup)):
        step()
    ms, clocks, launches = ctx.timed(lambda: step(True), args.steps)
    value, total = aggregate(p.nq * p.N * args.steps, sum(ms), device="cuda")
    ms_scan, ms_table = statistics.mean(scan), statistics.mean(table)
    # local scan per pair: distance 2d, knot search 5 x (compare + add), first-segment test and
    # select, two FMAs, two (compare + two selects) for the running extrema; one MUFU sqrt
    ip = 2 * p.d + 20
    # on the FMA pipe: the differences and squares (2d) and the two bound FMAs
    roof = ctx.roofline(f"loc_scan_kernel<{NNAME[p.norm]}> (d={p.d}, {LOCAL_KNOTS} knots)", p.nq * p.N,
                        ms_scan, ip, 1 if p.norm == W.NORM_L2 else 0, clocks,
                        traffic_for(args, name, p.norm), fma=2 * p.d + 2)
    e2e = None
    if not args.no_e2e:
        hX, hy, hQ = (torch.as_tensor(a).pin_memory() for a in (p.X, p.y, p.Q))
        outs = {k: torch.empty(p.nq, dtype=torch.float32).pin_memory() for k in ("g", "lo", "hi")}
        outs.update({k: torch.empty(p.nq, dtype=torch.int32).pin_memory() for k in ("idx_up", "idx_lo")})
        m.set_timing_events(None, None)
        dQ = torch.empty_like(Q)

        def step_host():
            m.clear()
            m.add_host(hX, hy)
            m.compute_local_lipschitz(LOCAL_KNOTS, LOCAL_SAMPLE, LOCAL_SEED)
            dQ.copy_(hQ, non_blocking=True)
            out = m.eval_local(dQ)
            for k, v in out.items():
                outs[k].copy_(v, non_blocking=True)

        step_host()
        torch.cuda.synchronize()
        e2e_ms = []
        for _ in range(args.steps):
            ctx.flush()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            step_host()
            torch.cuda.synchronize()
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
        ev_, tot = aggregate(p.nq * p.N * args.steps, sum(e2e_ms), device="cuda")
        e2e = {"value": ev_, "unit": UNIT, "ms_per_step": tot / args.steps,
               "h2d_bytes_per_step": sum(t.numel() * t.element_size() for t in (hX, hy, hQ)),
               "d2h_bytes_per_step": sum(t.numel() * t.element_size() for t in outs.values())}
    cpu = None
    if ctx.rank == 0 and not args.no_cpu_baseline:
        cpu = oracle_local_rate(p, args.cpu_seconds)[0]
    knots = m.local_knots()
    over, longest = m.local_stats()
    detail = {"table_ms": ms_table, "scan_ms": ms_scan,
              "scan_gpairs_per_s": p.nq * p.N / (ms_scan / 1e3) / 1e9,
              "table_gpairs_per_s": 1.0 * p.N * p.N / (ms_table / 1e3) / 1e9,
              "table_overflow_rows": over, "table_longest_list": longest,
              "knots": [float(v) for v in knots], "splits": m.tuning()["last_splits"], "sms": ctx.sms}
    m.close()
    config = {"workload": name, "d": p.d, "N": p.N, "Q": p.nq, "mon": None, "norms": [NNAME[p.norm]],
              "knots": LOCAL_KNOTS, "sample_pairs": LOCAL_SAMPLE,
              "step": "fit + local table (knot sample, N^2 screening scan with candidate lists) + local eval "
                      "of all queries",
              "l2": "flushed before every timed step (256 MB write)"}
    return ctx.line(value, total, args.steps, "f32", config, roof, cpu, e2e, clocks, launches, detail)


def oracle_smooth_rate(p, seconds: float, rng_seed=5):
    """Pairs/s of the FP64 oracle's smoothing objective and gradient (Eq. (optim)) on the
    first n points of the workload, n sized so one evaluation takes about `seconds`."""
    import oracle
    o = oracle.default()
    n = 2000
    t0 = time.perf_counter()
    eps = np.zeros(n)
    o.smooth_objective(p.X[:n], p.y[:n], eps, W.SMOOTH_M, W.SMOOTH_P, p.norm)
    per_pair = max(time.perf_counter() - t0, 1e-4) / (n * (n - 1))
    n = int(min(p.N, max(2000, np.sqrt(seconds / per_pair))))
    eps = 0.02 * np.random.default_rng(rng_seed).standard_normal(n)
    t0 = time.perf_counter()
    o.smooth_objective(p.X[:n], p.y[:n], eps, W.SMOOTH_M, W.SMOOTH_P, p.norm)
    dt = time.perf_counter() - t0
    pairs = n * (n - 1)
    return {"value": pairs / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{pairs:.3g} ordered pairs: one objective and gradient evaluation on the first {n} data "
                      f"points (FP64, single thread, {dt:.1f} s)"}, dt


def wl_smooth(ctx, name="smooth_d4"):
    """Penalty smoothing (Sec. 4.4): per step, fit + lip_smooth with a fixed SMOOTH_ITERS
    L-BFGS iterations (gtol 0).  value = ordered data pairs x objective evaluations / time."""
    from paper_2606_04670_b300 import lipfit as L
    torch, args = ctx.torch, ctx.args
    p = W.smooth_d4()
    X, y = (torch.as_tensor(a).cuda() for a in (p.X, p.y))
    m = L.LipFit(M=p.M, norm=p.norm, capacity=p.N, d=p.d)
    evals = []

    def step():
        m.clear()
        m.add(X, y)
        _, _, _, ev = m.smooth_lipschitz(W.SMOOTH_M, W.SMOOTH_P, max_iter=SMOOTH_ITERS, gtol=0.0)
        evals.append(ev)

    for _ in range(max(3, args.warmup)):
        step()
    evals.clear()
    ms, clocks, launches = ctx.timed(step, args.steps)
    pairs = float(p.N) * (p.N - 1)
    value, total = aggregate(pairs * sum(evals), sum(ms), device="cuda")
    # one objective pass alone, on the launching stream, for the roofline
    eps = torch.zeros(p.N, dtype=torch.float64, device="cuda")
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    m.smooth_objective(eps, W.SMOOTH_M, W.SMOOTH_P)
    pass_ms = []
    for _ in range(5):
        ctx.flush()
        torch.cuda.synchronize()
        a.record()
        m.smooth_objective(eps, W.SMOOTH_M, W.SMOOTH_P)
        b.record()
        torch.cuda.synchronize()
        pass_ms.append(a.elapsed_time(b))
    ms_pass = statistics.median(pass_ms)
    # the pass visits each unordered pair once: distance 2d, dz, the two term arguments, their
    # positive and negative parts and the share q, the R - C sum, one FMA for S and one
    # maximum for the vote; one MUFU sqrt
    ip = 2 * p.d + 9
    # on the FMA pipe: the differences and squares (2d), dz, the two term arguments, the
    # R - C sum and the FMA for S
    roof = ctx.roofline(f"smooth_pass_kernel<{NNAME[p.norm]}, DP=4> (+ layout and sums)", pairs / 2, ms_pass, ip,
                        1 if p.norm == W.NORM_L2 else 0, clocks, traffic_for(args, name, p.norm), fma=2 * p.d + 5)
    roof["pairs_per_launch"] = "N (N - 1) / 2 unordered pairs"
    e2e = None
    if not args.no_e2e:
        hX, hy = (torch.as_tensor(a).pin_memory() for a in (p.X, p.y))
        heps = torch.empty(p.N, dtype=torch.float64).pin_memory()
        ev2 = []

        def step_host():
            m.clear()
            m.add_host(hX, hy)
            e, _, _, ev = m.smooth_lipschitz(W.SMOOTH_M, W.SMOOTH_P, max_iter=SMOOTH_ITERS, gtol=0.0)
            heps.copy_(e, non_blocking=True)
            ev2.append(ev)

        step_host()
        torch.cuda.synchronize()
        ev2.clear()
        e2e_ms = []
        for _ in range(args.steps):
            ctx.flush()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            step_host()
            torch.cuda.synchronize()
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
        ev_, tot = aggregate(pairs * sum(ev2), sum(e2e_ms), device="cuda")
        e2e = {"value": ev_, "unit": UNIT, "ms_per_step": tot / args.steps,
               "h2d_bytes_per_step": hX.numel() * 4 + hy.numel() * 4, "d2h_bytes_per_step": heps.numel() * 8}
    cpu = None
    if ctx.rank == 0 and not args.no_cpu_baseline:
        cpu = oracle_smooth_rate(p, min(args.cpu_seconds, 10.0))[0]
    detail = {"objective_pass_ms": ms_pass, "pass_gpairs_per_s": pairs / (ms_pass / 1e3) / 1e9,
              "evaluations_per_step": statistics.mean(evals), "iterations_per_step": SMOOTH_ITERS}
    m.close()
    config = {"workload": name, "d": p.d, "N": p.N, "norms": [NNAME[p.norm]], "M": W.SMOOTH_M, "p": W.SMOOTH_P,
              "step": f"fit + lip_smooth ({SMOOTH_ITERS} L-BFGS iterations, every objective evaluation a pass over "
                      f"all N (N - 1) ordered pairs)",
              "l2": "flushed before every timed step (256 MB write)"}
    return ctx.line(value, total, args.steps, "f32", config, roof, cpu, e2e, clocks, launches, detail)


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        print(json.dumps({"metric": METRIC, "error": "no CUDA device"}), flush=True)
        return 1
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    ctx = Ctx(args)
    w = args.workload
    if w == "monotone_d4":
        # rank r evaluates query block r of the N-GPU query set (block 0 on one GPU)
        base = W.monotone_d4(norm=W.NORM_L2, query_block=rank)
        line = wl_single(ctx, w, [base.with_norm(n) for n in NORMS])
    elif w == "plain_d2":
        line = wl_single(ctx, w, [W.plain_d2(dtype=np.float64)], precisions=("fp32", "fp64"))
    elif w == "cluster_d16":
        line = wl_single(ctx, w, [W.cluster_d16()], with_est=False, flush=False)
    elif w == "cluster_d16_tc":
        line = wl_single(ctx, w, [W.cluster_d16()], precisions=("tc_tf32",), with_est=False, flush=False)
    elif w == "cluster_d16_bf16":
        line = wl_single(ctx, w, [W.cluster_d16()], precisions=("tc_bf16",), with_est=False, flush=False)
    elif w == "cluster_d16_fp16":
        line = wl_single(ctx, w, [W.cluster_d16()], precisions=("tc_fp16",), with_est=False, flush=False)
    elif w == "grad_d8":
        line = wl_single(ctx, w, [W.grad_d8()], with_bwd=True)
    elif w == "local_d4":
        line = wl_local(ctx)
    elif w == "smooth_d4":
        line = wl_smooth(ctx)
    else:
        line = wl_batch(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
