#!/usr/bin/env python
"""Throughput of the fused all-pairs Lipschitz envelope evaluation on a B300.

One step = the whole hot path over one batch of the monotone d=4 workload
(N = 100,000 data points, Q = 1,000,000 queries, increasing in x1 and x2), once per
norm (L1, L2, Linf):
  fit   (lip_clear + lip_add: copy and scan-layout transform, Sec. 5 add())
  eval  (lip_eval: scan kernel + split merge with FP64 re-evaluation, Eq. (upperlower), (eq:g))
  M_est (lip_estimate_M: all-pairs Lipschitz constant, Sec. 5)
Metric: query x datapoint pairs evaluated per second (G pairs/s) = 3 Q N / step time.

Timing: CUDA events per step on the launching stream; L2 (126 MB) is flushed before
every timed step by writing a 256 MB buffer (the inputs, 17.6 MB, are smaller than L2).
N > 1 (torchrun): every rank runs the same per-rank workload on its own GPU (weak
scaling; the method needs no exchange between ranks), value = all ranks' pairs / the
slowest rank's time.

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
# Algorithmic FP32 lane operations per pair for d = 4 with c = 2 constrained coordinates
# (minimal instruction counts, |.| and negation as free operand modifiers, plus 4 for the
# two bounds and the two extrema): L1 2(d-c)+4c+2+4, L2 2(d-c)+5c+2+4, Linf 2(d-c)+3c+2+4.
I_PAIR = {1: 18, 2: 20, 3: 16}
MUFU_PER_PAIR = {1: 0, 2: 2, 3: 0}
FP32_LANES_PER_SM = 128
# dram__bytes_read.sum + dram__bytes_write.sum per launch of the dominant scan kernel, from
# the ncu capture summarised in profiles/scan_exact_l2_monotone_d4.md (set to None whenever
# that kernel changes until it is captured again).
SCAN_DRAM_BYTES = {2: 18.106624e6 + 2.477824e6}
CONFIG = {"workload": "monotone_d4", "d": 4, "N": 100_000, "Q": 1_000_000, "mon": [1, 1, 0, 0],
          "norms": ["L1", "L2", "Linf"], "step": "per norm: fit + eval + M_est",
          "l2": "flushed before every timed step (256 MB write)"}


def parse():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the CPU-baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_bench_{os.getpid()}.csv")

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


# ------------------------------------------------------------------ CPU oracle timing

def oracle_rate(p, norms, seconds: float, rng_seed=5):
    """Pairs/s of the FP64 oracle on a sample of queries sized to take about `seconds`."""
    import oracle
    o = oracle.default()
    rng = np.random.default_rng(rng_seed)
    probe = p.Q[rng.choice(p.nq, 64, replace=False)]
    t0 = time.perf_counter()
    o.evaluate(p.X, p.y, probe, p.M_by_norm[W.NORM_L2], W.NORM_L2, mon=p.mon)
    dt = max(time.perf_counter() - t0, 1e-3)
    per_query = dt / 64
    nq = int(max(64, min(p.nq, seconds / len(norms) / per_query)))
    Qs = p.Q[rng.choice(p.nq, nq, replace=False)]
    t0 = time.perf_counter()
    for n in norms:
        o.evaluate(p.X, p.y, Qs, p.M_by_norm[n], n, mon=p.mon)
    dt = time.perf_counter() - t0
    pairs = nq * p.N * len(norms)
    return {"value": pairs / dt / 1e9, "unit": UNIT, "cores": oracle.default_threads(), "kind": "oracle",
            "sample": f"{nq} random queries x all {p.N} data points x {len(norms)} norms (FP64, "
                      f"{oracle.default_threads()} threads, {dt:.1f} s)"}, dt


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    p = W.monotone_d4(norm=W.NORM_L2)
    per_step = max(2.0, min(8.0, 60.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_rate(p, NORMS, per_step / 4)
    rates, times = [], []
    base = None
    for _ in range(args.steps):
        base, dt = oracle_rate(p, NORMS, per_step)
        rates.append(base["value"])
        times.append(dt)
    value = statistics.mean(rates)
    base = dict(base, value=value)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded, monotone d=4 workload)", "config": CONFIG, "cpu_baseline": base,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


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


# ------------------------------------------------------------------ GPU arm

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
    from paper_2606_04670_b300 import lipfit as L

    p = W.monotone_d4(norm=W.NORM_L2)
    N, d, nq = p.N, p.d, p.nq
    X = torch.as_tensor(p.X).cuda()
    y = torch.as_tensor(p.y).cuda()
    Q = torch.as_tensor(p.Q).cuda()
    models = {n: L.LipFit(M=p.M_by_norm[n], norm=n, mon=p.mon, capacity=N, d=d) for n in NORMS}
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")     # 256 MB > L2
    ev = {n: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for n in NORMS}
    for n in NORMS:
        models[n].set_timing_events(*ev[n])
    scan_ms = {n: [] for n in NORMS}
    est = {}

    def step(record_scan: bool):
        for n in NORMS:
            m = models[n]
            m.clear()
            m.add(X, y)
            r = m.eval(Q)
            if record_scan:
                torch.cuda.synchronize()      # estimate_M syncs anyway; read the scan time now
                scan_ms[n].append(ev[n][0].elapsed_time(ev[n][1]))
            est[n] = m.lipschitz_constant()
        return r

    for _ in range(max(3, args.warmup)):
        step(False)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = L.lip_kernel_launches()
    step_ms = []
    t_wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        step(True)
        b.record()
        torch.cuda.synchronize()
        step_ms.append(a.elapsed_time(b))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall0
    launches = L.lip_kernel_launches() - launches0
    clocks = sampler.stop()
    pairs_step = len(NORMS) * nq * N
    value, total_ms = aggregate(pairs_step * args.steps, sum(step_ms), device="cuda")

    # roofline of the dominant kernel (the scan with the largest time)
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    avg_scan = {n: statistics.mean(v) for n, v in scan_ms.items()}
    dom = max(avg_scan, key=avg_scan.get)
    peak_ops = sms * FP32_LANES_PER_SM * sm_max * 1e6
    achieved = I_PAIR[dom] * nq * N / (avg_scan[dom] / 1e3)
    roof = {"bound": "alu", "kernel": f"scan_exact_kernel<{NNAME[dom]}, C=2, U=2>",
            "achieved": achieved / 1e12, "peak": peak_ops / 1e12, "unit": "Tops/s (FP32 lane ops)",
            "frac": achieved / peak_ops, "traffic": SCAN_DRAM_BYTES.get(dom),
            "traffic_unit": "bytes per launch (ncu dram read + write)",
            "peak_source": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {sm_max:.0f} MHz (max SM clock"
                           f"{' of MEASURED_PEAKS.json' if peaks else ', nominal'})",
            "i_pair": I_PAIR[dom], "mufu_per_pair": MUFU_PER_PAIR[dom]}
    if clocks and clocks.get("sm_mhz"):
        roof["frac_at_measured_clock"] = achieved / (sms * FP32_LANES_PER_SM * clocks["sm_mhz"] * 1e6)

    # end to end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        Xh, yh, Qh = (torch.as_tensor(a).pin_memory() for a in (p.X, p.y, p.Q))
        outs = {k: torch.empty(nq, dtype=torch.float32).pin_memory() for k in ("g", "lo", "hi")}
        outs.update({k: torch.empty(nq, dtype=torch.int32).pin_memory() for k in ("idx_up", "idx_lo")})

        def step_host():
            for n in NORMS:
                m = models[n]
                m.clear()
                m.add_host(Xh, yh)
                m.eval_host(Qh, outs)
                m.lipschitz_constant()

        for n in NORMS:
            models[n].set_timing_events(None, None)
        step_host()
        torch.cuda.synchronize()
        e2e_ms = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            step_host()
            torch.cuda.synchronize()
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
        e2e_value, tot = aggregate(pairs_step * args.steps, sum(e2e_ms), device="cuda")
        h2d = len(NORMS) * (N * d * 4 + N * 4 + nq * d * 4)
        d2h = len(NORMS) * (nq * (3 * 4 + 2 * 4) + 24)
        e2e = {"value": e2e_value, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": tot / args.steps}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu, _ = oracle_rate(p, NORMS, args.cpu_seconds)

    tun = models[dom].tuning()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded, monotone d=4 workload)", "config": dict(CONFIG, parallelism=f"replicas{world}"),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": launches,
            "detail": {"scan_ms": {NNAME[n]: avg_scan[n] for n in NORMS},
                       "scan_gpairs_per_s": {NNAME[n]: nq * N / (avg_scan[n] / 1e3) / 1e9 for n in NORMS},
                       "M_est": {NNAME[n]: est[n][0] for n in NORMS},
                       "M_true": {NNAME[n]: p.M_by_norm[n] for n in NORMS},
                       "splits": tun["last_splits"], "tile_groups": tun["tile_groups"],
                       "queries_per_thread": tun["queries_per_thread"], "sms": sms,
                       "wall_s_timed": wall}}
    for m in models.values():
        m.close()
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
