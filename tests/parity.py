"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI, run the
FP64 oracle on the same seeded inputs, and compare element by element."""
from __future__ import annotations

import numpy as np

FP32_TOL = 1e-5      # |GPU - oracle| <= FP32_TOL * M * diam  (FP32 handles)
FP64_TOL = 1e-12     # FP64 handles


def diam(X, Q, norm, w=None):
    """Distance, in the evaluation norm with weights, between the corners of the bounding
    box of the data and the queries."""
    lo = np.minimum(X.min(0), Q.min(0)).astype(np.float64)
    hi = np.maximum(X.max(0), Q.max(0)).astype(np.float64)
    v = hi - lo
    if w is not None:
        v = v * np.asarray(w)
    return {1: v.sum(), 2: float(np.sqrt((v * v).sum())), 3: v.max()}[norm]


def gpu_eval(p, precision="fp32", Q=None, splits=None, tile_groups=None, variant=-1):
    import torch

    from paper_2606_04670_b300.lipfit import LipFit
    dt = torch.float64 if precision == "fp64" else torch.float32
    m = LipFit(torch.as_tensor(p.X).to("cuda", dt), torch.as_tensor(p.y).to("cuda", dt), p.M,
               norm=p.norm, mon=p.mon, w=p.w, precision=precision)
    if splits is not None or tile_groups is not None or variant >= 0:
        m.set_tuning(tile_groups or 0, splits or 0, variant)
    Qd = torch.as_tensor(p.Q if Q is None else Q).to("cuda", dt)
    r = m.eval(Qd)
    torch.cuda.synchronize()
    m.check()
    out = {k: v.cpu().numpy() for k, v in r.items()}
    m.close()
    return out


def compare(p, gpu, orc, tol_rel, label=""):
    """Values within tol_rel * M * diam; indices equal wherever the oracle's gap between
    the best and second-best bound exceeds the tolerance."""
    tol = tol_rel * max(p.M, 1e-30) * diam(p.X, p.Q[: len(orc["hi"])], p.norm, p.w)
    tol = max(tol, tol_rel)           # M = 0 or a single point still needs a scale
    report = {}
    for k in ("hi", "lo", "g"):
        err = np.abs(gpu[k].astype(np.float64) - orc[k])
        report[k] = float(np.nanmax(err)) if err.size else 0.0
        assert np.all(err <= tol), f"{label} {k}: max err {err.max():.3e} > tol {tol:.3e}"
    for k, gk in (("idx_up", "gap_up"), ("idx_lo", "gap_lo")):
        clear = orc[gk] > tol
        bad = np.nonzero(clear & (gpu[k].astype(np.int64) != orc[k]))[0]
        assert bad.size == 0, f"{label} {k}: {bad.size} index mismatches above the gap rule, first {bad[:5]}"
    return tol, report
