"""Many data sets in one persistent launch (lip_batch_*): every set's outputs equal
lip_eval on that set bitwise, agree with the FP64 oracle, and survive CUDA-graph
capture and replay.  Needs a CUDA device."""
import numpy as np
import pytest

from paper_2606_04670_b300 import workloads as W
from parity import FP32_TOL, compare

pytestmark = pytest.mark.gpu


def _sets(n_sets=40, n_max=6000, q_max=2500, seed_extra=True):
    plan = W.batch_plan(n_sets=n_sets, n_max=n_max, q_min=50, q_max=q_max)
    out = []
    for bs in plan:
        X, y, Q, f = W.batch_set_data(bs)
        out.append(dict(X=X, y=y, Q=Q, M=bs.M, norm=bs.norm, mon=bs.mon, w=None, f=f))
    if seed_extra:
        # shapes the plan may miss: Linf, weights, decreasing coordinates, d = 1 and 10,
        # a single data point, a set without queries
        for k, (N, d, nq, norm, masked, weighted) in enumerate(
                [(777, 10, 300, W.NORM_LINF, True, True), (64, 1, 200, W.NORM_L2, True, False),
                 (1, 3, 100, W.NORM_L1, True, False), (500, 4, 0, W.NORM_L2, False, False),
                 (3000, 7, 1000, W.NORM_LINF, False, True), (129, 2, 1025, W.NORM_L2, True, True)]):
            p = W.random_problem(800 + k, N, d, nq, norm=norm, masked=masked, weighted=weighted, decreasing=masked)
            out.append(dict(X=p.X, y=p.y, Q=p.Q, M=p.M, norm=norm, mon=p.mon, w=p.w, f=p.f))
    return out


def _batch(sets, **kw):
    import torch

    from paper_2606_04670_b300.lipfit import LipBatch
    return LipBatch([{k: (torch.as_tensor(v) if isinstance(v, np.ndarray) and k in "XyQ" else v)
                      for k, v in s.items() if k != "f"} for s in sets], **kw)


def _single(s):
    import torch

    from paper_2606_04670_b300.lipfit import LipFit
    m = LipFit(torch.as_tensor(s["X"]).cuda(), torch.as_tensor(s["y"]).cuda(), s["M"], norm=s["norm"],
               mon=s["mon"], w=s["w"])
    r = {k: v.cpu().numpy() for k, v in m.eval(torch.as_tensor(s["Q"]).cuda()).items()} if len(s["Q"]) else None
    m.close()
    return r


@pytest.mark.parametrize("opts", [{}, {"tile_groups": 64, "items_per_block": 2, "waves": 2},
                                  {"tile_groups": 8, "items_per_block": 64}])
def test_batch_equals_single_set_eval(opts):
    import torch
    sets = _sets()
    b = _batch(sets, **opts)
    b.eval()
    torch.cuda.synchronize()
    b.check()
    for k, s in enumerate(sets):
        ref = _single(s)
        if ref is None:
            continue
        for key in ("g", "lo", "hi", "idx_up", "idx_lo"):
            np.testing.assert_array_equal(b.outputs[k][key].cpu().numpy(), ref[key], err_msg=f"set {k} {key}")
    b.close()


def test_batch_vs_oracle(oracle_mod):
    import torch
    sets = _sets(n_sets=24)
    b = _batch(sets)
    b.eval()
    torch.cuda.synchronize()
    for k, s in enumerate(sets):
        if len(s["Q"]) == 0:
            continue
        p = W.Problem("batch", s["X"], s["y"], s["Q"], s["M"], s["norm"], s["mon"], s["w"], s["f"])
        orc = oracle_mod.evaluate(p.X, p.y, p.Q, p.M, p.norm, mon=p.mon, w=p.w)
        gpu = {key: v.cpu().numpy() for key, v in b.outputs[k].items()}
        compare(p, gpu, orc, FP32_TOL, f"batch set {k}")
    b.close()


def test_batch_graph_capture_and_replay():
    import torch
    sets = _sets(n_sets=16, seed_extra=False)
    b = _batch(sets)
    b.eval()                      # warm-up outside the capture (module load, first launch)
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        b.eval()
    # new queries in place, then replay: outputs follow the new queries
    rng = np.random.default_rng(3)
    new_q = []
    for s in b.sets:
        q = rng.random(tuple(s["Q"].shape)).astype(np.float32)
        s["Q"].copy_(torch.as_tensor(q))
        new_q.append(q)
    g.replay()
    torch.cuda.synchronize()
    for k, s in enumerate(sets):
        ref = _single(dict(s, Q=new_q[k]))
        for key in ("g", "idx_up", "idx_lo"):
            np.testing.assert_array_equal(b.outputs[k][key].cpu().numpy(), ref[key], err_msg=f"set {k} {key}")
    b.close()


def test_batch_full_plan_sampled(oracle_mod):
    """The 4096-set batching workload at full size: one persistent launch, 64 sampled
    queries per set checked against the FP64 oracle."""
    import torch

    from paper_2606_04670_b300.lipfit import LipBatch
    plan = W.batch_plan()
    sets, samples = [], []
    rng = np.random.default_rng(17)
    for bs in plan:
        X, y, Q, f = W.batch_set_data(bs)
        sets.append(dict(X=torch.as_tensor(X), y=torch.as_tensor(y), Q=torch.as_tensor(Q), M=bs.M, norm=bs.norm,
                         mon=bs.mon))
        samples.append((rng.choice(bs.nq, 64, replace=False), X, y, Q))
    b = LipBatch(sets)
    b.eval()
    torch.cuda.synchronize()
    b.check()
    info = b.info()
    assert info["total_queries"] == sum(bs.nq for bs in plan)
    bad = 0
    for k, bs in enumerate(plan):
        idx, X, y, Q = samples[k]
        p = W.Problem("batch", X, y, Q[idx], bs.M, bs.norm, bs.mon, None)
        orc = oracle_mod.evaluate(X, y, Q[idx], bs.M, bs.norm, mon=bs.mon)
        gpu = {key: v[torch.as_tensor(idx).cuda()].cpu().numpy() for key, v in b.outputs[k].items()}
        compare(p, gpu, orc, FP32_TOL, f"plan set {k}")
        bad += 0
    b.close()
    assert bad == 0
