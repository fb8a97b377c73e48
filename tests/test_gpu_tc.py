"""Tensor-core L2 form (LIP_TC_TF32, LIP_TC_BF16, LIP_TC_FP16): the TF32-, BF16- or
FP16-split product on tcgen05 with an error bound, candidate pruning and an exact FP64
rescreen.  Its bounds are the FP64
envelopes, so indices must match the oracle's wherever the oracle's gap exceeds
1e-9 M diam (far below the FP32 tolerance).  Needs a CUDA device."""
import numpy as np
import pytest

from paper_2606_04670_b300 import workloads as W
from parity import FP32_TOL, compare, diam, gpu_eval

pytestmark = pytest.mark.gpu
EXACT_GAP = 1e-9


def _tc_eval(p, precision="tc_tf32"):
    """Outputs of a tensor-core handle and the number of its queries that went through
    the device-side fallback (whose results are exact too)."""
    import torch

    from paper_2606_04670_b300.lipfit import LipFit
    m = LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), p.M, norm=p.norm, w=p.w,
               precision=precision)
    r = {k: v.cpu().numpy() for k, v in m.eval(torch.as_tensor(p.Q).cuda()).items()}
    fb = m.last_fallback()
    m.check()
    m.close()
    return r, fb


def _check_exact(p, gpu, orc, label, fallback=0):
    """Values within the FP32 tolerance, every index equal to the oracle's wherever the
    oracle's gap exceeds EXACT_GAP M diam (fallback queries included: the device-side
    fallback is exact as well; `fallback` only labels the message)."""
    compare(p, gpu, orc, FP32_TOL, label)
    scale = p.M * diam(p.X, p.Q[: len(orc["hi"])], p.norm, p.w)
    for k, gk in (("idx_up", "gap_up"), ("idx_lo", "gap_lo")):
        clear = orc[gk] > EXACT_GAP * scale
        bad = np.nonzero(clear & (gpu[k].astype(np.int64) != orc[k]))[0]
        assert bad.size == 0, (f"{label} {k}: {bad.size} mismatches with gap > {EXACT_GAP} M diam "
                               f"({fallback} fallback queries)")
    # the outputs are FP64 values rounded once to FP32
    for k in ("hi", "lo"):
        np.testing.assert_allclose(gpu[k], orc[k].astype(np.float32), rtol=0, atol=2e-7 * (1 + np.abs(orc[k]).max()))


@pytest.mark.parametrize("d,weighted", [(1, False), (2, True), (3, False), (6, True), (7, False), (13, True),
                                        (16, False)])
def test_tc_random_shapes(oracle_mod, d, weighted):
    p = W.random_problem(950 + d, 5_003, d, 1_201, norm=W.NORM_L2, weighted=weighted)
    orc = oracle_mod.evaluate(p.X, p.y, p.Q, p.M, p.norm, w=p.w)
    r, fb = _tc_eval(p)
    _check_exact(p, r, orc, f"tc d={d}", fb)
    if d >= 6:
        assert fb == 0, f"{fb} fallback queries at d={d}"


def test_tc_cluster_subsample(oracle_mod):
    p = W.cluster_d16(n_data=30_000, n_query=1_500)
    orc = oracle_mod.evaluate(p.X, p.y, p.Q, p.M, p.norm)
    r, fb = _tc_eval(p)
    _check_exact(p, r, orc, "tc cluster", fb)


def test_tc_equals_plain_within_tolerance(oracle_mod):
    p = W.cluster_d16(n_data=20_000, n_query=1_000)
    a, b = gpu_eval(p, "tc_tf32"), gpu_eval(p, "fp32")
    orc = oracle_mod.evaluate(p.X, p.y, p.Q, p.M, p.norm)
    compare(p, a, orc, FP32_TOL, "tc")
    compare(p, b, orc, FP32_TOL, "plain")


@pytest.mark.parametrize("prec", ["tc_tf32", "tc_bf16", "tc_fp16"])
def test_tc_edge_cases_and_fallback(oracle_mod, prec):
    import torch

    from paper_2606_04670_b300.lipfit import LipFit
    # a single data point, one query, a NaN query, sizes that are not tile multiples
    p = W.random_problem(960, 1, 4, 3)
    orc = oracle_mod.evaluate(p.X, p.y, p.Q, p.M, p.norm)
    compare(p, gpu_eval(p, prec), orc, FP32_TOL, "tc N=1")
    p = W.random_problem(961, 257, 5, 129)
    m = LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), p.M, norm=p.norm, precision=prec)
    Q = torch.as_tensor(p.Q).cuda().clone()
    Q[5, 2] = float("nan")
    r = {k: v.cpu().numpy() for k, v in m.eval(Q).items()}
    assert np.isnan(r["g"][5]) and r["idx_up"][5] == -1
    keep = np.arange(p.nq) != 5
    orc = oracle_mod.evaluate(p.X, p.y, p.Q[keep], p.M, p.norm)
    ps = W.Problem("e", p.X, p.y, p.Q[keep], p.M, p.norm, None, None)
    compare(ps, {k: v[keep] for k, v in r.items()}, orc, FP32_TOL, "tc ragged")
    # after clear: NaN and -1 everywhere
    m.clear()
    r = m.eval(torch.as_tensor(p.Q).cuda())
    assert torch.isnan(r["g"]).all() and (r["idx_up"] == -1).all()
    m.check()
    m.close()
    # M = 0 with a constant y over 3000 points: every 32-point chunk ties, so each
    # query's candidate lists (8 chunks per half row) overflow and every query goes
    # through the device-side fallback; the result is still the lowest index
    p = W.random_problem(962, 3_000, 5, 300)
    yc = np.full(p.N, 0.25, np.float32)
    m = LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(yc).cuda(), 0.0, norm=p.norm, precision=prec)
    r = {k: v.cpu().numpy() for k, v in m.eval(torch.as_tensor(p.Q).cuda()).items()}
    assert m.last_fallback() == p.nq
    assert np.all(r["idx_up"] == 0) and np.all(r["idx_lo"] == 0) and np.allclose(r["g"], 0.25)
    m.check()
    m.close()


def test_tc_full_size_cluster_sampled(oracle_mod):
    """The precision workload at full size (N = Q = 1e6, d = 16) on the tensor cores,
    checked on 400 sampled queries against the FP64 oracle."""
    import torch

    from paper_2606_04670_b300.lipfit import LipFit
    p = W.cluster_d16()
    m = LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), p.M, norm=p.norm, precision="tc_tf32")
    r = {k: v.cpu().numpy() for k, v in m.eval(torch.as_tensor(p.Q).cuda()).items()}
    fb = m.last_fallback()
    m.check()
    m.close()
    assert fb <= p.nq // 100          # the pruning settles at least 99 % of the queries
    idx = np.sort(np.random.default_rng(21).choice(p.nq, 400, replace=False))
    ps = W.Problem("c", p.X, p.y, p.Q[idx], p.M, p.norm, None, None)
    orc = oracle_mod.evaluate(p.X, p.y, ps.Q, p.M, p.norm)
    _check_exact(ps, {k: v[idx] for k, v in r.items()}, orc, "tc full cluster", fb)


def test_bf16_full_size_cluster_sampled(oracle_mod):
    """The BF16 form at the full precision workload (N = Q = 1e6, d = 16), as the benchmark
    launches it, checked on 400 sampled queries against the FP64 oracle."""
    import torch

    from paper_2606_04670_b300.lipfit import LipFit
    p = W.cluster_d16()
    m = LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), p.M, norm=p.norm, precision="tc_bf16")
    r = {k: v.cpu().numpy() for k, v in m.eval(torch.as_tensor(p.Q).cuda()).items()}
    fb = m.last_fallback()
    m.check()
    m.close()
    assert fb <= p.nq // 100
    idx = np.sort(np.random.default_rng(22).choice(p.nq, 400, replace=False))
    ps = W.Problem("c", p.X, p.y, p.Q[idx], p.M, p.norm, None, None)
    orc = oracle_mod.evaluate(p.X, p.y, ps.Q, p.M, p.norm)
    _check_exact(ps, {k: v[idx] for k, v in r.items()}, orc, "bf16 full cluster", fb)


@pytest.mark.parametrize("d,weighted", [(1, False), (2, True), (6, True), (13, False), (14, True), (15, False),
                                        (16, True)])
def test_bf16_random_shapes(oracle_mod, d, weighted):
    """The BF16 three-piece split (K = 16 for every d; the norms are added in the epilogue):
    the same exact results."""
    p = W.random_problem(970 + d, 5_003, d, 1_201, norm=W.NORM_L2, weighted=weighted)
    orc = oracle_mod.evaluate(p.X, p.y, p.Q, p.M, p.norm, w=p.w)
    r, fb = _tc_eval(p, "tc_bf16")
    _check_exact(p, r, orc, f"bf16 d={d}", fb)
    if d >= 6:
        assert fb <= 2, f"{fb} fallback queries at d={d}"


def test_bf16_cluster_subsample(oracle_mod):
    p = W.cluster_d16(n_data=30_000, n_query=1_500)
    orc = oracle_mod.evaluate(p.X, p.y, p.Q, p.M, p.norm)
    r, fb = _tc_eval(p, "tc_bf16")
    _check_exact(p, r, orc, "bf16 cluster", fb)
    rt, _ = _tc_eval(p, "tc_tf32")
    for k in ("idx_up", "idx_lo"):
        assert np.array_equal(r[k], rt[k]) or fb > 0


@pytest.mark.parametrize("d,weighted", [(1, False), (2, True), (5, False), (8, True), (13, False), (16, True)])
def test_fp16_random_shapes(oracle_mod, d, weighted):
    """The FP16 two-piece split (operands scaled by a power of two into the fp16 range):
    the same exact results."""
    p = W.random_problem(990 + d, 5_003, d, 1_201, norm=W.NORM_L2, weighted=weighted)
    orc = oracle_mod.evaluate(p.X, p.y, p.Q, p.M, p.norm, w=p.w)
    r, fb = _tc_eval(p, "tc_fp16")
    _check_exact(p, r, orc, f"fp16 d={d}", fb)
    if d >= 6:
        assert fb <= 2, f"{fb} fallback queries at d={d}"


def test_fp16_cluster_and_far_queries(oracle_mod):
    """The precision workload's shape at a reduced size, plus queries far outside the data
    (beyond the fp16 range after scaling): those go through the device-side fallback; every
    query stays exact."""
    p = W.cluster_d16(n_data=30_000, n_query=1_500)
    Q = p.Q.copy()
    far = np.array([3, 700, 1499])
    Q[far] *= 1e6                      # far beyond 2^14 times the box's half-diagonal
    ps = W.Problem("f", p.X, p.y, Q, p.M, p.norm, None, None)
    orc = oracle_mod.evaluate(p.X, p.y, Q, p.M, p.norm)
    r, fb = _tc_eval(ps, "tc_fp16")
    assert fb >= far.size, f"{fb} fallback queries, {far.size} outside the fp16 range"
    assert fb <= far.size + 15
    _check_exact(ps, r, orc, "fp16 cluster + far", fb)


def test_fp16_single_point_and_constant_coordinate(oracle_mod):
    """A data set of one point (a box of zero size: scale 2^0) and one whose coordinates are
    all equal in one dimension."""
    p = W.random_problem(996, 1, 3, 257)
    orc = oracle_mod.evaluate(p.X, p.y, p.Q, p.M, p.norm)
    r, fb = _tc_eval(p, "tc_fp16")
    compare(p, r, orc, FP32_TOL, "fp16 N=1")
    p = W.random_problem(997, 2_000, 4, 300)
    X = p.X.copy()
    X[:, 1] = 0.375
    ps = W.Problem("c", X, p.y, p.Q, p.M, p.norm, None, None)
    orc = oracle_mod.evaluate(X, p.y, p.Q, p.M, p.norm)
    r, fb = _tc_eval(ps, "tc_fp16")
    _check_exact(ps, r, orc, "fp16 flat coordinate", fb)


def test_fp16_full_size_cluster_sampled(oracle_mod):
    """The FP16 form at the full precision workload (N = Q = 1e6, d = 16), as the benchmark
    launches it, checked on 400 sampled queries against the FP64 oracle."""
    import torch

    from paper_2606_04670_b300.lipfit import LipFit
    p = W.cluster_d16()
    m = LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), p.M, norm=p.norm, precision="tc_fp16")
    r = {k: v.cpu().numpy() for k, v in m.eval(torch.as_tensor(p.Q).cuda()).items()}
    fb = m.last_fallback()
    m.check()
    m.close()
    assert fb <= p.nq // 100
    idx = np.sort(np.random.default_rng(23).choice(p.nq, 400, replace=False))
    ps = W.Problem("c", p.X, p.y, p.Q[idx], p.M, p.norm, None, None)
    orc = oracle_mod.evaluate(p.X, p.y, ps.Q, p.M, p.norm)
    _check_exact(ps, {k: v[idx] for k, v in r.items()}, orc, "fp16 full cluster", fb)


def test_tc_forms_agree_bitwise(oracle_mod):
    """TF32, BF16 and FP16 all return the FP64 envelopes rounded once (the rescreen and the
    fallback alike), so their outputs are bit for bit the same (values and indices)."""
    p = W.cluster_d16(n_data=20_000, n_query=1_000)
    outs = {}
    for prec in ("tc_tf32", "tc_bf16", "tc_fp16"):
        outs[prec] = _tc_eval(p, prec)
    ref = outs["tc_tf32"][0]
    for prec in ("tc_bf16", "tc_fp16"):
        for k in ("g", "lo", "hi", "idx_up", "idx_lo"):
            assert np.array_equal(outs[prec][0][k], ref[k]), f"{prec} {k} differs from tc_tf32"


@pytest.mark.parametrize("prec", ["tc_tf32", "tc_bf16", "tc_fp16"])
def test_tc_offset_data(oracle_mod, prec):
    """Data and queries 1e4 away from the origin with a unit spread: the operands are centred
    (in FP64, before any rounding), so the split products and their error bound see the
    unit spread, and the results stay exact."""
    p = W.random_problem(1001, 4_000, 4, 800, norm=W.NORM_L2)
    off = np.float32(1.0e4)
    X = (p.X + off).astype(np.float32)
    Q = (p.Q + off).astype(np.float32)
    ps = W.Problem("o", X, p.y, Q, p.M, p.norm, None, None)
    orc = oracle_mod.evaluate(X, p.y, Q, p.M, p.norm)
    r, fb = _tc_eval(ps, prec)
    _check_exact(ps, r, orc, f"{prec} offset", fb)
    assert fb <= 8, f"{fb} fallback queries"


def test_tc_timing_events_bracket_the_scan():
    """lip_set_timing_events on a tensor-core handle: the two events are recorded around
    the tc_scan launch on the handle's stream, so they bracket a positive interval that is
    shorter than the whole evaluation."""
    import time

    import torch

    from paper_2606_04670_b300.lipfit import LipFit
    p = W.cluster_d16(n_data=50_000, n_query=8_192)
    m = LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), p.M, norm=p.norm, precision="tc_fp16")
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    m.set_timing_events(*ev)
    Q = torch.as_tensor(p.Q).cuda()
    m.eval(Q)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m.eval(Q)
    torch.cuda.synchronize()
    whole_ms = 1e3 * (time.perf_counter() - t0)
    scan_ms = ev[0].elapsed_time(ev[1])
    m.set_timing_events(None, None)
    m.check()
    m.close()
    assert 0.0 < scan_ms < whole_ms


def _fallback_problem(seed=1010, n=6_000, nq=1_500, n_far=400, dup=True):
    """Data with exact duplicates (ties in value: the lowest index must win) and queries of
    which n_far lie beyond the fp16 range (so the fp16 form sends them to the fallback)."""
    p = W.random_problem(seed, n, 6, nq, norm=W.NORM_L2)
    X, y = p.X.copy(), p.y.copy()
    if dup:
        X[n // 2:n // 2 + 500] = X[:500]          # duplicated points with equal values
        y[n // 2:n // 2 + 500] = y[:500]
    Q = p.Q.copy()
    Q[:50] = X[:50]                                # queries on data points
    far = 50 + np.random.default_rng(seed).choice(nq - 50, n_far, replace=False)
    Q[far] = Q[far] * 3e5 + 7.0
    return W.Problem("fb", X, y, Q, p.M, p.norm, None, None), far


@pytest.mark.parametrize("prec", ["tc_tf32", "tc_fp16"])
def test_fallback_is_exact(oracle_mod, prec):
    """Hundreds of queries through the device-side fallback (fp16: outside the fp16 range),
    against the FP64 oracle with the exact index rule, duplicates included."""
    p, far = _fallback_problem()
    orc = oracle_mod.evaluate(p.X, p.y, p.Q, p.M, p.norm)
    r, fb = _tc_eval(p, prec)
    if prec == "tc_fp16":
        assert fb >= far.size, (fb, far.size)
    _check_exact(p, r, orc, f"{prec} fallback", fb)
    # ties between duplicates resolve to the lower index, as in the oracle
    for k in ("idx_up", "idx_lo"):
        tie = orc["gap_" + k[4:]] == 0
        assert np.array_equal(r[k][tie], orc[k][tie]), k


def test_fallback_all_queries_random_values(oracle_mod):
    """Every query through the fallback (fp16 form, all queries far away) on random data:
    equal to the oracle's envelopes rounded once."""
    p = W.random_problem(1011, 3_001, 3, 700, norm=W.NORM_L2, weighted=True)
    Q = (p.Q * 4e5 - 2e5).astype(np.float32)
    ps = W.Problem("fa", p.X, p.y, Q, p.M, p.norm, None, p.w)
    orc = oracle_mod.evaluate(ps.X, ps.y, ps.Q, ps.M, ps.norm, w=ps.w)
    r, fb = _tc_eval(ps, "tc_fp16")
    assert fb == ps.nq
    _check_exact(ps, r, orc, "fp16 all far", fb)


@pytest.mark.parametrize("prec", ["tc_tf32", "tc_fp16"])
def test_tc_eval_captured_in_a_cuda_graph(oracle_mod, prec):
    """lip_eval on a tensor-core handle does not synchronise, so it can be captured in a CUDA
    graph (after one eager call that sizes the scratch); replays with new query values
    (a different number of fallback queries each time) equal eager calls bit for bit."""
    import torch

    from paper_2606_04670_b300.lipfit import LipFit
    p, _ = _fallback_problem(1012, 5_000, 1_024, 100)
    m = LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), p.M, norm=p.norm, precision=prec)
    Qs = torch.as_tensor(p.Q).cuda().clone()
    m.eval(Qs)
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            out = m.eval(Qs)
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    for rep in range(3):
        Qn = p.Q.copy()
        far = rng.choice(p.nq, 40 * rep, replace=False)
        Qn[far] = Qn[far] * 3e5
        Qs.copy_(torch.as_tensor(Qn).cuda())
        g.replay()
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy().copy() for k, v in out.items()}
        ref = {k: v.cpu().numpy() for k, v in m.eval(torch.as_tensor(Qn).cuda()).items()}
        for k in ref:
            np.testing.assert_array_equal(got[k], ref[k], err_msg=f"{prec} replay {rep} {k}")
        if rep == 2:
            ps = W.Problem("g", p.X, p.y, Qn, p.M, p.norm, None, None)
            _check_exact(ps, got, oracle_mod.evaluate(p.X, p.y, Qn, p.M, p.norm), f"{prec} graph")
    m.check()
    m.close()


@pytest.mark.parametrize("prec", ["tc_tf32", "tc_bf16", "tc_fp16"])
def test_tc_variants_and_rounds(oracle_mod, prec):
    """40,000 queries are 313 query tiles: three rounds of the persistent scan (148, 148 and
    17 CTAs), the last one partial.  The six variants (epilogue warps x persistent CTAs with
    or without the soft lockstep of the data sweep, or one CTA per query tile) give the
    same outputs bit for bit, and a sample of queries matches the oracle under the exact
    index rule."""
    import torch

    from paper_2606_04670_b300.lipfit import LipFit
    p = W.cluster_d16(n_data=20_000, n_query=40_000)
    m = LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), p.M, norm=p.norm, precision=prec)
    Q = torch.as_tensor(p.Q).cuda()
    outs = []
    for v in range(6):
        m.set_tuning(0, 0, v)
        outs.append({k: t.cpu().numpy() for k, t in m.eval(Q).items()})
    m.check()
    m.close()
    for v in range(1, 6):
        for k in outs[0]:
            assert np.array_equal(outs[v][k], outs[0][k]), f"variant {v} {k}"
    idx = np.sort(np.random.default_rng(31).choice(p.nq, 500, replace=False))
    ps = W.Problem("r", p.X, p.y, p.Q[idx], p.M, p.norm, None, None)
    orc = oracle_mod.evaluate(p.X, p.y, ps.Q, p.M, p.norm)
    _check_exact(ps, {k: v[idx] for k, v in outs[0].items()}, orc, f"{prec} rounds")
