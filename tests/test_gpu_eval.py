"""GPU parity of lip_eval against the FP64 oracle (element by element), edge cases, and
the full-size monotone d=4 workload on sampled queries.  Needs a CUDA device."""
import numpy as np
import pytest

from paper_2606_04670_b300 import workloads as W
from parity import FP32_TOL, FP64_TOL, compare, gpu_eval

pytestmark = pytest.mark.gpu

NORMS = (W.NORM_L1, W.NORM_L2, W.NORM_LINF)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")


def test_plain_d2_fp32_fp64(oracle_mod):
    p = W.plain_d2()
    orc = oracle_mod.evaluate(p.X, p.y, p.Q, p.M, p.norm)
    compare(p, gpu_eval(p, "fp32"), orc, FP32_TOL, "plain_d2 fp32")
    p64 = W.plain_d2(dtype=np.float64)
    orc64 = oracle_mod.evaluate(p64.X, p64.y, p64.Q, p64.M, p64.norm)
    compare(p64, gpu_eval(p64, "fp64"), orc64, FP64_TOL, "plain_d2 fp64")


@pytest.mark.parametrize("norm", NORMS)
def test_monotone_d4_ragged(oracle_mod, norm):
    # several tiles and splits with a ragged tail (N, nq not multiples of anything)
    p = W.monotone_d4(norm=norm, n_data=20_011, n_query=3_001)
    orc = oracle_mod.evaluate(p.X, p.y, p.Q, p.M, norm, mon=p.mon)
    compare(p, gpu_eval(p), orc, FP32_TOL, f"monotone_d4 {norm}")


@pytest.mark.parametrize("norm", NORMS)
@pytest.mark.parametrize("shape", [(1, False, False), (3, True, False), (5, True, True), (7, False, True),
                                   (10, True, True), (12, True, False), (16, True, True), (16, False, False),
                                   (13, False, True)])
def test_random_shapes(oracle_mod, norm, shape):
    d, masked, weighted = shape
    p = W.random_problem(200 + d, 3_333, d, 777, norm=norm, masked=masked, weighted=weighted,
                         decreasing=masked)
    orc = oracle_mod.evaluate(p.X, p.y, p.Q, p.M, norm, mon=p.mon, w=p.w)
    compare(p, gpu_eval(p), orc, FP32_TOL, f"random d={d} {norm}")


@pytest.mark.parametrize("norm", NORMS)
def test_random_shapes_fp64(oracle_mod, norm):
    for d, masked in ((3, True), (9, False), (16, True)):
        p = W.random_problem(300 + d, 1_500, d, 300, norm=norm, masked=masked, weighted=True,
                             decreasing=masked, dtype=np.float64)
        orc = oracle_mod.evaluate(p.X, p.y, p.Q, p.M, norm, mon=p.mon, w=p.w)
        compare(p, gpu_eval(p, "fp64"), orc, FP64_TOL, f"fp64 d={d} {norm}")


@pytest.mark.parametrize("norm", NORMS)
def test_fp64_screen_equals_fp64_scan(oracle_mod, norm):
    """FP64 handles: the FP32 screen with FP64 candidates (variant 0, the default) and the
    FP64 scan throughout (variant 1) both give the oracle's FP64 envelopes; exact and
    generic float layouts (masked d > 10 has no exact FP32 kernel), ragged sizes."""
    for d, masked, weighted, N, nq in ((2, False, False, 1_001, 517), (4, True, True, 2_049, 300),
                                       (11, True, False, 700, 129), (16, False, True, 1_300, 260)):
        p = W.random_problem(320 + d, N, d, nq, norm=norm, masked=masked, weighted=weighted,
                             decreasing=masked, dtype=np.float64)
        orc = oracle_mod.evaluate(p.X, p.y, p.Q, p.M, norm, mon=p.mon, w=p.w)
        a = gpu_eval(p, "fp64", variant=0)
        b = gpu_eval(p, "fp64", variant=1)
        compare(p, a, orc, FP64_TOL, f"fp64 screen d={d} {norm}")
        compare(p, b, orc, FP64_TOL, f"fp64 scan d={d} {norm}")
        for k in ("idx_up", "idx_lo"):
            clear = orc["gap_up" if k == "idx_up" else "gap_lo"] > 0
            assert np.array_equal(a[k][clear], b[k][clear]), k


def test_fp64_screen_ties_and_edges(oracle_mod):
    """Every pair a candidate (M = 0, constant y: the lowest index wins), a single datum,
    and a NaN query."""
    X = np.random.default_rng(3).random((3000, 3))
    y = np.full(3000, 0.25)
    Q = np.random.default_rng(4).random((40, 3))
    Q[5, 1] = np.nan
    p = W.Problem("ties", X, y, Q, 0.0, 2, None, None)
    r = gpu_eval(p, "fp64")
    assert np.all(r["idx_up"][np.arange(40) != 5] == 0) and np.all(r["idx_lo"][np.arange(40) != 5] == 0)
    assert np.isnan(r["g"][5]) and r["idx_up"][5] == -1
    assert np.all(r["g"][np.arange(40) != 5] == 0.25)
    p1 = W.Problem("one", X[:1], np.array([1.5]), Q[:4], 2.0, 1, None, None)
    orc = oracle_mod.evaluate(p1.X, p1.y, p1.Q, p1.M, 1)
    compare(p1, gpu_eval(p1, "fp64"), orc, FP64_TOL, "fp64 one datum")


def test_workload_shapes(oracle_mod):
    for p in (W.toy_d3(), W.grad_d8(n_data=9_000, n_query=1_000), W.cluster_d16(n_data=12_000, n_query=500)):
        orc = oracle_mod.evaluate(p.X, p.y, p.Q, p.M, p.norm, mon=p.mon, w=p.w)
        compare(p, gpu_eval(p), orc, FP32_TOL, p.name)


@pytest.mark.parametrize("splits,tile_groups,variant", [(1, 8, 0), (3, 16, 1), (7, 32, 1), (64, 64, 0), (0, 8, 1)])
def test_launch_shape_does_not_change_results(splits, tile_groups, variant):
    p = W.monotone_d4(norm=W.NORM_L2, n_data=30_000, n_query=2_000)
    ref = gpu_eval(p)
    got = gpu_eval(p, splits=splits, tile_groups=tile_groups, variant=variant)
    for k in ref:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)


def test_edge_cases(oracle_mod):
    import torch

    from paper_2606_04670_b300.lipfit import LipFit
    p = W.random_problem(400, 1, 3, 50, norm=W.NORM_L2, masked=True)
    # N = 1
    orc = oracle_mod.evaluate(p.X, p.y, p.Q, p.M, p.norm, mon=p.mon)
    compare(p, gpu_eval(p), orc, FP32_TOL, "N=1")
    # nq = 1, nq = 0, NaN query
    p = W.random_problem(401, 5_000, 4, 3, norm=W.NORM_L1, masked=True)
    m = LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), p.M, norm=p.norm, mon=p.mon)
    r = m.eval(torch.as_tensor(p.Q[:1]).cuda())
    orc = oracle_mod.evaluate(p.X, p.y, p.Q[:1], p.M, p.norm, mon=p.mon)
    assert abs(r["g"].item() - orc.g[0]) <= FP32_TOL * p.M * 4
    assert m.eval(torch.zeros(0, 4, device="cuda"))["g"].numel() == 0
    Qn = torch.as_tensor(p.Q).cuda().clone()
    Qn[1, 2] = float("nan")
    r = m.eval(Qn)
    assert torch.isnan(r["g"][1]) and r["idx_up"][1].item() == -1 and r["idx_lo"][1].item() == -1
    assert torch.isfinite(r["g"][[0, 2]]).all()
    # M = 0 gives the data range
    m.set_M(0.0)
    r = m.eval(torch.as_tensor(p.Q).cuda())
    assert np.allclose(r["hi"].cpu().numpy(), p.y.min()) and np.allclose(r["lo"].cpu().numpy(), p.y.max())
    # empty after clear: NaN / -1
    m.clear()
    assert m.N == 0
    r = m.eval(torch.as_tensor(p.Q).cuda())
    assert torch.isnan(r["g"]).all() and (r["idx_up"] == -1).all()
    m.check()
    m.close()


def test_incremental_add_equals_fit(oracle_mod):
    import torch

    from paper_2606_04670_b300.lipfit import LipFit
    p = W.random_problem(402, 7_001, 5, 600, norm=W.NORM_LINF, masked=True, weighted=True)
    m = LipFit(M=p.M, norm=p.norm, mon=p.mon, w=p.w, capacity=10_000, d=5)
    for a, b in ((0, 1000), (1000, 1001), (1001, 7001)):
        m.add(torch.as_tensor(p.X[a:b]).cuda(), torch.as_tensor(p.y[a:b]).cuda())
    assert m.N == 7001
    r = {k: v.cpu().numpy() for k, v in m.eval(torch.as_tensor(p.Q).cuda()).items()}
    orc = oracle_mod.evaluate(p.X, p.y, p.Q, p.M, p.norm, mon=p.mon, w=p.w)
    compare(p, r, orc, FP32_TOL, "incremental")
    # beyond the capacity: refused, handle unchanged
    from paper_2606_04670_b300.lipfit import LipError, LIP_ERR_CAPACITY
    with pytest.raises(LipError) as e:
        m.add(torch.as_tensor(p.X[:5000]).cuda(), torch.as_tensor(p.y[:5000]).cuda())
    assert e.value.status == LIP_ERR_CAPACITY and m.N == 7001
    # non-finite data refused, handle unchanged
    from paper_2606_04670_b300.lipfit import LIP_ERR_NONFINITE
    Xb = torch.as_tensor(p.X[:10]).cuda().clone()
    Xb[3, 1] = float("inf")
    with pytest.raises(LipError) as e:
        m.add(Xb, torch.as_tensor(p.y[:10]).cuda())
    assert e.value.status == LIP_ERR_NONFINITE and m.N == 7001
    r2 = {k: v.cpu().numpy() for k, v in m.eval(torch.as_tensor(p.Q).cuda()).items()}
    for k in r:
        np.testing.assert_array_equal(r2[k], r[k])
    m.close()


def test_set_M_equals_refit(oracle_mod):
    p = W.random_problem(403, 4_000, 6, 500, norm=W.NORM_L2, masked=True)
    import torch

    from paper_2606_04670_b300.lipfit import LipFit
    m = LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), 1.0, norm=p.norm, mon=p.mon)
    m.set_M(p.M)
    r = {k: v.cpu().numpy() for k, v in m.eval(torch.as_tensor(p.Q).cuda()).items()}
    ref = gpu_eval(p)
    for k in r:
        np.testing.assert_array_equal(r[k], ref[k])
    m.close()


@pytest.mark.parametrize("variant", (0, 6))
def test_eval_host_equals_eval(variant):
    """The host path equals the device path bit for bit: in three chunks with copies
    overlapping the kernels (variant 0), in one chunk for the pruned scan (variant 6)."""
    import torch

    from paper_2606_04670_b300.lipfit import LipFit
    p = W.monotone_d4(norm=W.NORM_L1, n_data=10_000, n_query=1_200_000)
    m = LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), p.M, norm=p.norm, mon=p.mon)
    m.set_tuning(0, 0, variant)
    dev = {k: v.cpu().numpy() for k, v in m.eval(torch.as_tensor(p.Q).cuda()).items()}
    Qp = torch.as_tensor(p.Q).pin_memory()
    host = m.eval_host(Qp)
    for k in dev:
        np.testing.assert_array_equal(host[k], dev[k], err_msg=k)
    m.close()


def test_eval_host_async_on_several_handles():
    """lip_eval_host_async on three handles queued back to back (their copies overlap the
    others' kernels), the results read after lip_check: equal to the device path."""
    import torch

    from paper_2606_04670_b300.lipfit import LipFit
    runs = []
    for norm, variant in ((W.NORM_L1, 6), (W.NORM_L2, 0), (W.NORM_LINF, 6)):
        p = W.monotone_d4(norm=norm, n_data=20_000, n_query=700_000)
        m = LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), p.M, norm=p.norm, mon=p.mon)
        m.set_tuning(0, 0, variant)
        dev = {k: v.cpu().numpy() for k, v in m.eval(torch.as_tensor(p.Q).cuda()).items()}
        Qp = torch.as_tensor(p.Q).pin_memory()
        out = {k: torch.empty(p.nq, dtype=torch.float32).pin_memory() for k in ("g", "lo", "hi")}
        out.update({k: torch.empty(p.nq, dtype=torch.int32).pin_memory() for k in ("idx_up", "idx_lo")})
        runs.append((m, dev, Qp, out))
    for m, _, Qp, out in runs:
        m.eval_host(Qp, out, wait=False)
    for m, dev, _, out in runs:
        m.check()
        for k in dev:
            np.testing.assert_array_equal(out[k].numpy(), dev[k], err_msg=k)
        m.close()


@pytest.mark.parametrize("norm", NORMS)
def test_full_size_monotone_d4_sampled(oracle_mod, norm):
    """The benchmark workload at full size (N = 1e5, Q = 1e6, same launch shape as the
    benchmark), checked on 1500 sampled queries."""
    import torch

    from paper_2606_04670_b300.lipfit import LipFit
    p = W.monotone_d4(norm=norm)
    m = LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), p.M, norm=norm, mon=p.mon)
    r = {k: v.cpu().numpy() for k, v in m.eval(torch.as_tensor(p.Q).cuda()).items()}
    m.check()
    m.close()
    idx = np.random.default_rng(9).choice(p.nq, 1500, replace=False)
    idx.sort()
    ps = p.sub_queries(p.nq)
    ps.Q = p.Q[idx]
    orc = oracle_mod.evaluate(p.X, p.y, ps.Q, p.M, norm, mon=p.mon)
    compare(ps, {k: v[idx] for k, v in r.items()}, orc, FP32_TOL, f"full monotone_d4 {norm}")
    # properties that hold at any size, on every query: lo <= g <= hi (M is a valid bound)
    assert np.all(r["lo"] <= r["g"]) and np.all(r["g"] <= r["hi"])
    assert r["idx_up"].min() >= 0 and r["idx_up"].max() < p.N


def test_fma_pipe_square_root():
    """The FMA-pipe square root (Lomont's seed, three Newton steps) against FP64 sqrt: within
    4 ulps for normal inputs, exactly 0 at 0, NaN for NaN, and within 1.1e-19 below FLT_MIN."""
    import torch

    from paper_2606_04670_b300 import lipfit as L
    rng = np.random.default_rng(0)
    s = np.concatenate([np.exp(rng.uniform(np.log(1.2e-38), np.log(3e38), 200_000)), rng.random(50_000),
                        np.array([0.0, 1.0, 4.0, 2.0, 1e-42, 1e-39, 3.4e38, np.nan])]).astype(np.float32)
    sd = torch.as_tensor(s).cuda()
    out = torch.empty_like(sd)
    assert L.lip_debug_sqrt_fma(sd.data_ptr(), out.data_ptr(), len(s), torch.cuda.current_stream().cuda_stream) == 0
    r = out.cpu().numpy().astype(np.float64)
    ref = np.sqrt(s.astype(np.float64))
    normal = s >= np.float32(1.17549435e-38)
    rel = np.abs(r[normal] - ref[normal]) / ref[normal]
    assert rel.max() <= 4 * 2.0 ** -24, rel.max()
    assert r[s == 0].tolist() == [0.0] and np.isnan(r[np.isnan(s)]).all()
    tiny = (s > 0) & ~normal
    assert np.all(np.abs(r[tiny] - ref[tiny]) <= 1.1e-19)


@pytest.mark.parametrize("variant", [2, 3, 4, 5])
@pytest.mark.parametrize("d,seed", [(4, 0), (3, 1), (6, 2)])
def test_fma_sqrt_variants_vs_oracle(oracle_mod, variant, d, seed):
    """Variants 2-5 (a share of the L2 scan's square roots on the FMA pipe) against the oracle
    on monotone shapes, and independent of tiles and splits bit for bit."""
    p = W.random_problem(450 + 3 * d + seed, 6_007, d, 2_111, norm=W.NORM_L2, masked=True, weighted=(seed == 1),
                         decreasing=(seed == 2))
    if not np.any(p.mon):
        p.mon[0] = 1
    orc = oracle_mod.evaluate(p.X, p.y, p.Q, p.M, p.norm, mon=p.mon, w=p.w)
    a = gpu_eval(p, variant=variant)
    compare(p, a, orc, FP32_TOL, f"variant {variant} d={d}")
    b = gpu_eval(p, variant=variant, splits=5, tile_groups=16)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])


@pytest.mark.parametrize("precision", ["fp32", "fp64", "tc_tf32"])
def test_deferred_add_checks_on_the_device(oracle_mod, precision):
    """lip_add_async / lip_add_host_async do not wait for the GPU: finite data give the same
    handle as lip_add (bit for bit); a batch holding NaN / Inf is accepted, the bad points
    are replaced on the device by the handle's first point, lip_check then reports
    LIP_ERR_NONFINITE once, and the results equal those of the data with that replacement."""
    import torch

    from paper_2606_04670_b300 import lipfit as L
    dt = torch.float64 if precision == "fp64" else torch.float32
    ndt = np.float64 if precision == "fp64" else np.float32
    p = W.random_problem(1900, 3_000, 3, 500, norm=W.NORM_L2, dtype=ndt)
    X, y, Q = (torch.as_tensor(a).to("cuda", dt) for a in (p.X, p.y, p.Q))

    def model():
        return L.LipFit(M=p.M, norm=p.norm, capacity=2 * p.N, d=p.d, precision=precision)

    ref = model()
    ref.add(X[:1000], y[:1000])
    ref.add(X[1000:], y[1000:])
    r_ref = {k: v.cpu().numpy() for k, v in ref.eval(Q).items()}
    m = model()
    m.add_async(X[:1000], y[:1000])
    m.add_host_async(torch.as_tensor(p.X[1000:]).to(dt).pin_memory(), torch.as_tensor(p.y[1000:]).to(dt).pin_memory())
    r = {k: v.cpu().numpy() for k, v in m.eval(Q).items()}
    m.check()
    for k in r_ref:
        np.testing.assert_array_equal(r[k], r_ref[k], err_msg=k)
    # a batch with NaN and Inf: accepted, replaced by point 0, reported once by check()
    Xb, yb = p.X[:200].copy(), p.y[:200].copy()
    Xb[3, 1] = np.nan
    yb[17] = np.inf
    Xb[150] = -np.inf
    m.add_async(torch.as_tensor(Xb).to("cuda", dt), torch.as_tensor(yb).to("cuda", dt))
    assert m.N == p.N + 200
    r = {k: v.cpu().numpy() for k, v in m.eval(Q).items()}
    with pytest.raises(L.LipError) as e:
        m.check()
    assert e.value.status == L.LIP_ERR_NONFINITE
    m.check()                                  # reported once
    Xf, yf = Xb.copy(), yb.copy()
    for i in (3, 17, 150):
        Xf[i], yf[i] = p.X[0], p.y[0]
    Xall = np.concatenate([p.X, Xf]).astype(np.float64)
    yall = np.concatenate([p.y, yf]).astype(np.float64)
    orc = oracle_mod.evaluate(Xall, yall, p.Q, p.M, p.norm)
    tol = FP64_TOL if precision == "fp64" else FP32_TOL
    pf = W.Problem("d", Xall, yall, p.Q, p.M, p.norm, None, None)
    compare(pf, r, orc, tol, f"deferred {precision}")
    # an empty handle whose first new point is bad takes the first finite new point
    e2 = model()
    e2.add_async(torch.as_tensor(Xb[3:]).to("cuda", dt), torch.as_tensor(yb[3:]).to("cuda", dt))
    with pytest.raises(L.LipError):
        e2.check()
    Xg, yg = Xb[3:].copy(), yb[3:].copy()
    for i in (0, 14, 147):                     # rows 3, 17, 150 of the batch
        Xg[i], yg[i] = Xb[4], yb[4]
    orc = oracle_mod.evaluate(Xg.astype(np.float64), yg.astype(np.float64), p.Q, p.M, p.norm)
    r = {k: v.cpu().numpy() for k, v in e2.eval(Q).items()}
    compare(W.Problem("e", Xg, yg, p.Q, p.M, p.norm, None, None), r, orc, tol, f"deferred empty {precision}")
    for h in (ref, m, e2):
        h.close()
