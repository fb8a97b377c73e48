"""Dimensions above 16, up to LIP_D_MAX = 32, on every path against the FP64 oracle:
the plain evaluation (generic FP32 kernel) with monotone and weighted coordinates, FP64
handles (FP32 screen + FP64 candidates), the three tensor-core forms (K = 24 / 32 with a
shorter ring), the estimate (wide kernel), the backward pass, k > 1 neighbours, local
constants, smoothing and the batched launch.  d = 33 is refused."""
import numpy as np
import pytest

from paper_2606_04670_b300 import workloads as W
from parity import FP32_TOL, FP64_TOL, compare, diam, gpu_eval

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

WIDE = (17, 24, 32)


def _model(p, precision="fp32", M=None):
    from paper_2606_04670_b300.lipfit import LipFit
    dt = torch.float64 if precision == "fp64" else torch.float32
    return LipFit(torch.as_tensor(p.X).to("cuda", dt), torch.as_tensor(p.y).to("cuda", dt), p.M if M is None else M,
                  norm=p.norm, mon=p.mon, w=p.w, precision=precision)


@pytest.mark.parametrize("norm", (1, 2, 3))
@pytest.mark.parametrize("d", WIDE)
def test_eval_wide(oracle_mod, norm, d):
    p = W.random_problem(1100 + d, 4_111, d, 555, norm=norm, masked=True, weighted=True, decreasing=True)
    orc = oracle_mod.evaluate(p.X, p.y, p.Q, p.M, norm, mon=p.mon, w=p.w)
    compare(p, gpu_eval(p), orc, FP32_TOL, f"fp32 d={d} L{norm}")
    # tile and split choices do not change the results
    a = gpu_eval(p, splits=3)
    b = gpu_eval(p, splits=1)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])


@pytest.mark.parametrize("norm", (1, 2, 3))
def test_eval_wide_fp64(oracle_mod, norm):
    for d, masked in ((20, True), (32, False)):
        p = W.random_problem(1150 + d, 1_700, d, 300, norm=norm, masked=masked, weighted=True, decreasing=masked,
                             dtype=np.float64)
        orc = oracle_mod.evaluate(p.X, p.y, p.Q, p.M, norm, mon=p.mon, w=p.w)
        compare(p, gpu_eval(p, "fp64"), orc, FP64_TOL, f"fp64 d={d} L{norm}")
        compare(p, gpu_eval(p, "fp64", variant=1), orc, FP64_TOL, f"fp64 scan d={d} L{norm}")


@pytest.mark.parametrize("prec", ["tc_tf32", "tc_bf16", "tc_fp16"])
@pytest.mark.parametrize("d", WIDE)
def test_tensor_core_wide(oracle_mod, prec, d):
    p = W.random_problem(1200 + d, 6_001, d, 901, norm=W.NORM_L2, weighted=(d == 24))
    orc = oracle_mod.evaluate(p.X, p.y, p.Q, p.M, p.norm, w=p.w)
    m = _model(p, prec)
    r = {k: v.cpu().numpy() for k, v in m.eval(torch.as_tensor(p.Q).cuda()).items()}
    fb = m.last_fallback()
    m.check()
    m.close()
    compare(p, r, orc, FP32_TOL, f"{prec} d={d}")
    # the rescreened bounds are the FP64 envelopes rounded once
    for k in ("hi", "lo"):
        np.testing.assert_allclose(r[k], orc[k].astype(np.float32), rtol=0, atol=2e-7 * (1 + np.abs(orc[k]).max()))
    assert fb <= p.nq // 50, fb


@pytest.mark.parametrize("norm", (1, 2, 3))
@pytest.mark.parametrize("d", WIDE)
def test_estimate_wide(oracle_mod, norm, d):
    p = W.random_problem(1300 + d, 1_600, d, 1, norm=norm, weighted=True)
    m = _model(p, M=1.0)
    M, i, j = m.lipschitz_constant()
    parts = [m.estimate_M_part(k, 3) for k in range(3)]
    m.close()
    Mo, io, jo = oracle_mod.estimate_M(p.X, p.y, norm, w=p.w)
    assert abs(M - Mo) <= 1e-6 * Mo and (i, j) == (io, jo), (M, Mo, i, j, io, jo)
    from paper_2606_04670_b300 import shard as S
    best = [0.0, -1.0, -1.0, -1.0]
    for c in parts:
        if S._better(c, best):
            best = c
    assert (best[0], int(best[1]), int(best[2])) == (M, i, j)


def test_noalloc_estimate_wide(oracle_mod):
    from paper_2606_04670_b300 import lipfit as L
    p = W.random_problem(1350, 3_000, 29, 1, norm=W.NORM_L2)
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    s = L.lip_estimate_M_noalloc(torch.as_tensor(p.X).cuda().data_ptr(), torch.as_tensor(p.y).cuda().data_ptr(),
                                 p.N, p.d, p.norm, None, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert s == L.LIP_OK
    M, i, j = out.cpu().tolist()
    Mo, io, jo = oracle_mod.estimate_M(p.X, p.y, p.norm)
    assert abs(M - Mo) <= 1e-6 * Mo and (int(i), int(j)) == (io, jo)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_backward_wide(oracle_mod, prec):
    dt = torch.float64 if prec == "fp64" else torch.float32
    p = W.random_problem(1400, 3_000, 24, 1_000, norm=W.NORM_L2, masked=True, weighted=True, decreasing=True,
                         dtype=np.float64 if prec == "fp64" else np.float32)
    m = _model(p, prec)
    Q = torch.as_tensor(p.Q).to("cuda", dt)
    r = m.eval(Q)
    gbar = torch.as_tensor(np.random.default_rng(4).uniform(-1, 1, p.nq)).to("cuda", dt)
    gQ, gy, gM = m.backward(Q, r["idx_up"], r["idx_lo"], gbar)
    torch.cuda.synchronize()
    m.close()
    oQ, oy, oM = oracle_mod.gradient(p.X, p.y, p.Q, p.M, r["idx_up"].cpu().numpy(), r["idx_lo"].cpu().numpy(),
                                     gbar.cpu().numpy().astype(np.float64), p.norm, p.mon, p.w)
    rt = 1e-10 if prec == "fp64" else 1e-4
    np.testing.assert_allclose(gQ.cpu().numpy(), oQ, rtol=rt, atol=rt * p.M)
    np.testing.assert_allclose(gy.cpu().numpy(), oy, rtol=rt, atol=rt)
    assert abs(gM.item() - oM) <= rt * max(1.0, abs(oM))


@pytest.mark.parametrize("d,k", [(20, 3), (32, 8)])
def test_k_neighbours_wide(oracle_mod, d, k):
    p = W.random_problem(1500 + d, 2_000, d, 300, norm=(d % 3) + 1, masked=True, weighted=True)
    wk = np.random.default_rng(k).random(k)
    wk /= wk.sum()
    m = _model(p)
    r = {key: v.cpu().numpy() for key, v in m.eval_k(torch.as_tensor(p.Q).cuda(), k, wk).items()}
    m.close()
    o = oracle_mod.evaluate_k(p.X, p.y, p.Q, p.M, k, wk, p.norm, mon=p.mon, w=p.w)
    tol = FP32_TOL * p.M * diam(p.X, p.Q, p.norm, p.w)
    for key in ("hi", "lo", "g"):
        assert np.abs(r[key].astype(np.float64) - o[key]).max() <= tol, key


def test_local_constants_wide():
    import oracle as O
    from test_gpu_local import _check_eval, _table
    p = W.random_problem(1600, 1_200, 24, 300, norm=W.NORM_L2, weighted=True)
    m = _model(p, M=1.0)
    X, y, Q = (np.asarray(a, np.float64) for a in (p.X, p.y, p.Q))
    T = m.compute_local_lipschitz(12, 4000, 3)
    assert np.array_equal(T, O.local_knots(X, 12, 4000, 3, p.norm, w=p.w)[0])
    tab = _table(m)
    for a, b in zip(tab, O.local_table(X, y, T, p.norm, w=p.w)):
        assert np.array_equal(a, b)
    _check_eval(p, X, y, Q, T, tab, m.eval_local(torch.as_tensor(p.Q).cuda()), "local d=24")
    m.close()


def test_smoothing_objective_wide():
    import oracle as O
    p = W.random_problem(1700, 800, 20, 1, norm=W.NORM_L1, masked=True, weighted=True)
    y = (p.y.astype(np.float64) + 0.3 * np.random.default_rng(0).standard_normal(p.N)).astype(np.float32)
    p = W.Problem(p.name, p.X, y, p.Q, p.M, p.norm, p.mon, p.w, p.f)
    m = _model(p)
    eps = 0.05 * np.random.default_rng(1).standard_normal(p.N)
    M, pen = 0.7 * p.M, 50.0
    f, g = m.smooth_objective(torch.as_tensor(eps).cuda(), M, pen)
    fo, go, _, _ = O.smooth_objective(p.X, p.y, eps, M, pen, p.norm, mon=p.mon, w=p.w)
    m.close()
    assert abs(f - fo) <= 1e-4 * max(fo, 1.0), (f, fo)
    assert np.abs(g.cpu().numpy() - go).max() <= 1e-3 * max(1.0, np.abs(go).max())


def test_batch_wide_sets_equal_single_set_eval(oracle_mod):
    from paper_2606_04670_b300.lipfit import LipBatch
    probs = [W.random_problem(1800 + d, 700 + 37 * d, d, 150 + d, norm=(d % 3) + 1, masked=(d % 2 == 1),
                              weighted=True, decreasing=(d % 2 == 1)) for d in (3, 12, 17, 32, 10)]
    sets = [dict(X=torch.as_tensor(p.X), y=torch.as_tensor(p.y), Q=torch.as_tensor(p.Q), M=p.M, norm=p.norm,
                 mon=p.mon, w=p.w) for p in probs]
    b = LipBatch(sets)
    b.eval()
    torch.cuda.synchronize()
    b.check()
    for p, out in zip(probs, b.outputs):
        got = {k: v.cpu().numpy() for k, v in out.items()}
        ref = gpu_eval(p)
        orc = oracle_mod.evaluate(p.X, p.y, p.Q, p.M, p.norm, mon=p.mon, w=p.w)
        compare(p, got, orc, FP32_TOL, f"batch d={p.d}")
        if p.d <= 10:        # the exact bodies equal lip_eval bit for bit
            for k in got:
                np.testing.assert_array_equal(got[k], ref[k], err_msg=f"d={p.d} {k}")
        else:                # both pick by their own FP32 values: the same FP64 values up to ties
            compare(p, got, {k: orc[k] for k in orc}, FP32_TOL, f"batch d={p.d} vs oracle")
    b.close()


def test_dimension_limit():
    from paper_2606_04670_b300 import lipfit as L
    assert L.LIP_D_MAX == 32
    X = torch.zeros(4, 33, device="cuda")
    y = torch.zeros(4, device="cuda")
    params, keep = L.make_params()
    s, h = L.lip_fit(X.data_ptr(), y.data_ptr(), 4, 33, 1.0, params)
    assert s == L.LIP_ERR_ARG and not h.value
