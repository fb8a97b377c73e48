"""GPU parity of lip_estimate_M and lip_backward against the FP64 oracle; gradcheck of the
autograd Function on an FP64 handle.  Needs a CUDA device."""
import numpy as np
import pytest

from paper_2606_04670_b300 import workloads as W
from parity import diam

pytestmark = pytest.mark.gpu

NORMS = (W.NORM_L1, W.NORM_L2, W.NORM_LINF)


def _model(p, precision="fp32", M=None):
    import torch

    from paper_2606_04670_b300.lipfit import LipFit
    dt = torch.float64 if precision == "fp64" else torch.float32
    return LipFit(torch.as_tensor(p.X).to("cuda", dt), torch.as_tensor(p.y).to("cuda", dt),
                  p.M if M is None else M, norm=p.norm, mon=p.mon, w=p.w, precision=precision)


def _ratio(p, i, j):
    v = np.abs(p.X[i].astype(np.float64) - p.X[j].astype(np.float64))
    if p.w is not None:
        v = v * p.w
    dist = {1: v.sum(), 2: np.sqrt((v * v).sum()), 3: v.max()}[p.norm]
    return abs(float(p.y[i]) - float(p.y[j])) / dist


@pytest.mark.parametrize("norm", NORMS)
@pytest.mark.parametrize("N,d,weighted", [(2, 1, False), (700, 3, True), (2_500, 4, False), (1_537, 9, True),
                                          (999, 16, False)])
def test_estimate_M_small(oracle_mod, norm, N, d, weighted):
    p = W.random_problem(500 + d, N, d, 1, norm=norm, weighted=weighted, masked=True)
    m = _model(p)
    M, i, j = m.lipschitz_constant()
    m.close()
    Mo, io, jo = oracle_mod.estimate_M(p.X, p.y, norm, w=p.w)
    assert abs(M - Mo) <= 1e-5 * Mo, (M, Mo)
    assert 0 <= i < j < N
    assert abs(_ratio(p, i, j) - M) <= 1e-12 * M      # reported value is the FP64 ratio of (i, j)


def test_estimate_M_duplicates():
    X = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 0.0], [0.5, 0.5]], np.float32)
    p = W.random_problem(510, 4, 2, 1)
    p.X = X
    # pairs (0,1) and (1,2) have ratio 1, (0,3), (1,3), (2,3) ratio 0.5/sqrt(0.5) = 0.707,
    # (0,2) is a duplicate with equal y and is skipped
    p.y = np.array([0.0, 1.0, 0.0, 0.5], np.float32)
    m = _model(p)
    M, i, j = m.lipschitz_constant()
    assert M == pytest.approx(1.0) and (i, j) == (0, 1)
    m.close()
    p.y = np.array([0.0, 1.0, 0.5, 0.5], np.float32)
    m = _model(p)
    M, i, j = m.lipschitz_constant()
    assert M == np.inf and (i, j) == (0, 2)
    m.close()


@pytest.mark.parametrize("norm", NORMS)
def test_estimate_M_full_size(oracle_mod, norm):
    """N = 1e5 on the GPU; the oracle on a 5,000-point subsample bounds it from below,
    the closed-form M from above, and the same subsample is checked exactly."""
    p = W.monotone_d4(norm=norm, n_query=1)
    m = _model(p)
    M, i, j = m.lipschitz_constant()
    m.close()
    assert abs(_ratio(p, i, j) - M) <= 1e-12 * M
    sub = np.random.default_rng(11).choice(p.N, 5000, replace=False)
    ps = W.monotone_d4(norm=norm, n_query=1)
    ps.X, ps.y = p.X[sub], p.y[sub]
    Ms, _, _ = oracle_mod.estimate_M(ps.X, ps.y, norm)
    assert Ms * (1 - 1e-6) <= M <= p.M * (1 + 1e-6)
    m = _model(ps)
    Mg, _, _ = m.lipschitz_constant()
    m.close()
    assert abs(Mg - Ms) <= 1e-5 * Ms


@pytest.mark.parametrize("norm", NORMS)
@pytest.mark.parametrize("masked,weighted", [(False, False), (True, True)])
def test_backward_vs_oracle(oracle_mod, norm, masked, weighted):
    import torch
    p = W.random_problem(600 + norm, 5_000, 6, 2_000, norm=norm, masked=masked, weighted=weighted,
                         decreasing=masked)
    m = _model(p)
    Q = torch.as_tensor(p.Q).cuda()
    r = m.eval(Q)
    gbar = torch.as_tensor(np.random.default_rng(2).uniform(-1, 1, p.nq).astype(np.float32)).cuda()
    gQ, gy, gM = m.backward(Q, r["idx_up"], r["idx_lo"], gbar)
    torch.cuda.synchronize()
    m.close()
    oQ, oy, oM = oracle_mod.gradient(p.X, p.y, p.Q, p.M, r["idx_up"].cpu().numpy(), r["idx_lo"].cpu().numpy(),
                                     gbar.cpu().numpy().astype(np.float64), norm, p.mon, p.w)
    np.testing.assert_allclose(gQ.cpu().numpy(), oQ, rtol=1e-4, atol=1e-4 * p.M)
    np.testing.assert_allclose(gy.cpu().numpy(), oy, rtol=1e-6, atol=1e-6)
    assert abs(gM.item() - oM) <= 1e-4 * max(1.0, abs(oM))


def test_backward_grad_d8(oracle_mod):
    """The differentiation workload (d=8, monotone in x1..x4, L2): GPU backward vs the
    oracle's analytic gradient on 10,000 queries, and against central differences of
    the FP64 oracle (h = 1e-3) on 1,000 queries whose argmin/argmax are stable."""
    import torch
    p = W.grad_d8(n_query=10_000)
    m = _model(p)
    Q = torch.as_tensor(p.Q).cuda()
    r = m.eval(Q)
    gbar = torch.ones(p.nq, device="cuda")
    gQ, gy, gM = m.backward(Q, r["idx_up"], r["idx_lo"], gbar)
    torch.cuda.synchronize()
    m.close()
    iu, il = r["idx_up"].cpu().numpy(), r["idx_lo"].cpu().numpy()
    oQ, oy, oM = oracle_mod.gradient(p.X, p.y, p.Q, p.M, iu, il, None, p.norm, p.mon, p.w)
    np.testing.assert_allclose(gQ.cpu().numpy(), oQ, rtol=1e-4, atol=1e-4 * p.M)
    np.testing.assert_allclose(gy.cpu().numpy(), oy, rtol=1e-6, atol=1e-6)
    assert abs(gM.item() - oM) <= 1e-4 * abs(oM)
    # finite differences of the FP64 oracle on the first 1,000 queries with gap > 1e-3
    h = 1e-3
    Qs = p.Q[:1000].astype(np.float64)
    o = oracle_mod.evaluate(p.X, p.y, Qs, p.M, p.norm, mon=p.mon)
    ok = (o.gap_up > 1e-3) & (o.gap_lo > 1e-3) & (o.idx_up == iu[:1000]) & (o.idx_lo == il[:1000])
    checked = 0
    for i in range(p.d):
        E = np.zeros(p.d)
        E[i] = h
        a = oracle_mod.evaluate(p.X, p.y, Qs + E, p.M, p.norm, mon=p.mon)
        b = oracle_mod.evaluate(p.X, p.y, Qs - E, p.M, p.norm, mon=p.mon)
        st = ok & (a.idx_up == o.idx_up) & (b.idx_up == o.idx_up) & (a.idx_lo == o.idx_lo) & (b.idx_lo == o.idx_lo)
        # no kink of a positive part within h
        st &= np.abs(Qs[:, i] - p.X[o.idx_up, i]) > h
        st &= np.abs(Qs[:, i] - p.X[o.idx_lo, i]) > h
        fd = (a.g - b.g) / (2 * h)
        np.testing.assert_allclose(gQ.cpu().numpy()[:1000][st, i], fd[st], rtol=1e-3, atol=1e-3)
        checked += int(st.sum())
    assert checked > 2000


def test_backward_grad_d8_full_size(oracle_mod):
    """The differentiation workload at the benchmark's size (N = 200,000, Q = 262,144): the
    backward pass of the GPU's own argmin/argmax against the oracle's analytic gradient on
    every query (given the indices, the gradient is O(Q d), so the oracle takes all of it)."""
    import torch
    p = W.grad_d8()
    m = _model(p)
    Q = torch.as_tensor(p.Q).cuda()
    r = m.eval(Q)
    gbar = torch.as_tensor(np.random.default_rng(5).uniform(0.5, 1.5, p.nq).astype(np.float32)).cuda()
    gQ, gy, gM = m.backward(Q, r["idx_up"], r["idx_lo"], gbar)
    torch.cuda.synchronize()
    m.close()
    iu, il = r["idx_up"].cpu().numpy(), r["idx_lo"].cpu().numpy()
    assert (iu >= 0).all() and (il >= 0).all()
    oQ, oy, oM = oracle_mod.gradient(p.X, p.y, p.Q, p.M, iu, il, gbar.cpu().numpy().astype(np.float64), p.norm,
                                     p.mon, p.w)
    np.testing.assert_allclose(gQ.cpu().numpy(), oQ, rtol=1e-4, atol=1e-4 * p.M)
    np.testing.assert_allclose(gy.cpu().numpy(), oy, rtol=1e-5, atol=1e-5 * np.abs(oy).max())
    assert abs(gM.item() - oM) <= 1e-4 * max(1.0, abs(oM))


def test_autograd_gradcheck_fp64():
    import torch

    from paper_2606_04670_b300.lipfit import LipEvalFn, LipFit
    p = W.random_problem(700, 40, 3, 12, norm=W.NORM_L2, masked=True, dtype=np.float64)
    X = torch.as_tensor(p.X).cuda()
    y = torch.as_tensor(p.y).cuda().requires_grad_(True)
    M = torch.tensor(p.M, dtype=torch.float64, device="cuda", requires_grad=True)
    m = LipFit(X, y.detach(), p.M, norm=p.norm, mon=p.mon, precision="fp64")
    Q = torch.as_tensor(p.Q).cuda().requires_grad_(True)
    g = LipEvalFn.apply(Q, y, M, m)
    g.sum().backward()
    # Q-gradient by central differences of the GPU FP64 forward, away from switches
    eps = 1e-6
    for i in range(3):
        E = torch.zeros_like(Q)
        E[:, i] = eps
        gp = m.values((Q + E).detach())
        gm = m.values((Q - E).detach())
        fd = (gp - gm) / (2 * eps)
        close = torch.isclose(Q.grad[:, i], fd, rtol=1e-5, atol=1e-7)
        assert close.float().mean() > 0.9       # a few queries may sit within eps of a switch
    assert y.grad is not None and abs(y.grad.sum().item() - p.nq) < 1e-9   # each query: 1/2 + 1/2
    assert M.grad is not None
    m.close()


def test_backward_deterministic_mode(oracle_mod):
    """deterministic=True: grad_y bitwise identical across runs and equal to the atomic path
    within rounding; grad_Q and grad_M unchanged."""
    import torch

    from paper_2606_04670_b300.lipfit import LipFit
    p = W.grad_d8(n_data=5_000, n_query=40_000)
    m = LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), p.M, norm=p.norm, mon=p.mon)
    Q = torch.as_tensor(p.Q).cuda()
    r = m.eval(Q)
    gb = torch.as_tensor(np.random.default_rng(2).standard_normal(p.nq).astype(np.float32)).cuda()
    a = m.backward(Q, r["idx_up"], r["idx_lo"], gb)
    b1 = m.backward(Q, r["idx_up"], r["idx_lo"], gb, deterministic=True)
    b2 = m.backward(Q, r["idx_up"], r["idx_lo"], gb, deterministic=True)
    torch.cuda.synchronize()
    assert torch.equal(b1[1], b2[1]) and torch.equal(b1[0], a[0]) and torch.equal(b1[2], a[2])
    np.testing.assert_allclose(b1[1].cpu().numpy(), a[1].cpu().numpy(), rtol=1e-5, atol=1e-5)
    _, oy, _ = oracle_mod.gradient(p.X, p.y, p.Q, p.M, r["idx_up"].cpu().numpy(), r["idx_lo"].cpu().numpy(),
                                   gb.cpu().numpy().astype(np.float64), p.norm, p.mon)
    np.testing.assert_allclose(b1[1].cpu().numpy(), oy, rtol=1e-5, atol=1e-5)
    m.close()
