"""Penalty smoothing (Sec. 4.4, Eq. (optim)) on the GPU against the FP64 oracle.

The objective pass forms every pair term in FP32 and sums in FP64 (FP64 handles: FP64
pair terms, checked separately).  A term
v = z_i - z_k - M d has an FP32 error below 2^-20 (|z_i| + |z_k| + M d) (the scaled
coordinates, the distance and two subtractions, each a few ulps); a row of the gradient
adds 4 N such terms, and the objective adds 2 |v| dv per positive term.  The tolerances
below are those sums.  The L-BFGS result is checked through the objective's strong
convexity (modulus 2/p): any point x lies within (p/2) |grad Phi(x)|_2 of the unique
minimiser, so the GPU's and the oracle's results lie within (p/2) of the sum of their exact
gradient norms, which the oracle evaluates."""
import numpy as np
import pytest

import oracle as O
from paper_2606_04670_b300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EPS32 = 2.0 ** -20


def _model(p, precision="fp32"):
    from paper_2606_04670_b300.lipfit import LipFit
    dt = torch.float64 if precision == "fp64" else torch.float32
    return LipFit(torch.as_tensor(p.X).to("cuda", dt), torch.as_tensor(p.y).to("cuda", dt), p.M, norm=p.norm,
                  mon=p.mon, w=p.w, precision=precision, capacity=p.N + 8)


def _noisy(seed, N, d, norm, masked=False, weighted=False, decreasing=False, noise=0.4):
    p = W.random_problem(seed, N, d, 1, norm=norm, masked=masked, weighted=weighted, decreasing=decreasing)
    r = np.random.default_rng(seed)
    y = (p.y.astype(np.float64) + noise * r.standard_normal(N)).astype(np.float32)
    return W.Problem(p.name, p.X, y, p.Q, p.M, norm, p.mon, p.w, p.f, p.M_by_norm)


def _scale(p, M):
    Z = np.asarray(p.X, np.float64) * (1.0 if p.w is None else np.asarray(p.w))
    span = Z.max(0) - Z.min(0)
    diam = {1: span.sum(), 2: float(np.sqrt((span ** 2).sum())), 3: span.max()}[p.norm]
    return 2.0 * float(np.abs(p.y).max()) + M * diam + 1.0


CASES = []
for _norm in (1, 2, 3):
    CASES.append(_noisy(400 + _norm, 37, 2, _norm))
    CASES.append(_noisy(410 + _norm, 700, 3, _norm, masked=True, weighted=True, decreasing=True))
    CASES.append(_noisy(420 + _norm, 1500, 5, _norm, weighted=True))
CASES.append(_noisy(430, 900, 16, 2, masked=True))
CASES.append(_noisy(431, 600, 1, 1, masked=True))


@pytest.mark.parametrize("case", range(len(CASES)), ids=lambda i: f"L{CASES[i].norm}-N{CASES[i].N}-d{CASES[i].d}")
def test_objective_and_gradient_match_oracle(case):
    p = CASES[case]
    m = _model(p)
    r = np.random.default_rng(case)
    M, pen = 1.3 * p.M, 50.0
    for scale in (0.0, 0.05):
        eps = scale * r.standard_normal(p.N)
        f, g = m.smooth_objective(torch.as_tensor(eps).cuda(), M, pen)
        g = g.cpu().numpy()
        fo, go, s1, s2 = O.smooth_objective(p.X, p.y, eps, M, pen, p.norm, mon=p.mon, w=p.w)
        dv = EPS32 * _scale(p, M)
        tol_g = 4.0 * p.N * dv + 1e-9
        assert np.abs(g - go).max() <= tol_g, (np.abs(g - go).max(), tol_g)
        # 2 S1 + 2 S2 terms: each positive v contributes 2 |v| dv (twice: both sums)
        tol_f = 4.0 * dv * (np.sqrt(s1 + s2) * p.N) + 1e-9 * max(fo, 1.0)
        assert abs(f - fo) <= tol_f, (f, fo, tol_f)
    m.close()


@pytest.mark.parametrize("case", range(len(CASES)), ids=lambda i: f"L{CASES[i].norm}-N{CASES[i].N}-d{CASES[i].d}")
def test_fp64_handles_use_fp64_pair_terms(case):
    """FP64 handles form the pair terms in FP64: each term's error is a few units of 2^-52
    of |z_i| + |z_k| + M d, and the column terms are summed in fixed point with a resolution
    of N (max z - min z) 2^-60 per term, so the gradient and the objective agree with the
    oracle far below the FP32 path's tolerance."""
    q = CASES[case]
    p = W.Problem(q.name, np.asarray(q.X, np.float64), np.asarray(q.y, np.float64), q.Q, q.M, q.norm, q.mon, q.w)
    m = _model(p, precision="fp64")
    r = np.random.default_rng(100 + case)
    M, pen = 1.3 * p.M, 50.0
    for scale in (0.0, 0.05):
        eps = scale * r.standard_normal(p.N)
        f, g = m.smooth_objective(torch.as_tensor(eps).cuda(), M, pen)
        fo, go, s1, s2 = O.smooth_objective(p.X, p.y, eps, M, pen, p.norm, mon=p.mon, w=p.w)
        sc = _scale(p, M)
        tol_g = 4.0 * p.N * 2.0 ** -45 * sc + p.N ** 2 * sc * 2.0 ** -58
        err = np.abs(g.cpu().numpy() - go).max()
        assert err <= tol_g, (err, tol_g)
        assert abs(f - fo) <= 1e-10 * max(fo, 1.0) + 4.0 * 2.0 ** -45 * sc * np.sqrt(s1 + s2) * p.N, (f, fo)
    m.close()


def test_smooth_matches_oracle_minimiser():
    for k, p in enumerate([CASES[0], CASES[1], _noisy(440, 250, 4, 2, masked=True), _noisy(441, 300, 3, 3)]):
        M, pen = p.M, 30.0
        m = _model(p)
        eps, f, it, ev = m.smooth_lipschitz(M, pen, max_iter=500, gtol=1e-7)
        assert it >= 1 and ev >= it + 1
        e_gpu = eps.cpu().numpy()
        e_or, f_or, _ = O.smooth(p.X, p.y, M, pen, p.norm, mon=p.mon, w=p.w, max_iter=1000, gtol=1e-6)
        fg, gg, _, _ = O.smooth_objective(p.X, p.y, e_gpu, M, pen, p.norm, mon=p.mon, w=p.w)
        _, go, _, _ = O.smooth_objective(p.X, p.y, e_or, M, pen, p.norm, mon=p.mon, w=p.w)
        bound = pen / 2.0 * (np.linalg.norm(gg) + np.linalg.norm(go))
        assert np.abs(e_gpu - e_or).max() <= bound, (k, np.abs(e_gpu - e_or).max(), bound)
        assert bound <= 5e-2 * max(1.0, np.abs(e_or).max()), (k, bound)
        dv = EPS32 * _scale(p, M)
        assert abs(f - fg) <= 4.0 * dv * np.sqrt(fg) * p.N + 1e-9 * max(fg, 1.0), (k, f, fg)
        # the handle now holds y + eps and the constant M: lip_eval is the oracle on those data
        assert m.M == M
        ys = (p.y.astype(np.float64) + e_gpu).astype(np.float32)
        Q = np.random.default_rng(k).random((200, p.d)).astype(np.float32)
        out = m.eval(torch.as_tensor(Q).cuda())
        ro = O.evaluate(p.X, ys, Q, M, p.norm, mon=p.mon, w=p.w)
        tol = 1e-5 * _scale(p, M)
        assert np.abs(out["hi"].cpu().numpy() - ro.hi).max() <= tol
        assert np.abs(out["lo"].cpu().numpy() - ro.lo).max() <= tol
        m.close()


def test_two_points_closed_form():
    X = np.array([[0.0, 0.0], [0.6, 0.8]], np.float32)
    y = np.array([2.0, -1.0], np.float32)
    p = W.Problem("two", X, y, X, 1.0, 2, None, None)
    for pen in (1.0, 100.0):
        m = _model(p)
        eps, f, it, _ = m.smooth_lipschitz(1.0, pen, max_iter=100, gtol=1e-10)
        a = 3.0 - 1.0
        t = 2 * a * pen / (1 + 4 * pen)
        assert np.allclose(eps.cpu().numpy(), [-t, t], rtol=1e-5, atol=1e-6)
        m.close()


def test_consistent_data_unchanged_and_errors():
    from paper_2606_04670_b300.lipfit import LIP_ERR_ARG, LipError
    p = W.random_problem(450, 300, 3, 1, norm=2)
    m = _model(p)
    f0, g0 = m.smooth_objective(torch.zeros(p.N, dtype=torch.float64, device="cuda"), p.M, 10.0)
    assert f0 == 0.0 and torch.all(g0 == 0)
    eps, f, it, ev = m.smooth_lipschitz(p.M, 10.0)
    assert it == 0 and ev == 1 and f == 0.0 and torch.all(eps == 0)
    for kw in ({"p": 0.0}, {"p": float("inf")}, {"history": 0}, {"max_iter": -1}):
        args = dict(M=p.M, p=10.0)
        args.update(kw)
        with pytest.raises(LipError) as e:
            m.smooth_lipschitz(**args)
        assert e.value.status == LIP_ERR_ARG
    m.close()
    # FP64 handles smooth too: objective and gradient against the oracle, y + eps kept in FP64
    q = _noisy(451, 300, 2, 2)
    q = W.Problem(q.name, q.X.astype(np.float64), q.y.astype(np.float64), q.Q, q.M, 2, None, None)
    m = _model(q, precision="fp64")
    eps0 = 0.01 * np.random.default_rng(1).standard_normal(q.N)
    f, g = m.smooth_objective(torch.as_tensor(eps0).cuda(), q.M, 10.0)
    fo, go, _, _ = O.smooth_objective(q.X, q.y, eps0, q.M, 10.0, 2)
    assert np.abs(g.cpu().numpy() - go).max() <= 1e-9 * _scale(q, q.M)
    eps, f, it, _ = m.smooth_lipschitz(q.M, 10.0)
    out = m.eval(torch.as_tensor(q.X).cuda())
    ro = O.evaluate(q.X, q.y + eps.cpu().numpy(), q.X, q.M, 2)
    assert np.abs(out["hi"].cpu().numpy() - ro.hi).max() <= 1e-10
    m.close()


def test_full_size_gradient_rows():
    """The benchmark's smoothing workload (N = 100,000): 48 gradient rows at a random eps
    against the oracle's O(N) rows, and Phi >= |eps|^2 / p."""
    p = W.smooth_d4()
    m = _model(p)
    M, pen = W.SMOOTH_M, W.SMOOTH_P
    eps = 0.02 * np.random.default_rng(0).standard_normal(p.N)
    f, g = m.smooth_objective(torch.as_tensor(eps).cuda(), M, pen)
    g = g.cpu().numpy()
    rows = np.random.default_rng(1).choice(p.N, 48, replace=False)
    go = O.smooth_grad_rows(p.X, p.y, eps, rows, M, pen, p.norm, mon=p.mon, w=p.w)
    tol = 4.0 * p.N * EPS32 * _scale(p, M)
    assert np.abs(g[rows] - go).max() <= tol, (np.abs(g[rows] - go).max(), tol)
    assert f >= eps @ eps / pen
    m.close()


def test_objective_reproducible_bit_for_bit():
    """The column terms arrive through atomics in any order; they are summed in 64-bit fixed
    point, so two evaluations at a point with many violating pairs agree bit for bit."""
    p = _noisy(460, 3000, 3, 2, noise=0.8)
    m = _model(p)
    eps = torch.as_tensor(0.3 * np.random.default_rng(3).standard_normal(p.N)).cuda()
    f1, g1 = m.smooth_objective(eps, 0.5 * p.M, 20.0)
    f2, g2 = m.smooth_objective(eps, 0.5 * p.M, 20.0)
    assert f1 == f2 and torch.equal(g1, g2)
    _, go, s1, _ = O.smooth_objective(p.X, p.y, eps.cpu().numpy(), 0.5 * p.M, 20.0, p.norm)
    assert s1 > 0.0 and np.abs(g1.cpu().numpy() - go).max() <= 4.0 * p.N * EPS32 * _scale(p, 0.5 * p.M)
    m.close()
