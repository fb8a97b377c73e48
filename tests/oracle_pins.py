"""Checks that pin the FP64 oracle to facts fixed by the paper and by mathematics.

Each check takes an ``Oracle`` instance, so the same checks can be run against
deliberately broken copies of the oracle (see test_oracle_mutants.py).  None of
them retypes the oracle's formula: they compare against hand-derived values,
an O(log N) 1-D closed form, scipy's distance routines, finite differences, or
inequalities the optimal interpolant must satisfy.
"""
from __future__ import annotations

import bisect
import json
import os

import numpy as np
from scipy.spatial.distance import cdist, pdist, squareform

from paper_2606_04670_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "hand_examples.json")
GOLDEN_LOCAL = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "local_lipschitz_1d.json")
GOLDEN_SPLITMIX = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "splitmix64.json")
METRIC = {1: "cityblock", 2: "euclidean", 3: "chebyshev"}


def _scaled(Z, w):
    return Z if w is None else Z * np.asarray(w)[None, :]


# ---------------------------------------------------------------- hand examples

def check_hand_examples(O):
    """Sec. 3 Eq. (upperlower)/(eq:g), Sec. 4.1 Eq. (distmon), Sec. 5: worked by hand."""
    G = json.load(open(GOLDEN))
    e = G["one_d"]
    for norm in (1, 2, 3):
        r = O.evaluate(e["X"], e["y"], e["Q"], e["M"], norm)
        np.testing.assert_allclose(r.hi, e["hi"], atol=1e-15)
        np.testing.assert_allclose(r.lo, e["lo"], atol=1e-15)
        np.testing.assert_allclose(r.g, e["g"], atol=1e-15)
        assert list(r.idx_up) == e["idx_up"] and list(r.idx_lo) == e["idx_lo"]
        M, i, j = O.estimate_M(e["X"], e["y"], norm)
        assert abs(M - e["M_est"]) < 1e-15 and [i, j] == e["M_est_pair"]
    e = G["two_d"]
    for c in e["cases"]:
        mon = None if c["mon"] is None else np.array(c["mon"], np.int8)
        r = O.evaluate(e["X"], e["y"], e["Q"], e["M"], c["norm"], mon=mon, w=c["w"])
        assert abs(r.hi[0] - c["hi"]) < 1e-14, c
        assert abs(r.lo[0] - c["lo"]) < 1e-14, c
        assert abs(r.g[0] - 0.5 * (c["hi"] + c["lo"])) < 1e-14, c
        assert r.idx_up[0] == c["idx_up"] and r.idx_lo[0] == c["idx_lo"], c
    for norm, (Mv, i, j) in e["M_est"].items():
        M, a, b = O.estimate_M(e["X"], e["y"], int(norm))
        assert abs(M - Mv) < 1e-15 and (a, b) == (i, j)


# ------------------------------------------------------------- 1-D closed form

def closed_form_1d(xs, ys, M, q, mon):
    """H_up, H_lo of 1-D data consistent with M (and with the monotonicity).

    Sorted data; between neighbours x_j <= q < x_{j+1} only those two points
    matter (Sec. 4: the two neighbours lie on opposite sides in 1-D), giving
    the piecewise-linear 'sawtooth' with slopes +-M.  For increasing data
    (Sec. 4.1) the point to the right bounds from above with its own value and
    the point to the left bounds from below with its own value.
    """
    if mon < 0:
        hi, lo = closed_form_1d([-x for x in xs[::-1]], list(ys[::-1]), M, -q, 1)
        return hi, lo
    n = len(xs)
    j = bisect.bisect_right(xs, q) - 1
    up, dn = [], []
    if j >= 0:
        up.append(ys[j] + M * (q - xs[j]))
        dn.append(ys[j] if mon > 0 else ys[j] - M * (q - xs[j]))
    if j + 1 < n:
        up.append(ys[j + 1] if mon > 0 else ys[j + 1] + M * (xs[j + 1] - q))
        dn.append(ys[j + 1] - M * (xs[j + 1] - q))
    return min(up), max(dn)


def check_closed_form_1d(O):
    rng = np.random.default_rng(7)
    for mon in (0, 1, -1):
        for norm in (1, 2, 3):
            for wv in (None, 2.5):
                xs = np.sort(rng.uniform(0, 1, 40))
                if mon == 0:
                    ys = np.sin(5 * xs)
                    Mt = 5.0
                else:
                    ys = mon * (xs + 0.3 * np.sin(2 * xs))     # derivative in [0.4, 1.6]
                    Mt = 1.6
                M = 1.25 * Mt
                # a weight w on the only coordinate scales distances by w
                Meff = M * (1.0 if wv is None else wv)
                Q = np.concatenate([rng.uniform(-0.3, 1.3, 200), xs[:5]])
                r = O.evaluate(xs[:, None], ys, Q[:, None], M, norm,
                               mon=None if mon == 0 else np.array([mon], np.int8),
                               w=None if wv is None else [wv])
                for k, q in enumerate(Q):
                    hi, lo = closed_form_1d(list(xs), list(ys), Meff, q, mon)
                    assert abs(r.hi[k] - hi) < 1e-12, (mon, norm, q)
                    assert abs(r.lo[k] - lo) < 1e-12, (mon, norm, q)


# ------------------------------------------------- unmasked case = scipy cdist

def check_unmasked_cdist(O):
    """Unmasked envelopes are min/max of y +- M * cdist (library distance routine)."""
    for seed, (N, d, nq) in enumerate([(57, 3, 41), (200, 5, 64), (33, 1, 10), (90, 9, 30)]):
        for norm in (1, 2, 3):
            for weighted in (False, True):
                p = W.random_problem(seed, N, d, nq, norm=norm, weighted=weighted, dtype=np.float64)
                D = cdist(_scaled(p.Q, p.w), _scaled(p.X, p.w), METRIC[norm])
                up = p.y[None, :] + p.M * D
                dn = p.y[None, :] - p.M * D
                r = O.evaluate(p.X, p.y, p.Q, p.M, norm, w=p.w)
                np.testing.assert_allclose(r.hi, up.min(1), rtol=0, atol=1e-12)
                np.testing.assert_allclose(r.lo, dn.max(1), rtol=0, atol=1e-12)
                np.testing.assert_allclose(r.g, 0.5 * (up.min(1) + dn.max(1)), rtol=0, atol=1e-12)
                # first index of the extremum (ties -> lowest index), where the gap is clear
                su = np.sort(up, 1)
                ok = (su[:, 1] - su[:, 0]) > 1e-9
                assert np.all(r.idx_up[ok] == up.argmin(1)[ok])
                sl = np.sort(dn, 1)
                ok = (sl[:, -1] - sl[:, -2]) > 1e-9
                assert np.all(r.idx_lo[ok] == dn.argmax(1)[ok])
                # the reported gaps match the sorted values
                np.testing.assert_allclose(r.gap_up, su[:, 1] - su[:, 0], atol=1e-12)


# ------------------------------------------------------------------ invariants

def _problems():
    out = []
    for norm in (1, 2, 3):
        out.append(W.monotone_d4(norm=norm, n_data=400, n_query=300, dtype=np.float64))
        for masked, weighted, dec in [(False, False, False), (True, False, False),
                                      (True, True, True), (False, True, False)]:
            out.append(W.random_problem(11 + norm, 150, 4, 120, norm=norm, masked=masked,
                                        weighted=weighted, decreasing=dec, dtype=np.float64))
    out.append(W.plain_d2(dtype=np.float64, n_data=300, n_query=300))
    out.append(W.toy_d3(dtype=np.float64, n_data=300, n_query=300))
    out.append(W.grad_d8(dtype=np.float64, n_data=300, n_query=200))
    out.append(W.cluster_d16(dtype=np.float64, n_data=500, n_query=100))
    return out


def check_interpolation(O):
    """Data consistent with M (and the monotonicity) are interpolated: g(x^k)=y^k (Sec. 3)."""
    for p in _problems():
        r = O.evaluate(p.X, p.y, p.X, p.M, p.norm, mon=p.mon, w=p.w)
        np.testing.assert_allclose(r.hi, p.y, atol=1e-12)
        np.testing.assert_allclose(r.lo, p.y, atol=1e-12)
        np.testing.assert_allclose(r.g, p.y, atol=1e-12)


def check_enclosure(O):
    """H_lo <= f <= H_up for the generating f (Sec. 4: the bounds enclose every admissible f)."""
    for p in _problems():
        r = O.evaluate(p.X, p.y, p.Q, p.M, p.norm, mon=p.mon, w=p.w)
        fq = p.f(p.Q)
        assert np.all(r.lo <= fq + 1e-12), p.name
        assert np.all(fq <= r.hi + 1e-12), p.name


def _mono_gap(a, b, mon, w):
    """m(a-b): positive part on increasing coordinates, (b-a)_+ on decreasing, |.| elsewhere."""
    t = a - b
    m = np.abs(t)
    if mon is not None:
        m = np.where(mon > 0, np.maximum(t, 0), m)
        m = np.where(mon < 0, np.maximum(-t, 0), m)
    return m if w is None else m * np.asarray(w)


def _norm(v, norm):
    return {1: np.abs(v).sum(-1), 2: np.sqrt((v * v).sum(-1)), 3: np.abs(v).max(-1)}[norm]


def check_lipschitz_monotone(O):
    """g(a)-g(b) <= M ||w m(a-b)||: M-Lipschitz, and monotone where constrained (Sec. 4, 4.1)."""
    rng = np.random.default_rng(3)
    for p in _problems():
        n = 150
        A = rng.random((n, p.d))
        B = rng.random((n, p.d))
        # coordinate-step pairs along each coordinate
        i = rng.integers(0, p.d, n)
        C = A.copy()
        C[np.arange(n), i] = np.clip(A[np.arange(n), i] - rng.uniform(0, 0.2, n), 0, 1)
        for P1, P2 in ((A, B), (B, A), (A, C), (C, A)):
            r1 = O.evaluate(p.X, p.y, P1, p.M, p.norm, mon=p.mon, w=p.w)
            r2 = O.evaluate(p.X, p.y, P2, p.M, p.norm, mon=p.mon, w=p.w)
            bound = p.M * _norm(_mono_gap(P1, P2, p.mon, p.w), p.norm)
            for key in ("hi", "lo", "g"):
                assert np.all(r1[key] - r2[key] <= bound + 1e-12), (p.name, key)


def check_width_bound(O):
    """H_up - H_lo <= 2 M min_k dist_sym(q, x^k) (Sec. 3 error bound, twice the worst-case error)."""
    for p in _problems():
        r = O.evaluate(p.X, p.y, p.Q, p.M, p.norm, mon=p.mon, w=p.w)
        D = cdist(_scaled(p.Q, p.w), _scaled(p.X, p.w), METRIC[p.norm])
        assert np.all(r.hi - r.lo <= 2 * p.M * D.min(1) + 1e-12), p.name


def check_special_cases(O):
    rng = np.random.default_rng(5)
    for norm in (1, 2, 3):
        p = W.random_problem(21, 80, 3, 50, norm=norm, masked=True, dtype=np.float64)
        # M = 0: the bounds collapse to the data range
        r = O.evaluate(p.X, p.y, p.Q, 0.0, norm, mon=p.mon)
        assert np.all(r.hi == p.y.min()) and np.all(r.lo == p.y.max())
        assert np.all(r.idx_up == np.argmin(p.y)) and np.all(r.idx_lo == np.argmax(p.y))
        # M = 0 with the extreme value repeated: the lowest index is kept on the tie
        yt = p.y.copy()
        yt[[5, 9, 30]] = yt.min() - 1.0
        yt[[7, 12]] = yt.max() + 1.0
        r = O.evaluate(p.X, yt, p.Q, 0.0, norm, mon=p.mon)
        assert np.all(r.idx_up == 5) and np.all(r.idx_lo == 7)
        # N = 1, unmasked: y0 +- M * distance (numpy norm)
        X1, y1 = p.X[:1], p.y[:1]
        r = O.evaluate(X1, y1, p.Q, p.M, norm)
        dd = np.linalg.norm(p.Q - X1, ord={1: 1, 2: 2, 3: np.inf}[norm], axis=1)
        np.testing.assert_allclose(r.hi, y1[0] + p.M * dd, atol=1e-12)
        np.testing.assert_allclose(r.lo, y1[0] - p.M * dd, atol=1e-12)
        # huge M: both bounds pick the nearest neighbour (Sec. 4 "among the closest points")
        D = cdist(p.Q, p.X, METRIC[norm])
        Ds = np.sort(D, 1)
        ok = (Ds[:, 1] - Ds[:, 0]) > 1e-6
        r = O.evaluate(p.X, p.y, p.Q, 1e9, norm)
        nn = D.argmin(1)
        assert np.all(r.idx_up[ok] == nn[ok]) and np.all(r.idx_lo[ok] == nn[ok])
        # a query on a datum with the monotone distance: g = y there (Sec. 4.1)
        r = O.evaluate(p.X, p.y, p.X[:7], p.M, norm, mon=p.mon)
        np.testing.assert_allclose(r.g, p.y[:7], atol=1e-12)
    # monotone bounds: x below x^k (all coords) => H_up(x) <= y^k; x above => H_lo(x) >= y^k
    p = W.random_problem(22, 60, 3, 10, masked=True, dtype=np.float64)
    mon = np.ones(3, np.int8)
    for k in range(10):
        xk = p.X[k]
        below = xk - rng.uniform(0, 0.3, 3)
        above = xk + rng.uniform(0, 0.3, 3)
        r = O.evaluate(p.X, p.y, np.stack([below, above]), 50.0, 2, mon=mon)
        assert r.hi[0] <= p.y[k] + 1e-15 and r.lo[1] >= p.y[k] - 1e-15


def check_estimate_M(O):
    """M_est = max_{i<j} |dy| / dist (Sec. 5) against scipy pdist; M_est <= M_true; interpolation."""
    for seed, (N, d) in enumerate([(2, 1), (37, 2), (120, 4), (64, 7)]):
        for norm in (1, 2, 3):
            for weighted in (False, True):
                p = W.random_problem(30 + seed, N, d, 1, norm=norm, weighted=weighted, dtype=np.float64)
                D = pdist(_scaled(p.X, p.w), METRIC[norm])
                dy = pdist(p.y[:, None], "cityblock")
                ratio = dy / D
                M, i, j = O.estimate_M(p.X, p.y, norm, w=p.w)
                assert abs(M - ratio.max()) <= 1e-12 * ratio.max()
                R = squareform(ratio)
                assert abs(R[i, j] - M) <= 1e-12 * M and i < j
                srt = np.sort(ratio)
                if len(srt) > 1 and srt[-1] - srt[-2] > 1e-9:
                    iu = np.triu_indices(N, 1)
                    k = int(np.argmax(R[iu]))
                    assert (iu[0][k], iu[1][k]) == (i, j)
                assert M <= p.M_by_norm[norm] * (1 + 1e-12)
                r = O.evaluate(p.X, p.y, p.X, M, norm, w=p.w)
                np.testing.assert_allclose(r.g, p.y, atol=1e-12)
    # duplicates: equal y is skipped, different y gives +inf
    X = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 0.0]])
    assert O.estimate_M(X, np.array([0.0, 1.0, 0.0]))[0] == 1.0
    M, i, j = O.estimate_M(X, np.array([0.0, 1.0, 0.5]))
    assert M == np.inf and (i, j) == (0, 2)
    # constant y at distinct points: every ratio is 0, so M = 0 with the first pair;
    # only repeated points with equal y leave no pair at all (-1, -1)
    Xd = np.array([[0.3, 0.1], [0.9, 0.4], [0.2, 0.8]])
    for norm in (1, 2, 3):
        assert O.estimate_M(Xd, np.full(3, 2.5), norm) == (0.0, 0, 1)
        assert O.estimate_M(np.tile(Xd[:1], (4, 1)), np.full(4, 2.5), norm) == (0.0, -1, -1)
    # the configured workloads' closed-form M bounds the data's estimate
    for p in (W.plain_d2(dtype=np.float64, n_data=400), W.toy_d3(dtype=np.float64, n_data=400),
              W.grad_d8(dtype=np.float64, n_data=400)):
        assert O.estimate_M(p.X, p.y, p.norm)[0] <= p.M
    for norm in (1, 2, 3):
        p = W.monotone_d4(norm=norm, n_data=400, n_query=1, dtype=np.float64)
        assert O.estimate_M(p.X, p.y, norm)[0] <= p.M


def check_gradient_fd(O):
    """Analytic gradient = central finite differences of the oracle, away from kinks and ties."""
    h = 1e-6
    for norm in (1, 2, 3):
        for masked, weighted, dec in [(False, False, False), (True, True, True), (True, False, False)]:
            p = W.random_problem(40 + norm, 60, 3, 40, norm=norm, masked=masked, weighted=weighted,
                                 decreasing=dec, dtype=np.float64)
            r = O.evaluate(p.X, p.y, p.Q, p.M, norm, mon=p.mon, w=p.w)
            gbar = np.random.default_rng(1).uniform(-1, 1, p.nq)
            gQ, gy, gM = O.gradient(p.X, p.y, p.Q, p.M, r.idx_up, r.idx_lo, gbar, norm, p.mon, p.w)
            checked = 0
            for i in range(p.d):
                E = np.zeros(p.d)
                E[i] = h
                rp = O.evaluate(p.X, p.y, p.Q + E, p.M, norm, mon=p.mon, w=p.w)
                rm = O.evaluate(p.X, p.y, p.Q - E, p.M, norm, mon=p.mon, w=p.w)
                stable = ((rp.idx_up == r.idx_up) & (rm.idx_up == r.idx_up) &
                          (rp.idx_lo == r.idx_lo) & (rm.idx_lo == r.idx_lo) &
                          (r.gap_up > 1e-4) & (r.gap_lo > 1e-4))
                # stay away from coordinate kinks of the chosen pairs
                tu = p.Q[:, i] - p.X[r.idx_up, i]
                tl = p.Q[:, i] - p.X[r.idx_lo, i]
                stable &= (np.abs(tu) > 1e-4) & (np.abs(tl) > 1e-4)
                fd = (rp.g - rm.g) / (2 * h)
                np.testing.assert_allclose(gQ[stable, i], gbar[stable] * fd[stable], atol=2e-6)
                checked += int(stable.sum())
            assert checked > p.nq
            # dg/dM by finite differences in M (indices are stable for a tiny step)
            rp = O.evaluate(p.X, p.y, p.Q, p.M + h, norm, mon=p.mon, w=p.w)
            rm = O.evaluate(p.X, p.y, p.Q, p.M - h, norm, mon=p.mon, w=p.w)
            st = (rp.idx_up == r.idx_up) & (rm.idx_up == r.idx_up) & (rp.idx_lo == r.idx_lo) & (rm.idx_lo == r.idx_lo)
            fdM = (gbar * (rp.g - rm.g) / (2 * h))[st].sum()
            _, _, gM_st = O.gradient(p.X, p.y, p.Q[st], p.M, r.idx_up[st], r.idx_lo[st], gbar[st],
                                     norm, p.mon, p.w)
            assert abs(fdM - gM_st) < 1e-5 * max(1.0, abs(fdM))
            # dg/dy_k by finite differences in y_k for a few data points
            for k in np.unique(np.concatenate([r.idx_up[:5], r.idx_lo[:5]])):
                yp = p.y.copy()
                yp[k] += h
                ym = p.y.copy()
                ym[k] -= h
                a = O.evaluate(p.X, yp, p.Q, p.M, norm, mon=p.mon, w=p.w)
                b = O.evaluate(p.X, ym, p.Q, p.M, norm, mon=p.mon, w=p.w)
                st = (a.idx_up == r.idx_up) & (b.idx_up == r.idx_up) & (a.idx_lo == r.idx_lo) & (b.idx_lo == r.idx_lo)
                if st.all():
                    fdy = (gbar * (a.g - b.g) / (2 * h)).sum()
                    assert abs(fdy - gy[k]) < 1e-6, (k, fdy, gy[k])


def check_k_neighbours(O):
    """k > 1 neighbours (Sec. 5, extra features): weighted sums of the k best bounds.

    Unmasked: the k smallest of y + M cdist and the k largest of y - M cdist, taken with a
    stable sort (equal values in index order); M = 0: the k smallest / largest y."""
    for seed, (N, d, nq, k) in enumerate([(40, 2, 17, 3), (120, 4, 30, 5), (64, 1, 12, 8)]):
        for norm in (1, 2, 3):
            p = W.random_problem(70 + seed, N, d, nq, norm=norm, weighted=True, dtype=np.float64)
            wk = np.random.default_rng(seed).random(k)
            wk /= wk.sum()
            r = O.evaluate_k(p.X, p.y, p.Q, p.M, k, wk, norm, w=p.w)
            D = cdist(_scaled(p.Q, p.w), _scaled(p.X, p.w), METRIC[norm])
            up = p.y[None, :] + p.M * D
            dn = p.y[None, :] - p.M * D
            ou = np.argsort(up, axis=1, kind="stable")[:, :k]
            od = np.argsort(-dn, axis=1, kind="stable")[:, :k]
            np.testing.assert_allclose(r.hi, (np.take_along_axis(up, ou, 1) * wk).sum(1), atol=1e-12)
            np.testing.assert_allclose(r.lo, (np.take_along_axis(dn, od, 1) * wk).sum(1), atol=1e-12)
            np.testing.assert_allclose(r.g, 0.5 * (r.hi + r.lo), atol=1e-15)
            su = np.sort(up, 1)
            clear = np.all(np.diff(su[:, :k + 1], axis=1) > 1e-9, axis=1)
            assert np.all(r.idx_up[clear] == ou[clear])
            # M = 0: the k smallest (largest) y in index order among equal values
            r0 = O.evaluate_k(p.X, p.y, p.Q[:3], 0.0, k, wk, norm, w=p.w)
            ys = p.y[np.argsort(p.y, kind="stable")[:k]]
            yl = p.y[np.argsort(-p.y, kind="stable")[:k]]
            np.testing.assert_allclose(r0.hi, (ys * wk).sum(), atol=1e-12)
            np.testing.assert_allclose(r0.lo, (yl * wk).sum(), atol=1e-12)
    # consistency with k = 1, also for masked problems and for trailing zero weights
    for norm in (1, 2, 3):
        p = W.random_problem(80, 90, 3, 25, norm=norm, masked=True, decreasing=True, dtype=np.float64)
        r1 = O.evaluate(p.X, p.y, p.Q, p.M, norm, mon=p.mon)
        for k, wk in ((1, [1.0]), (4, [1.0, 0.0, 0.0, 0.0])):
            rk = O.evaluate_k(p.X, p.y, p.Q, p.M, k, wk, norm, mon=p.mon)
            np.testing.assert_allclose(rk.hi, r1.hi, atol=1e-15)
            np.testing.assert_allclose(rk.lo, r1.lo, atol=1e-15)
            assert np.all(rk.idx_up[:, 0] == r1.idx_up) and np.all(rk.idx_lo[:, 0] == r1.idx_lo)



# ------------------------------------------------- local Lipschitz constants (Sec. 4.3)

def check_splitmix64(O):
    """The knot sampler's generator reproduces SplitMix64's published test vector."""
    G = json.load(open(GOLDEN_SPLITMIX))
    assert [O.splitmix64(G["seed"], c) for c in range(len(G["outputs"]))] == [int(v) for v in G["outputs"]]


def _local_problems():
    out = []
    for norm in (1, 2, 3):
        for weighted in (False, True):
            p = W.random_problem(90 + norm, 70, 3, 40, norm=norm, weighted=weighted, dtype=np.float64)
            out.append(p)
    out.append(W.toy_d3(dtype=np.float64, n_data=120, n_query=60))
    return out


def check_local_hand_example(O):
    """Sec. 4.3 worked by hand on 1-D data with explicit knots (tests/golden)."""
    G = json.load(open(GOLDEN_LOCAL))
    X = np.array(G["X"])[:, None]
    Q = np.array(G["Q"])[:, None]
    for norm in (1, 2, 3):
        d1, F, Mtab = O.local_table(X, G["y"], G["knots"], norm)
        np.testing.assert_allclose(d1, G["d1"], rtol=1e-15)
        np.testing.assert_allclose(F, G["F"], rtol=1e-15)
        np.testing.assert_allclose(Mtab, G["Mtab"], rtol=1e-15)
        r = O.evaluate_local(X, G["y"], Q, G["knots"], (d1, F, Mtab), norm)
        np.testing.assert_allclose(r.hi, G["hi"], atol=1e-15)
        np.testing.assert_allclose(r.lo, G["lo"], atol=1e-15)
        assert list(r.idx_up) == G["idx_up"] and list(r.idx_lo) == G["idx_lo"]


def check_local_knots(O):
    """Knots = inverted-CDF quantiles (numpy) of the positive distances (scipy) of the pairs
    SplitMix64 draws."""
    for p in _local_problems():
        N = p.X.shape[0]
        for m, S, seed in ((8, 300, 5), (16, 1000, 123456789), (5, 7, 2**63 + 11)):
            T, pairs, dist = O.local_knots(p.X, m, S, seed, p.norm, w=p.w)
            want = np.array([[O.splitmix64(seed, 2 * s) % N, O.splitmix64(seed, 2 * s + 1) % N] for s in range(S)])
            assert np.array_equal(pairs, want)
            Z = _scaled(p.X, p.w)
            ref = np.array([cdist(Z[a][None], Z[b][None], METRIC[p.norm])[0, 0] for a, b in pairs])
            np.testing.assert_allclose(dist, ref, rtol=1e-13, atol=1e-15)
            D = dist[dist > 0]
            q = np.quantile(D, np.arange(1, m + 1) / m, method="inverted_cdf")
            assert np.array_equal(T, np.unique(q))
            assert np.all(np.diff(T) > 0)
    # no sample, or only repeated points: no knots
    p = _local_problems()[0]
    assert O.local_knots(p.X, 8, 0, 1)[0].size == 0
    assert O.local_knots(np.zeros((5, 2)), 8, 50, 1)[0].size == 0


def _brute_table(Z, y, T, metric):
    """d1, F, Mtab from scipy distances: masks, not loops."""
    D = cdist(Z, Z, metric)
    R = np.abs(y[:, None] - y[None, :]) / np.where(D > 0, D, 1.0)
    pos = D > 0
    d1 = np.where(pos, D, np.inf).min(1)
    near = pos & (D <= d1[:, None] * (1 + 1e-12))
    F = np.where(near, R, 0.0).max(1)
    cols = [np.maximum(F, np.where(pos & (D <= t), R, 0.0).max(1)) for t in list(T) + [np.inf]]
    return d1, F, np.stack(cols, 1)


def check_local_table(O):
    """d1, F, Mtab (Sec. 4.3) against scipy distances; M_k non-decreasing; the last segment
    is the row maximum and its maximum over k is M_est (Sec. 5)."""
    rng = np.random.default_rng(7)
    for p in _local_problems():
        Z = _scaled(p.X, p.w)
        D = cdist(Z, Z, METRIC[p.norm])
        # knots away from every distance, so a 1-ulp difference between scipy and the
        # oracle cannot move a pair across a knot
        T = np.sort(rng.uniform(D[D > 0].min(), D.max(), 9))
        d1, F, Mtab = O.local_table(p.X, p.y, T, p.norm, w=p.w)
        bd1, bF, bM = _brute_table(Z, p.y, T, METRIC[p.norm])
        np.testing.assert_allclose(d1, bd1, rtol=1e-12)
        np.testing.assert_allclose(F, bF, rtol=1e-12)
        np.testing.assert_allclose(Mtab, bM, rtol=1e-12)
        # sampled knots: structural facts only
        T, _, _ = O.local_knots(p.X, 12, 400, 99, p.norm, w=p.w)
        d1, F, Mtab = O.local_table(p.X, p.y, T, p.norm, w=p.w)
        assert np.all(np.diff(Mtab, axis=1) >= 0) and np.all(Mtab[:, 0] >= F)
        R = np.abs(p.y[:, None] - p.y[None, :]) / np.where(D > 0, D, np.inf)
        np.testing.assert_allclose(Mtab[:, -1], R.max(1), rtol=1e-12)
        M_est = O.estimate_M(p.X, p.y, p.norm, w=p.w)[0]
        assert abs(Mtab[:, -1].max() - M_est) <= 1e-12 * M_est
        np.testing.assert_allclose(d1, np.where(D > 0, D, np.inf).min(1), rtol=1e-12)
        rows = np.array([5, 0, len(p.y) - 1, 5])
        sub = O.local_table_rows(p.X, p.y, T, rows, p.norm, w=p.w)
        for a, b in zip(sub, (d1, F, Mtab)):
            assert np.array_equal(a, b[rows])
    # a single datum, or only repeated points: no neighbour, constant 0
    d1, F, Mtab = O.local_table(np.zeros((3, 2)), np.array([1.0, 1.0, 1.0]), [0.5])
    assert np.all(np.isinf(d1)) and np.all(F == 0) and np.all(Mtab == 0)


def check_local_eval(O):
    """Local evaluation (Sec. 4.3): interpolates the data; bounds no wider than the global ones
    with M_est; searchsorted form of M_k(t) (the paper's primitive) on scipy distances; with
    every ratio equal (1-D linear data) it is the global evaluation with that M."""
    for p in _local_problems():
        T, _, _ = O.local_knots(p.X, 10, 500, 3, p.norm, w=p.w)
        tab = O.local_table(p.X, p.y, T, p.norm, w=p.w)
        r = O.evaluate_local(p.X, p.y, p.X, T, tab, p.norm, w=p.w)
        np.testing.assert_allclose(r.hi, p.y, atol=1e-12)
        np.testing.assert_allclose(r.lo, p.y, atol=1e-12)
        M_est = O.estimate_M(p.X, p.y, p.norm, w=p.w)[0]
        rl = O.evaluate_local(p.X, p.y, p.Q, T, tab, p.norm, w=p.w)
        rg = O.evaluate(p.X, p.y, p.Q, M_est, p.norm, w=p.w)
        assert np.all(rl.hi <= rg.hi + 1e-12) and np.all(rl.lo >= rg.lo - 1e-12)
        D = cdist(_scaled(p.Q, p.w), _scaled(p.X, p.w), METRIC[p.norm])
        d1, F, Mtab = tab
        seg = np.searchsorted(T, D, side="left")
        Mq = np.where(D <= d1[None, :], F[None, :], Mtab[np.arange(len(d1))[None, :], seg])
        np.testing.assert_allclose(rl.hi, (p.y[None, :] + Mq * D).min(1), atol=1e-12)
        np.testing.assert_allclose(rl.lo, (p.y[None, :] - Mq * D).max(1), atol=1e-12)
        np.testing.assert_allclose(rl.g, 0.5 * (rl.hi + rl.lo), atol=1e-15)
        assert not rl.amb_up.any() and not rl.amb_lo.any()        # eta = 0: no flags
    rng = np.random.default_rng(3)
    X = rng.uniform(-1, 1, (40, 1))
    y = -2.5 * X[:, 0]
    Q = rng.uniform(-1.5, 1.5, (30, 1))
    T, _, _ = O.local_knots(X, 6, 200, 8)
    tab = O.local_table(X, y, T)
    np.testing.assert_allclose(tab[2], 2.5, rtol=1e-13)
    for norm in (1, 2, 3):
        rl = O.evaluate_local(X, y, Q, T, tab, norm)
        rg = O.evaluate(X, y, Q, 2.5, norm)
        np.testing.assert_allclose(rl.hi, rg.hi, atol=1e-12)
        np.testing.assert_allclose(rl.lo, rg.lo, atol=1e-12)



def _local_M_searchsorted(T, tab, D):
    """M_k(t) for the distance matrix D [q, k] by the paper's primitive (Sec. 5,
    torch.searchsorted): F_k on [0, d1_k], else Mtab_k[#{i : T_i < t}]."""
    d1, F, Mtab = tab
    seg = np.searchsorted(np.asarray(T), D, side="left")
    return np.where(D <= d1[None, :], F[None, :], Mtab[np.arange(len(d1))[None, :], seg])


def check_local_terms(O):
    """The value of a chosen datum with its constant at a shifted distance (the GPU tests'
    yardstick): y_k +- M_k(t + shift) t on scipy distances, for both sides, shifts of 0 and
    +-eta, and indices outside the data (NaN)."""
    rng = np.random.default_rng(17)
    for p in _local_problems()[:4] + _local_problems()[-1:]:
        T, _, _ = O.local_knots(p.X, 9, 600, 5, p.norm, w=p.w)
        tab = O.local_table(p.X, p.y, T, p.norm, w=p.w)
        D = cdist(_scaled(p.Q, p.w), _scaled(p.X, p.w), METRIC[p.norm])
        eta = 0.05 * float(np.median(D))
        N = len(p.y)
        idx = rng.integers(-1, N + 1, len(p.Q))
        ok = (idx >= 0) & (idx < N)
        rows = np.arange(len(p.Q))
        for shift in (0.0, -eta, eta):
            Ms = _local_M_searchsorted(T, tab, D + shift)
            for side in (+1, -1):
                want = np.where(ok, (p.y[None, :] + side * Ms * D)[rows, np.clip(idx, 0, N - 1)], np.nan)
                got = O.local_terms(p.X, p.y, p.Q, T, tab, idx, side, p.norm, w=p.w, shift=shift)
                assert np.array_equal(np.isnan(got), ~ok)
                np.testing.assert_allclose(got[ok], want[ok], rtol=1e-12, atol=1e-13)
        # at the evaluation's own indices the terms are its envelopes
        r = O.evaluate_local(p.X, p.y, p.Q, T, tab, p.norm, w=p.w)
        assert np.array_equal(O.local_terms(p.X, p.y, p.Q, T, tab, r.idx_up, +1, p.norm, w=p.w), r.hi)
        assert np.array_equal(O.local_terms(p.X, p.y, p.Q, T, tab, r.idx_lo, -1, p.norm, w=p.w), r.lo)


def check_local_eval_flags(O):
    """The ambiguity flags of the local evaluation (eta > 0) against brute force: a query is
    flagged exactly when some datum, given its lowest constant within eta (M_k(t - eta))
    while every other datum takes its highest (M_j(t + eta)) and bound values are off by
    tau / 2 against it, wins the minimum (maximum) although its exact value is more than
    tau from the envelope.  Random perturbations of the distances and values never pick a
    datum beyond tau of the envelope on an unflagged query, and every datum they pick
    passes the possible-winner test against hi_plus / lo_minus.  Flags grow with eta."""
    rng = np.random.default_rng(23)
    for seed, (N, d, norm) in enumerate([(45, 2, 2), (60, 3, 1), (52, 2, 3), (70, 1, 2)]):
        p = W.random_problem(700 + seed, N, d, 48, norm=norm, dtype=np.float64)
        T, _, _ = O.local_knots(p.X, 8, 800, 3 + seed, norm)
        tab = O.local_table(p.X, p.y, T, norm)
        D = cdist(p.Q, p.X, METRIC[norm])
        eta = 0.04 * float(D.max())
        scale = float(np.abs(p.y).max() + tab[2].max() * D.max())
        tau = 1e-3 * scale
        r = O.evaluate_local(p.X, p.y, p.Q, T, tab, norm, eta=eta, tau=tau)
        Mt, Ml, Mh = (_local_M_searchsorted(T, tab, D + s) for s in (0.0, -eta, eta))
        y = p.y[None, :]
        exact_u, exact_l = y + Mt * D, y - Mt * D
        bu, bl = exact_u.min(1), exact_l.max(1)
        np.testing.assert_allclose(r.hi, bu, rtol=1e-12, atol=1e-13)
        high_u, high_l = y + Mh * D, y - Mh * D
        np.testing.assert_allclose(r.hi_plus, high_u.min(1), rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(r.lo_minus, high_l.max(1), rtol=1e-12, atol=1e-13)
        flag_u = np.zeros(len(p.Q), bool)
        flag_l = np.zeros(len(p.Q), bool)
        for q in range(len(p.Q)):
            for k in range(N):
                others_u = np.delete(high_u[q], k).min() if N > 1 else np.inf
                others_l = np.delete(high_l[q], k).max() if N > 1 else -np.inf
                if (p.y[k] + Ml[q, k] * D[q, k]) - tau / 2 <= others_u + tau / 2 and exact_u[q, k] > bu[q] + tau:
                    flag_u[q] = True
                if (p.y[k] - Ml[q, k] * D[q, k]) + tau / 2 >= others_l - tau / 2 and exact_l[q, k] < bl[q] - tau:
                    flag_l[q] = True
        assert np.array_equal(r.amb_up, flag_u), (seed, np.nonzero(r.amb_up != flag_u)[0])
        assert np.array_equal(r.amb_lo, flag_l), (seed, np.nonzero(r.amb_lo != flag_l)[0])
        assert 0 < flag_u.sum() < len(p.Q) and 0 < flag_l.sum() < len(p.Q), (seed, flag_u.sum(), flag_l.sum())
        rows = np.arange(len(p.Q))
        for _ in range(300):
            Dp = np.clip(D + rng.uniform(-eta, eta, D.shape), 0.0, None)
            Mp = _local_M_searchsorted(T, tab, Dp)
            vu = y + Mp * D + rng.uniform(-tau / 2, tau / 2, D.shape)
            vl = y - Mp * D + rng.uniform(-tau / 2, tau / 2, D.shape)
            ku, kl = vu.argmin(1), vl.argmax(1)
            assert np.all(~(exact_u[rows, ku] > bu + tau) | r.amb_up)
            assert np.all(~(exact_l[rows, kl] < bl - tau) | r.amb_lo)
            assert np.all(p.y[ku] + Ml[rows, ku] * D[rows, ku] <= r.hi_plus + tau)
            assert np.all(p.y[kl] - Ml[rows, kl] * D[rows, kl] >= r.lo_minus - tau)
        half = O.evaluate_local(p.X, p.y, p.Q, T, tab, norm, eta=eta / 2, tau=tau)
        assert np.all(r.amb_up | ~half.amb_up) and np.all(r.amb_lo | ~half.amb_lo)


def _one_sided(A, B, mon, w, norm, side):
    """dist_up (side +1) or dist_lo (side -1) of Eq. (distmon) between every row of A and
    every row of B, with numpy: differences mirrored where decreasing and weighted, positive
    (side +1) or negative (side -1) parts on the constrained coordinates, |.| elsewhere."""
    sg = np.where(np.asarray(mon) < 0, -1.0, 1.0) * (1.0 if w is None else np.asarray(w))
    T = (A[:, None, :] - B[None, :, :]) * sg
    con = np.asarray(mon) != 0
    V = np.where(con, np.maximum(side * T, 0.0), np.abs(T))
    if norm == 1:
        return V.sum(2)
    if norm == 2:
        return np.sqrt((V * V).sum(2))
    return V.max(2)


def check_local_monotone(O):
    """Local constants with monotone coordinates (Sec. 5: values_local follows values()'s
    monotonicity convention).  Reading: datum k's table takes, from every other datum j, the
    event (dist_up(x^j, x^k), (y^j - y^k)_+ / dist) that its upper bound at x^j needs and the
    event (dist_lo(x^j, x^k), (y^k - y^j)_+ / dist) that its lower bound needs; the bounds use
    M_k at the one-sided distance of their side.  Pins: the table against numpy events;
    interpolation of monotone data; the envelopes non-decreasing along constrained
    coordinates (non-increasing along decreasing ones); 1-D linear increasing data give the
    global monotone evaluation; an all-zero mask gives the symmetric results bit for bit."""
    rng = np.random.default_rng(31)
    for seed, (N, d, norm, weighted) in enumerate([(60, 3, 2, False), (75, 2, 1, True), (50, 4, 3, True),
                                                   (40, 1, 2, False)]):
        p = W.random_problem(740 + seed, N, d, 40, norm=norm, masked=True, weighted=weighted, decreasing=True,
                             dtype=np.float64)
        mon = p.mon if np.any(p.mon != 0) else np.ones(d, np.int8)
        T, _, dist = O.local_knots(p.X, 8, 600, 5 + seed, norm, w=p.w, mon=mon)
        # the knots sample the upper-side distances of the drawn pairs
        _, pairs, _ = O.local_knots(p.X, 1, 600, 5 + seed, norm, w=p.w)
        want = np.array([_one_sided(p.X[a][None], p.X[b][None], mon, p.w, norm, +1)[0, 0] for a, b in pairs])
        np.testing.assert_allclose(dist, want, rtol=1e-13, atol=1e-15)
        # the table against numpy events, with knots away from every event distance
        U = _one_sided(p.X, p.X, mon, p.w, norm, +1)        # U[j, k] = dist_up(x^j, x^k)
        L = _one_sided(p.X, p.X, mon, p.w, norm, -1)
        y = p.y
        D = np.concatenate([U.T, L.T], 1)                   # row k: the events of datum k
        dy = np.concatenate([np.maximum(y[None, :] - y[:, None], 0.0), np.maximum(y[:, None] - y[None, :], 0.0)], 1)
        pos = D > 0
        R = np.where(pos, dy / np.where(pos, D, 1.0), 0.0)
        Tf = np.sort(rng.uniform(D[pos].min(), D.max(), 7))
        d1 = np.where(pos, D, np.inf).min(1)
        near = pos & (D <= d1[:, None] * (1 + 1e-12))
        F = np.where(near, R, 0.0).max(1)
        cols = [np.maximum(F, np.where(pos & (D <= t), R, 0.0).max(1)) for t in list(Tf) + [np.inf]]
        od1, oF, oM = O.local_table(p.X, p.y, Tf, norm, w=p.w, mon=mon)
        np.testing.assert_allclose(od1, d1, rtol=1e-12)
        np.testing.assert_allclose(oF, F, rtol=1e-12, atol=1e-300)
        np.testing.assert_allclose(oM, np.stack(cols, 1), rtol=1e-12, atol=1e-300)
        tab = O.local_table(p.X, p.y, T, norm, w=p.w, mon=mon)
        # evaluation by the searchsorted form on the one-sided distances
        Uq = _one_sided(p.Q, p.X, mon, p.w, norm, +1)
        Lq = _one_sided(p.Q, p.X, mon, p.w, norm, -1)
        r = O.evaluate_local(p.X, p.y, p.Q, T, tab, norm, w=p.w, mon=mon)
        np.testing.assert_allclose(r.hi, (y[None, :] + _local_M_searchsorted(T, tab, Uq) * Uq).min(1), atol=1e-12)
        np.testing.assert_allclose(r.lo, (y[None, :] - _local_M_searchsorted(T, tab, Lq) * Lq).max(1), atol=1e-12)
        # interpolation of monotone data
        rd = O.evaluate_local(p.X, p.y, p.X, T, tab, norm, w=p.w, mon=mon)
        np.testing.assert_allclose(rd.hi, p.y, atol=1e-12)
        np.testing.assert_allclose(rd.lo, p.y, atol=1e-12)
        # monotone along the constrained coordinates
        for i in np.nonzero(mon)[0]:
            Qs = p.Q.copy()
            Qs[:, i] += float(mon[i]) * rng.uniform(0.0, 0.3, len(Qs))
            rs = O.evaluate_local(p.X, p.y, Qs, T, tab, norm, w=p.w, mon=mon)
            assert np.all(rs.hi >= r.hi - 1e-12) and np.all(rs.lo >= r.lo - 1e-12), (seed, i)
        # local terms take the side's distance
        ti = rng.integers(0, N, len(p.Q))
        np.testing.assert_allclose(O.local_terms(p.X, p.y, p.Q, T, tab, ti, +1, norm, w=p.w, mon=mon),
                                   y[ti] + _local_M_searchsorted(T, tab, Uq)[np.arange(len(ti)), ti]
                                   * Uq[np.arange(len(ti)), ti], atol=1e-12)
        np.testing.assert_allclose(O.local_terms(p.X, p.y, p.Q, T, tab, ti, -1, norm, w=p.w, mon=mon),
                                   y[ti] - _local_M_searchsorted(T, tab, Lq)[np.arange(len(ti)), ti]
                                   * Lq[np.arange(len(ti)), ti], atol=1e-12)
        # an all-zero mask is the symmetric method
        z = np.zeros(d, np.int8)
        assert np.array_equal(O.local_knots(p.X, 8, 600, 5, norm, w=p.w, mon=z)[0], O.local_knots(p.X, 8, 600, 5, norm, w=p.w)[0])
        for a, b in zip(O.local_table(p.X, p.y, T, norm, w=p.w, mon=z), O.local_table(p.X, p.y, T, norm, w=p.w)):
            assert np.array_equal(a, b)
    # 1-D linear increasing data: every event ratio is the slope, so the local evaluation is
    # the global monotone one with that M (Sec. 4.1)
    X = rng.uniform(-1, 1, (35, 1))
    y = 1.7 * X[:, 0]
    Q = rng.uniform(-1.5, 1.5, (25, 1))
    one = np.ones(1, np.int8)
    T, _, _ = O.local_knots(X, 6, 300, 2, mon=one)
    tab = O.local_table(X, y, T, mon=one)
    # (ratios of differences of nearby points carry a few hundred ulps)
    np.testing.assert_allclose(tab[2], 1.7, rtol=1e-10)
    for norm in (1, 2, 3):
        rl = O.evaluate_local(X, y, Q, T, tab, norm, mon=one)
        rg = O.evaluate(X, y, Q, 1.7, norm, mon=one)
        np.testing.assert_allclose(rl.hi, rg.hi, atol=1e-10)
        np.testing.assert_allclose(rl.lo, rg.lo, atol=1e-10)


def check_local_k_neighbours(O):
    """k > 1 neighbours with the local constants: the k smallest / largest of the local bound
    values built from scipy distances and the searchsorted form of M_k (stable sort); k = 1
    equals the local evaluation; 1-D linear data equal the global k-neighbour evaluation."""
    for p in _local_problems()[:4]:
        T, _, _ = O.local_knots(p.X, 8, 300, 4, p.norm, w=p.w)
        tab = O.local_table(p.X, p.y, T, p.norm, w=p.w)
        d1, F, Mtab = tab
        D = cdist(_scaled(p.Q, p.w), _scaled(p.X, p.w), METRIC[p.norm])
        seg = np.searchsorted(T, D, side="left")
        Mq = np.where(D <= d1[None, :], F[None, :], Mtab[np.arange(len(d1))[None, :], seg])
        up, dn = p.y[None, :] + Mq * D, p.y[None, :] - Mq * D
        for k in (1, 3, 5):
            wk = np.linspace(1.0, 0.2, k)
            wk /= wk.sum()
            r = O.evaluate_local_k(p.X, p.y, p.Q, T, tab, k, wk, p.norm, w=p.w)
            ou = np.argsort(up, axis=1, kind="stable")[:, :k]
            od = np.argsort(-dn, axis=1, kind="stable")[:, :k]
            np.testing.assert_allclose(r.hi, (np.take_along_axis(up, ou, 1) * wk).sum(1), atol=1e-12)
            np.testing.assert_allclose(r.lo, (np.take_along_axis(dn, od, 1) * wk).sum(1), atol=1e-12)
            if k == 1:
                r1 = O.evaluate_local(p.X, p.y, p.Q, T, tab, p.norm, w=p.w)
                assert np.array_equal(r.hi, r1.hi) and np.array_equal(r.idx_up[:, 0], r1.idx_up)
    rng = np.random.default_rng(5)
    X = rng.uniform(-1, 1, (30, 1))
    y = 1.5 * X[:, 0]
    Q = rng.uniform(-1.5, 1.5, (20, 1))
    T, _, _ = O.local_knots(X, 5, 100, 2)
    tab = O.local_table(X, y, T)
    wk = np.array([0.5, 0.3, 0.2])
    rl = O.evaluate_local_k(X, y, Q, T, tab, 3, wk)
    rg = O.evaluate_k(X, y, Q, 1.5, 3, wk)
    np.testing.assert_allclose(rl.hi, rg.hi, atol=1e-12)
    np.testing.assert_allclose(rl.lo, rg.lo, atol=1e-12)


# --------------------------------------------------------- penalty smoothing (Sec. 4.4)

def _two_point_eps(a, p):
    """Minimiser of Eq. (optim) for two data with one violated constraint of size a > 0:
    by symmetry eps = (-t, t) and Phi = 2 t^2 / p + 2 (a - 2t)^2, so t = 2 a p / (1 + 4 p)."""
    return 2.0 * a * p / (1.0 + 4.0 * p)


def check_smoothing(O):
    """Eq. (optim): the two-point closed form (plain and monotone), gradient against central
    differences, the two penalty sums equal (Eq. (const2) is Eq. (const1) with i and k
    swapped), consistent data untouched, and the returned point a minimiser."""
    for p in (0.5, 10.0, 1e4):
        for M, x2, y1, y2 in ((1.0, 1.0, 3.0, 0.0), (2.0, 0.5, -1.0, 4.0), (0.0, 2.0, 1.0, 0.25)):
            X = np.array([[0.0], [x2]])
            y = np.array([y1, y2])
            a = abs(y1 - y2) - M * x2
            e, f, _ = O.smooth(X, y, M, p, 1, max_iter=200, gtol=1e-13)
            t = _two_point_eps(a, p)
            sgn = 1.0 if y1 > y2 else -1.0
            np.testing.assert_allclose(e, [-sgn * t, sgn * t], rtol=1e-9, atol=1e-12)
            np.testing.assert_allclose(f, 2 * t * t / p + 2 * (a - 2 * t) ** 2, rtol=1e-9, atol=1e-15)
        # increasing in x1: x^1 < x^2 with y^1 > y^2 violates with distance 0
        X = np.array([[0.0, 0.3], [0.4, 0.3]])
        e, _, _ = O.smooth(X, np.array([1.0, 0.2]), 5.0, p, 2, mon=np.array([1, 0], np.int8), gtol=1e-13)
        t = _two_point_eps(0.8, p)
        np.testing.assert_allclose(e, [-t, t], rtol=1e-9, atol=1e-12)
    rng = np.random.default_rng(11)
    for norm in (1, 2, 3):
        for mon, w in ((None, None), (np.array([1, -1, 0], np.int8), np.array([0.5, 2.0, 1.0]))):
            X = rng.random((25, 3))
            y = np.sin(4 * X[:, 0]) + 0.5 * rng.standard_normal(25)
            eps = 0.1 * rng.standard_normal(25)
            M, p = 1.5, 20.0
            f, g, s1, s2 = O.smooth_objective(X, y, eps, M, p, norm, mon=mon, w=w)
            assert s1 > 0 and abs(s1 - s2) <= 1e-12 * s1
            assert abs(f - (eps @ eps / p + s1 + s2)) <= 1e-12 * f
            h = 1e-6
            for j in range(0, 25, 3):
                ep, em = eps.copy(), eps.copy()
                ep[j] += h
                em[j] -= h
                fd = (O.smooth_objective(X, y, ep, M, p, norm, mon=mon, w=w)[0] -
                      O.smooth_objective(X, y, em, M, p, norm, mon=mon, w=w)[0]) / (2 * h)
                assert abs(fd - g[j]) <= 1e-5 * (1 + abs(g[j])), (norm, j, fd, g[j])
            rows = np.array([0, 7, 24, 7])
            assert np.allclose(O.smooth_grad_rows(X, y, eps, rows, M, p, norm, mon=mon, w=w), g[rows],
                               rtol=1e-12, atol=1e-12)
            e, fmin, it = O.smooth(X, y, M, p, norm, mon=mon, w=w, max_iter=3000, gtol=1e-8)
            fe, ge, _, _ = O.smooth_objective(X, y, e, M, p, norm, mon=mon, w=w)
            assert np.abs(ge).max() <= 1e-8 and abs(fe - fmin) <= 1e-14 * max(1.0, fe)
            for _ in range(5):                        # convex: no nearby point is lower
                dlt = 1e-3 * rng.standard_normal(25)
                assert O.smooth_objective(X, y, e + dlt, M, p, norm, mon=mon, w=w)[0] >= fe
    # data consistent with M: nothing to change
    pr = W.random_problem(301, 40, 2, 1, norm=2)
    e, f, it = O.smooth(pr.X, pr.y, pr.M, 100.0, 2)
    assert it == 0 and f == 0.0 and np.all(e == 0.0)
    # a large penalty weight leaves (almost) consistent data
    X = rng.random((30, 2))
    y = X[:, 0] + 0.3 * rng.standard_normal(30)
    e, _, _ = O.smooth(X, y, 1.0, 1e6, 2, max_iter=5000, gtol=1e-8)
    M_after = O.estimate_M(X, y + e, 2)[0]
    assert M_after <= 1.0 + 1e-3, M_after


ALL_CHECKS = [check_hand_examples, check_closed_form_1d, check_unmasked_cdist, check_interpolation,
              check_enclosure, check_lipschitz_monotone, check_width_bound, check_special_cases,
              check_estimate_M, check_gradient_fd, check_k_neighbours, check_splitmix64,
              check_local_hand_example, check_local_knots, check_local_table, check_local_eval,
              check_local_terms, check_local_eval_flags, check_local_monotone, check_local_k_neighbours,
              check_smoothing]
