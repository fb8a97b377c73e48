"""Local Lipschitz constants (Sec. 4.3) on the GPU against the FP64 oracle.

The knots and the table decide integer outcomes (segment, nearest datum) with exact FP64
arithmetic on both sides, so they must agree bit for bit.  The evaluation selects its data
in FP32: a query passes when the GPU's bounds are the exact values of the data it returned
and, unless the oracle flags the query as decided within FP32 rounding of a knot, those
values are within the FP32 tolerance of the exact envelopes."""
import numpy as np
import pytest

from scipy.spatial.distance import cdist

import oracle as O
from paper_2606_04670_b300 import workloads as W
from parity import FP32_TOL, diam

METRIC = {1: "cityblock", 2: "euclidean", 3: "chebyshev"}

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _model(X, y, norm, w=None, mon=None, precision="fp32"):
    from paper_2606_04670_b300.lipfit import LipFit
    return LipFit(torch.as_tensor(X).cuda(), torch.as_tensor(y).cuda(), 1.0, norm=norm, w=w, mon=mon,
                  precision=precision)


def _f64(a):
    return np.asarray(a, np.float64)


def _table(m):
    return tuple(t.cpu().numpy() for t in m.local_table())


def _cases():
    out = []
    for norm in (1, 2, 3):
        for seed, (N, d, weighted) in enumerate([(37, 2, False), (700, 3, True), (2049, 5, False), (1500, 8, True)]):
            out.append(W.random_problem(200 + 10 * norm + seed, N, d, 300, norm=norm, weighted=weighted))
    out.append(W.random_problem(230, 900, 16, 200, norm=2, weighted=True))
    out.append(W.random_problem(231, 600, 1, 300, norm=1))
    out.append(W.local_d4(n_data=3000, n_query=2000))
    return out


CASES = _cases()


def _one_sided(A, B, mon, w, norm, side):
    """dist_up (side +1) / dist_lo (side -1) of Eq. (distmon) between the rows of A and B."""
    sg = np.where(np.asarray(mon) < 0, -1.0, 1.0) * (1.0 if w is None else np.asarray(w))
    V = (A[:, None, :] - B[None, :, :]) * sg
    V = np.where(np.asarray(mon) != 0, np.maximum(side * V, 0.0), np.abs(V))
    return V.sum(2) if norm == 1 else (np.sqrt((V * V).sum(2)) if norm == 2 else V.max(2))


def _check_eval(p, X, y, Q, T, tab, out, label):
    """Every query, both bounds (the upper shown; the lower is its mirror):
    * the returned bound is the exact FP64 value of the returned datum, rounded once;
    * it is never better than the exact envelope H_up;
    * the returned datum is one an FP32 evaluation can pick: its value with the lowest
      constant its distance error allows, y_k + M_k(t - eta) t, is at most tau above
      hi_plus, the envelope with every constant at its highest, M_j(t + eta) (so a far-off
      datum cannot pass, flagged or not);
    * where the oracle finds that no datum such an evaluation could pick has an exact value
      more than tau above H_up (the query is not flagged), the bound is within tau of H_up;
    * a query is flagged only where some datum's constant can change within eta of its
      distance (M_k(t - eta) < M_k(t + eta)): the flags are a subset of those queries."""
    hi, lo, g = (_f64(out[k].cpu().numpy()) for k in ("hi", "lo", "g"))
    iu, il = (out[k].cpu().numpy().astype(np.int64) for k in ("idx_up", "idx_lo"))
    Z = np.abs(np.concatenate([X, Q]) * (1.0 if p.w is None else np.asarray(p.w)))
    dm = diam(X, Q, p.norm, p.w)
    eta = 2.0 ** -20 * (X.shape[1] + 2) * (Z.max() + dm)
    mmax = float(tab[2].max()) if tab[2].size else 0.0
    scale = float(np.abs(y).max()) + mmax * dm + 1e-30
    tau = max(FP32_TOL * scale, 2.0 * (mmax * eta + 2.0 ** -21 * scale))
    mon = p.mon
    r = O.evaluate_local(X, y, Q, T, tab, p.norm, w=p.w, eta=eta, tau=tau, mon=mon)
    tu = O.local_terms(X, y, Q, T, tab, iu, +1, p.norm, w=p.w, mon=mon)
    tl = O.local_terms(X, y, Q, T, tab, il, -1, p.norm, w=p.w, mon=mon)
    # the returned values are the exact FP64 values of the returned data, rounded once
    assert np.array_equal(hi.astype(np.float32), tu.astype(np.float32)), label
    assert np.array_equal(lo.astype(np.float32), tl.astype(np.float32)), label
    assert np.array_equal(g.astype(np.float32), (0.5 * (tu + tl)).astype(np.float32)), label
    # never better than the exact envelope
    assert np.all(tu >= r.hi - 1e-12 * scale) and np.all(tl <= r.lo + 1e-12 * scale), label
    # a datum an FP32 evaluation can pick (every query)
    tu_low = O.local_terms(X, y, Q, T, tab, iu, +1, p.norm, w=p.w, shift=-eta, mon=mon)
    tl_low = O.local_terms(X, y, Q, T, tab, il, -1, p.norm, w=p.w, shift=-eta, mon=mon)
    assert np.all(tu_low <= r.hi_plus + tau), (label, np.max(tu_low - r.hi_plus), tau)
    assert np.all(tl_low >= r.lo_minus - tau), (label, np.max(r.lo_minus - tl_low), tau)
    # unflagged queries: within tau of the exact envelope
    su, sl = ~r.amb_up, ~r.amb_lo
    assert np.all(np.abs(tu - r.hi)[su] <= tau), (label, np.abs(tu - r.hi)[su].max(), tau)
    assert np.all(np.abs(tl - r.lo)[sl] <= tau), (label, np.abs(tl - r.lo)[sl].max(), tau)
    # flags only where a constant can change within eta
    if len(Q) * len(X) <= 8_000_000:
        d1, F, Mtab = tab

        def mk(Dm):
            seg = np.searchsorted(np.asarray(T), Dm, side="left")
            return np.where(Dm <= d1[None, :], F[None, :], Mtab[np.arange(len(d1))[None, :], seg])
        if mon is None or not np.any(mon):
            D = cdist(Q * (1.0 if p.w is None else np.asarray(p.w)), X * (1.0 if p.w is None else np.asarray(p.w)),
                      METRIC[p.norm])
            Ds = (D, D)
        else:
            Ds = (_one_sided(Q, X, mon, p.w, p.norm, +1), _one_sided(Q, X, mon, p.w, p.norm, -1))
        near_u = np.any(mk(Ds[0] - eta) < mk(Ds[0] + eta), axis=1)
        near_l = np.any(mk(Ds[1] - eta) < mk(Ds[1] + eta), axis=1)
        assert np.all(near_u | ~r.amb_up) and np.all(near_l | ~r.amb_lo), label
    return r


@pytest.mark.parametrize("case", range(len(CASES)), ids=lambda i: f"{CASES[i].name}-L{CASES[i].norm}-N{CASES[i].N}")
def test_knots_table_and_eval_match_oracle(case):
    p = CASES[case]
    m = _model(p.X, p.y, p.norm, w=p.w)
    X, y, Q = _f64(p.X), _f64(p.y), _f64(p.Q)
    for nknots, S, seed in ((16, 4096, 7), (5, 300, 2**64 - 3)):
        T = m.compute_local_lipschitz(nknots, S, seed)
        To, _, _ = O.local_knots(X, nknots, S, seed, p.norm, w=p.w)
        assert np.array_equal(T, To), (p.name, T, To)
        d1, F, Mtab = _table(m)
        od1, oF, oM = O.local_table(X, y, T, p.norm, w=p.w)
        assert np.array_equal(d1, od1) and np.array_equal(F, oF), p.name
        assert np.array_equal(Mtab, oM), (p.name, np.abs(Mtab - oM).max())
        out = m.eval_local(torch.as_tensor(p.Q).cuda())
        torch.cuda.synchronize()
        _check_eval(p, X, y, Q, T, (d1, F, Mtab), out, p.name)
        # interpolation at the data (Sec. 4.3: the approximation interpolates the data)
        outd = m.eval_local(torch.as_tensor(p.X).cuda())
        _check_eval(p, X, y, X, T, (d1, F, Mtab), outd, p.name + "@data")
        tol = 1e-6 * (np.abs(y).max() + 1)
        assert np.all(np.abs(outd["g"].cpu().numpy() - y) <= tol)
    m.check()
    m.close()


def test_explicit_knots_at_pair_distances():
    """Knots equal to interpoint distances: the <= at a knot decides whole segments."""
    p = W.random_problem(240, 800, 3, 400, norm=2, weighted=True)
    X, y = _f64(p.X), _f64(p.y)
    _, pairs, dist = O.local_knots(X, 1, 64, 99, 2, w=p.w)
    T = np.unique(dist[dist > 0])[::3][:31]
    m = _model(p.X, p.y, 2, w=p.w)
    got = m.compute_local_lipschitz(knots=T)
    assert np.array_equal(got, T)
    d1, F, Mtab = _table(m)
    od1, oF, oM = O.local_table(X, y, T, 2, w=p.w)
    assert np.array_equal(d1, od1) and np.array_equal(F, oF) and np.array_equal(Mtab, oM)
    # data points at knot distances from others: still interpolated
    out = m.eval_local(torch.as_tensor(p.X).cuda())
    _check_eval(p, X, y, X, T, (d1, F, Mtab), out, "knots-at-pairs")
    m.close()


def test_edge_cases():
    from paper_2606_04670_b300.lipfit import LIP_ERR_ARG, LIP_ERR_STATE, LIP_ERR_UNSUPPORTED, LipError
    # a single datum: M_k = 0, the bounds are y
    m = _model(np.array([[0.3, 0.7]], np.float32), np.array([2.5], np.float32), 2)
    assert m.compute_local_lipschitz(8, 100, 1).size == 0
    d1, F, Mtab = _table(m)
    assert np.isinf(d1[0]) and F[0] == 0 and np.all(Mtab == 0)
    Q = torch.tensor([[0.0, 0.0], [5.0, -1.0], [float("nan"), 0.0]], device="cuda")
    out = m.eval_local(Q)
    hi, lo = out["hi"].cpu().numpy(), out["lo"].cpu().numpy()
    assert np.all(hi[:2] == 2.5) and np.all(lo[:2] == 2.5)
    assert np.isnan(hi[2]) and out["idx_up"][2].item() == -1 and out["idx_lo"][2].item() == -1
    # nq = 0 and no knots
    assert m.eval_local(torch.empty((0, 2), device="cuda"))["g"].numel() == 0
    m.close()
    # duplicated points are skipped as neighbours; no sample gives no knots
    from paper_2606_04670_b300.lipfit import LipFit
    X = np.array([[0, 0], [0, 0], [1, 0], [3, 0]], np.float32)
    y = np.array([0, 0, 2, 3], np.float32)
    m = LipFit(torch.as_tensor(X).cuda(), torch.as_tensor(y).cuda(), 1.0, norm="L1", capacity=8)
    assert m.compute_local_lipschitz(4, 0, 1).size == 0
    d1, F, Mtab = _table(m)
    od1, oF, oM = O.local_table(_f64(X), _f64(y), [], 1)
    assert np.array_equal(d1, od1) and np.array_equal(F, oF) and np.array_equal(Mtab, oM)
    # the table is invalidated by new data
    m.add(torch.tensor([[2.0, 2.0]], device="cuda"), torch.tensor([1.0], device="cuda"))
    with pytest.raises(LipError) as e:
        m.eval_local(torch.zeros((1, 2), device="cuda"))
    assert e.value.status == LIP_ERR_STATE
    m.compute_local_lipschitz(4, 64, 3)
    out = m.eval_local(torch.as_tensor(X).cuda())
    assert np.allclose(out["g"].cpu().numpy(), y, atol=1e-6)
    with pytest.raises(LipError) as e:
        m.compute_local_lipschitz(knots=[1.0, 0.5])
    assert e.value.status == LIP_ERR_ARG
    with pytest.raises(LipError) as e:
        m.compute_local_lipschitz(32, 10, 1)
    assert e.value.status == LIP_ERR_ARG
    m.clear()
    with pytest.raises(LipError) as e:
        m.compute_local_lipschitz(4, 10, 1)
    assert e.value.status == LIP_ERR_ARG
    m.close()
    # monotone handles with a table: the one-sided distances (test_monotone_local_constants)
    m = _model(X, y, 2, mon=[1, 0])
    T = m.compute_local_lipschitz(4, 10, 1)
    assert np.array_equal(T, O.local_knots(_f64(X), 4, 10, 1, 2, mon=np.array([1, 0], np.int8))[0])
    m.close()


def test_fp64_handle_local():
    """FP64 data: knots and table bit-exact against the oracle on the double values, the
    evaluation in double outputs by validity and the envelope."""
    p = W.random_problem(280, 1200, 3, 500, norm=2, weighted=True, dtype=np.float64)
    m = _model(p.X, p.y, 2, w=p.w, precision="fp64")
    T = m.compute_local_lipschitz(10, 4000, 3)
    assert np.array_equal(T, O.local_knots(p.X, 10, 4000, 3, 2, w=p.w)[0])
    tab = _table(m)
    for a, b in zip(tab, O.local_table(p.X, p.y, T, 2, w=p.w)):
        assert np.array_equal(a, b)
    out = m.eval_local(torch.as_tensor(p.Q).cuda())
    assert out["g"].dtype == torch.float64
    r = O.evaluate_local(p.X, p.y, p.Q, T, tab, 2, w=p.w, eta=1e-5, tau=1e-5)
    tu = O.local_terms(p.X, p.y, p.Q, T, tab, out["idx_up"].cpu().numpy().astype(np.int64), +1, 2, w=p.w)
    assert np.allclose(out["hi"].cpu().numpy(), tu, rtol=0, atol=1e-12)
    clear = ~r.amb_up
    assert np.all(np.abs(out["hi"].cpu().numpy() - r.hi)[clear] <= 1e-5)
    m.close()


def test_tensor_core_handle_uses_local_path():
    p = W.random_problem(250, 1200, 6, 500, norm=2)
    m = _model(p.X, p.y, 2, precision="tc_tf32")
    X, y, Q = _f64(p.X), _f64(p.y), _f64(p.Q)
    T = m.compute_local_lipschitz(12, 2000, 5)
    tab = _table(m)
    assert np.array_equal(tab[2], O.local_table(X, y, T, 2)[2])
    _check_eval(p, X, y, Q, T, tab, m.eval_local(torch.as_tensor(p.Q).cuda()), "tc-handle")
    m.close()


def test_full_size_local_d4_sampled():
    """The benchmark's workload (N = 100,000, d = 4, 16 knots from 32,768 pairs): the knots
    exactly, 64 table rows against the oracle's rows, and 512 sampled queries of the full
    evaluation by properties that hold at any size: each returned value is the exact value
    of the returned datum (its table row from the oracle), and no datum of a random subset
    of 2,048 (rows from the oracle) has a better value beyond the FP32 tolerance."""
    p = W.local_d4()
    X, y = _f64(p.X), _f64(p.y)
    m = _model(p.X, p.y, 2)
    T = m.compute_local_lipschitz(16, 32768, 0)
    assert np.array_equal(T, O.local_knots(X, 16, 32768, 0, 2)[0])
    d1, F, Mtab = _table(m)
    rng = np.random.default_rng(0)
    rows = rng.choice(p.N, 64, replace=False)
    od1, oF, oM = O.local_table_rows(X, y, T, rows, 2)
    assert np.array_equal(d1[rows], od1) and np.array_equal(F[rows], oF) and np.array_equal(Mtab[rows], oM)
    assert np.all(np.diff(Mtab, axis=1) >= 0)
    out = m.eval_local(torch.as_tensor(p.Q).cuda())
    torch.cuda.synchronize()
    sel = np.sort(rng.choice(p.nq, 512, replace=False))
    Qs = _f64(p.Q[sel])
    hi = _f64(out["hi"].cpu().numpy()[sel])
    lo = _f64(out["lo"].cpu().numpy()[sel])
    iu = out["idx_up"].cpu().numpy()[sel].astype(np.int64)
    il = out["idx_lo"].cpu().numpy()[sel].astype(np.int64)
    sub = np.unique(np.concatenate([iu, il, rng.choice(p.N, 2048, replace=False)]))
    sd1, sF, sM = O.local_table_rows(X, y, T, sub, 2)
    # a table holding the oracle's rows for `sub` only (other rows are never read)
    td1, tF, tM = np.full(p.N, np.nan), np.full(p.N, np.nan), np.full((p.N, T.size + 1), np.nan)
    td1[sub], tF[sub], tM[sub] = sd1, sF, sM
    tab = (td1, tF, tM)
    tu = O.local_terms(X, y, Qs, T, tab, iu, +1, 2)
    tl = O.local_terms(X, y, Qs, T, tab, il, -1, 2)
    assert np.array_equal(hi.astype(np.float32), tu.astype(np.float32))
    assert np.array_equal(lo.astype(np.float32), tl.astype(np.float32))
    scale = float(np.abs(y).max()) + float(sM.max()) * 2.0
    tol = FP32_TOL * scale
    others = rng.choice(sub, 2048, replace=False)
    for k in others:
        kk = np.full(len(sel), k)
        assert np.all(tu <= O.local_terms(X, y, Qs, T, tab, kk, +1, 2) + tol)
        assert np.all(tl >= O.local_terms(X, y, Qs, T, tab, kk, -1, 2) - tol)
    m.check()
    m.close()


def test_two_knots_in_one_bucket_table_segments():
    """Knots 0.5 and 0.50002 share a lookup bucket (width 1/2048 with the last knot at 1).
    Datum 0's pair at distance 0.50003 lies beyond both; its ratio (6) must not bound
    segment 1, which holds only the pair at 0.50001 (ratio 2): Mtab_0 = [F, 2, 6, 6]."""
    X = np.array([[0.0], [0.2], [0.50001], [0.50003]], np.float32)
    y = np.array([0.0, 0.01, 1.0, 3.0], np.float32)
    T = np.array([0.5, 0.50002, 1.0])
    m = _model(X, y, 2)
    assert np.array_equal(m.compute_local_lipschitz(knots=T), T)
    d1, F, Mtab = _table(m)
    od1, oF, oM = O.local_table(_f64(X), _f64(y), T, 2)
    assert np.array_equal(d1, od1) and np.array_equal(F, oF)
    assert np.array_equal(Mtab, oM), (Mtab[0], oM[0])
    assert oM[0, 1] > oF[0] and oM[0, 2] > oM[0, 1]
    m.close()


def test_candidate_list_overflow_rows():
    """150 copies of each of two points after 500 random ones: the copies' rows list every
    duplicate (distance 0 passes the nearest-neighbour test), overflow the candidate list and
    take the second scan; the table is still exact."""
    r = np.random.default_rng(7)
    X = np.concatenate([r.random((500, 3)), np.tile([[0.25, 0.5, 0.75]], (150, 1)),
                        np.tile([[0.6, 0.1, 0.3]], (150, 1))]).astype(np.float32)
    y = (np.sin(3 * X[:, 0]) + X[:, 1] * X[:, 2]).astype(np.float32)
    for norm in (1, 2, 3):
        m = _model(X, y, norm)
        T = m.compute_local_lipschitz(12, 4096, 5)
        over, longest = m.local_stats()
        assert 300 <= over < 800, over
        assert 0 < longest <= 64
        d1, F, Mtab = _table(m)
        od1, oF, oM = O.local_table(_f64(X), _f64(y), T, norm)
        assert np.array_equal(d1, od1) and np.array_equal(F, oF) and np.array_equal(Mtab, oM), norm
        m.close()


def test_close_knots_use_the_search_lookup():
    """Two knots in one lookup bucket switch the evaluation to the binary search over the
    knots; results still match the oracle."""
    p = W.random_problem(260, 1000, 2, 600, norm=1, weighted=True)
    X, y, Q = _f64(p.X), _f64(p.y), _f64(p.Q)
    T = np.array([0.2, 0.5, 0.5000001, 0.9, 1.4])
    m = _model(p.X, p.y, 1, w=p.w)
    assert np.array_equal(m.compute_local_lipschitz(knots=T), T)
    tab = _table(m)
    for a, b in zip(tab, O.local_table(X, y, T, 1, w=p.w)):
        assert np.array_equal(a, b)
    _check_eval(p, X, y, Q, T, tab, m.eval_local(torch.as_tensor(p.Q).cuda()), "search-lookup")
    m.close()



@pytest.mark.parametrize("k", [1, 2, 3, 5, 8])
def test_local_k_neighbours(k):
    """values_local(query, model, k): the weighted sums of the k best local bounds.  Indices
    are compared where the oracle's k-th and (k+1)-th values are clearly apart and no knot
    is within FP32 rounding; the values always, within the FP32 tolerance."""
    p = W.random_problem(270 + k, 1500, 3, 700, norm=(k % 3) + 1, weighted=True)
    X, y, Q = _f64(p.X), _f64(p.y), _f64(p.Q)
    m = _model(p.X, p.y, p.norm, w=p.w)
    T = m.compute_local_lipschitz(12, 3000, 9)
    tab = _table(m)
    wk = np.linspace(1.0, 0.3, k)
    wk /= wk.sum()
    out = m.eval_local_k(torch.as_tensor(p.Q).cuda(), k, wk)
    torch.cuda.synchronize()
    r = O.evaluate_local_k(X, y, Q, T, tab, k, wk, p.norm, w=p.w)
    Z = np.abs(np.concatenate([X, Q]) * np.asarray(p.w))
    eta = 2.0 ** -20 * (X.shape[1] + 2) * (Z.max() + diam(X, Q, p.norm, p.w))
    tol = FP32_TOL * (float(np.abs(y).max()) + float(tab[2].max()) * diam(X, Q, p.norm, p.w))
    amb = O.evaluate_local(X, y, Q, T, tab, p.norm, w=p.w, eta=eta, tau=tol)
    # validity: the outputs are the weighted sums of the exact values of the returned data,
    # which come sorted by value
    for key, idx, side in (("hi", "idx_up", +1), ("lo", "idx_lo", -1)):
        ix = out[idx].cpu().numpy().astype(np.int64)
        vals = np.stack([O.local_terms(X, y, Q, T, tab, ix[:, j], side, p.norm, w=p.w) for j in range(k)], 1)
        assert np.all(side * np.diff(vals, axis=1) >= 0)
        got = out[key].cpu().numpy()
        assert np.array_equal(got, (vals @ wk).astype(np.float32)) or np.allclose(got, vals @ wk, rtol=1e-6, atol=1e-7)
    # the envelope sums within the FP32 tolerance wherever no knot decision is within rounding
    clear = ~(amb.amb_up | amb.amb_lo)
    for key in ("hi", "lo", "g"):
        err = np.abs(out[key].cpu().numpy().astype(np.float64) - r[key])
        assert np.mean(err[clear] <= tol) >= 0.995, (key, err[clear].max(), tol)
    same = np.all(out["idx_up"].cpu().numpy() == r.idx_up, axis=1)
    assert same.mean() > 0.95, same.mean()
    m.close()


MONO_CASES = [W.random_problem(290 + 7 * n + d, N, d, 300, norm=n, masked=True, weighted=(d % 2 == 0),
                               decreasing=(n != 2))
              for n, (N, d) in zip((1, 2, 3, 2, 1), [(900, 3), (1500, 4), (700, 2), (1100, 8), (600, 20)])]


@pytest.mark.parametrize("case", range(len(MONO_CASES)),
                         ids=lambda i: f"L{MONO_CASES[i].norm}-N{MONO_CASES[i].N}-d{MONO_CASES[i].d}")
def test_monotone_local_constants(case):
    """Monotone coordinates (one-sided distances of Eq. (distmon)): knots and table bit for
    bit against the oracle, the evaluation by validity and the envelope (both bounds with
    their own one-sided distance), interpolation at the data, and k > 1 neighbours."""
    p = MONO_CASES[case]
    if not np.any(p.mon):
        p.mon[0] = 1
    m = _model(p.X, p.y, p.norm, w=p.w, mon=p.mon)
    X, y, Q = _f64(p.X), _f64(p.y), _f64(p.Q)
    T = m.compute_local_lipschitz(14, 5000, 11 + case)
    To, _, _ = O.local_knots(X, 14, 5000, 11 + case, p.norm, w=p.w, mon=p.mon)
    assert np.array_equal(T, To), (T, To)
    tab = _table(m)
    for a, b in zip(tab, O.local_table(X, y, T, p.norm, w=p.w, mon=p.mon)):
        assert np.array_equal(a, b), np.abs(a - b).max()
    _check_eval(p, X, y, Q, T, tab, m.eval_local(torch.as_tensor(p.Q).cuda()), f"mono {case}")
    outd = m.eval_local(torch.as_tensor(p.X).cuda())
    _check_eval(p, X, y, X, T, tab, outd, f"mono {case} @data")
    assert np.all(np.abs(outd["g"].cpu().numpy() - y) <= 1e-6 * (np.abs(y).max() + 1))
    k = 3
    wk = np.array([0.5, 0.3, 0.2])
    outk = m.eval_local_k(torch.as_tensor(p.Q).cuda(), k, wk)
    rk = O.evaluate_local_k(X, y, Q, T, tab, k, wk, p.norm, w=p.w, mon=p.mon)
    tol = FP32_TOL * (float(np.abs(y).max()) + float(tab[2].max()) * diam(X, Q, p.norm, p.w))
    for key in ("hi", "lo"):
        err = np.abs(outk[key].cpu().numpy().astype(np.float64) - rk[key])
        assert np.mean(err <= tol) >= 0.99, (key, err.max(), tol)
    m.check()
    m.close()
