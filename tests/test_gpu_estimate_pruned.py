"""lip_estimate_M against the FP64 oracle exactly -- the value bit for bit, then the lowest
i, then the lowest j, exact FP64 ties included -- in both forms: the pruned one (FP32
handles, d <= 8, forced for every norm) and the full all-pairs kernel, each
an FP32 screen followed by the FP64 selection among the pairs within the screen's error
bound of its maximum.  Every norm, weights (and the weighted differences of points one
FP32 unit apart), ragged and tiny N, duplicated points (infinite ratios), constant values
(all ratios 0) and the benchmark's size."""
import numpy as np
import pytest

from paper_2606_04670_b300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _both(X, y, norm, w=None):
    from paper_2606_04670_b300.lipfit import LipFit
    m = LipFit(torch.as_tensor(X).cuda(), torch.as_tensor(y).cuda(), 1.0, norm=norm, w=w)
    m.set_estimate_form("pruned")
    a = m.lipschitz_constant()
    m.set_estimate_form("full")
    b = m.lipschitz_constant()
    m.close()
    return a, b


def _ratio64(X, y, i, j, norm, w=None):
    v = np.abs(X[i].astype(np.float64) - X[j].astype(np.float64))
    if w is not None:
        v = v * w
    dist = {1: v.sum(), 2: np.sqrt((v * v).sum()), 3: v.max()}[norm]
    return abs(float(y[i]) - float(y[j])) / dist


@pytest.mark.parametrize("norm", (1, 2, 3))
@pytest.mark.parametrize("d", (1, 2, 4, 6, 8))
def test_estimate_equals_oracle_both_forms(oracle_mod, norm, d):
    for N in (2, 3, 513, 2_777):
        p = W.random_problem(3000 + 10 * d + norm + N, N, d, 1, norm=norm, weighted=(N % 2 == 1))
        a, b = _both(p.X, p.y, norm, p.w)
        o = oracle_mod.estimate_M(p.X, p.y, norm, w=p.w)
        assert a == b == o, (N, a, b, o)


def test_estimate_near_coincident_weighted(oracle_mod):
    """Points one or two FP32 units apart with weights that are not powers of two: the
    weighted difference is formed from the exact FP32 difference, so the closest pairs'
    ratios survive (a weight rounded into each coordinate first would leave an error as
    large as the difference)."""
    rng = np.random.default_rng(21)
    X = rng.random((4_000, 2)).astype(np.float32)
    y = (rng.random(4_000) * 1e-3).astype(np.float32)
    up = np.float32(2)
    for k, (i, j) in enumerate(((700, 3_100), (12, 2_048), (1_500, 3_999))):
        X[j, 0] = X[i, 0] if k == 1 else np.nextafter(X[i, 0], up)
        X[j, 1] = np.nextafter(np.nextafter(X[i, 1], up), up)
        y[j] = y[i] + np.float32(1e-6 * (k + 1))
    w = np.array([1.7, 0.3])
    for norm in (1, 2, 3):
        a, b = _both(X, y, norm, w)
        o = oracle_mod.estimate_M(X, y, norm, w=w)
        assert a == b == o, (norm, a, b, o)


def test_estimate_degenerate_data(oracle_mod):
    rng = np.random.default_rng(7)
    # duplicated points with different values: an infinite ratio, the lowest pair
    X = rng.random((3_000, 3)).astype(np.float32)
    y = rng.random(3_000).astype(np.float32)
    X[2_500] = X[1_700]
    X[2_900] = X[40]
    a, b = _both(X, y, 2)
    assert a == b == (float("inf"), 40, 2_900), (a, b)
    # duplicates with equal values only: those pairs drop out
    y2 = y.copy()
    y2[2_500], y2[2_900] = y2[1_700], y2[40]
    a, b = _both(X, y2, 1)
    assert a == b == oracle_mod.estimate_M(X, y2, 1) and np.isfinite(a[0])
    # constant values: every ratio is 0, the lowest pair (0, 1)
    a, b = _both(X, np.full(3_000, 0.25, np.float32), 3)
    assert a == b == (0.0, 0, 1), (a, b)
    # constant values and a repeated first point: (0, 1) is left out, (0, 2) is the lowest
    X3 = X.copy()
    X3[1] = X3[0]
    a, b = _both(X3, np.full(3_000, 0.25, np.float32), 2)
    assert a == b == (0.0, 0, 2), (a, b)
    # one point: no pair
    a, b = _both(X[:1], y[:1], 2)
    assert a == b and a[1] == -1


@pytest.mark.parametrize("norm", (1, 2, 3))
def test_estimate_benchmark_size(norm):
    """N = 1e5 (the benchmark's data): both forms agree bit for bit, the result is its
    pair's FP64 ratio, and the pruned screen evaluates part of the (warp, chunk) pairs."""
    from paper_2606_04670_b300.lipfit import LipFit
    p = W.monotone_d4(norm=norm, n_query=16)
    m = LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), 1.0, norm=norm)
    a = m.lipschitz_constant()                       # the default form: pruned
    entered, evaluated, total = m.last_estimate_work()
    nb = (p.N + 511) // 512
    assert 0 < entered <= nb * (nb + 1) // 2 and 0 < evaluated < 0.5 * total, (entered, evaluated, total)
    m.set_estimate_form("full")
    b = m.lipschitz_constant()
    assert m.last_estimate_work() == [-1, -1, -1]
    m.close()
    assert a == b, (a, b)
    assert 0 <= a[1] < a[2] < p.N
    assert abs(_ratio64(p.X, p.y, a[1], a[2], norm) - a[0]) <= 1e-15 * a[0]


def test_estimate_async_on_several_streams(oracle_mod):
    """lip_estimate_M_async on three handles, each on its own stream, all queued before
    the first result is read: each result equals lip_estimate_M's and the oracle's, in
    both forms, and reading a result twice is an error."""
    from paper_2606_04670_b300 import lipfit as L
    from paper_2606_04670_b300.lipfit import LipFit
    probs = [W.random_problem(3100 + k, 40_000 + 1_111 * k, 4, 1, norm=k + 1, weighted=(k == 1)) for k in range(3)]
    probs.append(W.random_problem(3104, 1, 3, 1))                   # one point: known on the host
    for form in ("pruned", "full"):
        ms, streams = [], []
        for p in probs:
            m = LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), 1.0, norm=p.norm, w=p.w)
            m.set_estimate_form(form)
            ms.append(m)
            streams.append(torch.cuda.Stream())
        torch.cuda.synchronize()
        for m, s in zip(ms, streams):
            with torch.cuda.stream(s):
                m.lipschitz_constant_async()
        got = []
        for m, s in zip(ms, streams):
            got.append(m.lipschitz_constant_result())
            with torch.cuda.stream(s):
                assert L.lip_estimate_M_result(m.h)[0] == L.LIP_ERR_STATE
                if m.N > 1:
                    work = m.last_estimate_work()
                    assert (work[0] > 0) == (form == "pruned"), work
                assert m.lipschitz_constant() == got[-1]
                m.check()
        for m in ms:
            m.close()
        for p, g in zip(probs[:3], got):
            assert g == oracle_mod.estimate_M(p.X, p.y, p.norm, w=p.w), (form, g)
        assert got[3][1] == -1 and got[3][0] == 0.0
