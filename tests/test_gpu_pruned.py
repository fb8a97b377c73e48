"""The pruned scan (lip_set_tuning variants 6 and 7): the data in spatial order with a
bounding box and value range per 16-point chunk, chunks skipped when their exact FP32 bound
shows they cannot change any query's extrema.  Against the FP64 oracle on every norm and
shape up to d = 8 (monotone, decreasing, weighted), ragged sizes, edge cases, tile sizes
(bit for bit), incremental data, and the benchmark workload at full size on sampled
queries.  Among exactly equal FP32 values the pruned scan may choose another datum than
the unpruned one, so it is compared with the oracle (and with variant 1 through the FP64
values of the chosen data), not index for index with variant 1."""
import numpy as np
import pytest

from paper_2606_04670_b300 import workloads as W
from parity import FP32_TOL, compare, diam, gpu_eval

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHAPES = [(1, 0), (1, 1), (2, 0), (2, 2), (3, 1), (4, 2), (4, 4), (5, 3), (6, 0), (7, 2), (8, 3), (8, 8), (9, 0),
          (12, 0), (16, 0)]


@pytest.mark.parametrize("norm", (1, 2, 3))
@pytest.mark.parametrize("d,c", SHAPES)
def test_pruned_matches_oracle(oracle_mod, norm, d, c):
    rng = np.random.default_rng(100 * d + 10 * c + norm)
    p = W.random_problem(2000 + 10 * d + c, 3_001 + 97 * d, d, 1_111, norm=norm, masked=c > 0, weighted=True,
                         decreasing=c > 0)
    if c > 0:                       # exactly c constrained coordinates, some of them decreasing
        mon = np.zeros(d, np.int8)
        mon[rng.choice(d, c, replace=False)] = rng.choice([-1, 1], c)
        p = W.Problem(p.name, p.X, p.y, p.Q, p.M, norm, mon, p.w)
    orc = oracle_mod.evaluate(p.X, p.y, p.Q, p.M, norm, mon=p.mon, w=p.w)
    for v in (6, 7):
        compare(p, gpu_eval(p, variant=v), orc, FP32_TOL, f"pruned v{v} d={d} c={c} L{norm}")


def test_pruned_tile_sizes_bit_for_bit():
    """The start chunk is aligned to 64 groups, so the order of the chunks, and with it
    every result, is the same for every tile size."""
    p = W.monotone_d4(norm=W.NORM_L2, n_data=20_000, n_query=7_777)
    ref = gpu_eval(p, variant=6, tile_groups=64)
    for tg in (8, 16, 32):
        got = gpu_eval(p, variant=6, tile_groups=tg)
        for k in ref:
            np.testing.assert_array_equal(got[k], ref[k], err_msg=f"tile {tg} {k}")


@pytest.mark.parametrize("norm", (1, 2, 3))
def test_pruned_equals_unpruned_values(norm):
    """Same extrema as the unpruned scan: the FP64 bounds of the chosen data agree with
    variant 1 wherever the chosen data agree, and within FP32 ties elsewhere."""
    p = W.monotone_d4(norm=norm, n_data=30_000, n_query=20_000)
    a, b = gpu_eval(p, variant=1), gpu_eval(p, variant=6)
    scale = p.M * diam(p.X, p.Q, norm) + np.abs(p.y).max()
    for kv, ki in (("hi", "idx_up"), ("lo", "idx_lo")):
        same = a[ki] == b[ki]
        assert same.mean() > 0.999, (kv, same.mean())
        np.testing.assert_array_equal(a[kv][same], b[kv][same])
        assert np.all(np.abs(a[kv].astype(np.float64) - b[kv]) <= 4e-7 * scale), kv


def test_pruned_edge_cases(oracle_mod):
    from paper_2606_04670_b300.lipfit import LipFit
    # one datum; NaN and infinite queries; fewer queries than a block; a cleared handle
    p = W.random_problem(2100, 1, 3, 5, norm=W.NORM_L2, masked=True)
    orc = oracle_mod.evaluate(p.X, p.y, p.Q, p.M, p.norm, mon=p.mon)
    compare(p, gpu_eval(p, variant=6), orc, FP32_TOL, "N=1")
    p = W.random_problem(2101, 2_000, 4, 300, norm=W.NORM_L1, masked=True, decreasing=True)
    Q = p.Q.copy()
    Q[7, 1] = np.nan
    Q[9, 0] = np.inf
    m = LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), p.M, norm=p.norm, mon=p.mon)
    m.set_tuning(0, 0, 6)
    r = {k: v.cpu().numpy() for k, v in m.eval(torch.as_tensor(Q).cuda()).items()}
    for i in (7, 9):
        assert np.isnan(r["g"][i]) and r["idx_up"][i] == -1 and r["idx_lo"][i] == -1
    keep = np.isfinite(Q).all(1)
    ps = W.Problem("e", p.X, p.y, Q[keep], p.M, p.norm, p.mon, None)
    compare(ps, {k: v[keep] for k, v in r.items()}, oracle_mod.evaluate(p.X, p.y, Q[keep], p.M, p.norm, mon=p.mon),
            FP32_TOL, "nan queries")
    m.clear()
    r = m.eval(torch.as_tensor(p.Q).cuda())
    assert torch.isnan(r["g"]).all() and (r["idx_up"] == -1).all()
    m.check()
    m.close()


def test_pruned_incremental_data_and_M(oracle_mod):
    """The position-ordered layout is rebuilt after add, clear and set_M."""
    from paper_2606_04670_b300.lipfit import LipFit
    p = W.random_problem(2200, 5_000, 3, 900, norm=W.NORM_L2, masked=True, weighted=True)
    m = LipFit(M=p.M, norm=p.norm, mon=p.mon, w=p.w, capacity=p.N, d=p.d)
    m.set_tuning(0, 0, 6)
    Q = torch.as_tensor(p.Q).cuda()
    m.add(torch.as_tensor(p.X[:1500]).cuda(), torch.as_tensor(p.y[:1500]).cuda())
    r1 = {k: v.cpu().numpy() for k, v in m.eval(Q).items()}
    p1 = W.Problem("a", p.X[:1500], p.y[:1500], p.Q, p.M, p.norm, p.mon, p.w)
    compare(p1, r1, oracle_mod.evaluate(p1.X, p1.y, p.Q, p.M, p.norm, mon=p.mon, w=p.w), FP32_TOL, "first add")
    m.add_async(torch.as_tensor(p.X[1500:]).cuda(), torch.as_tensor(p.y[1500:]).cuda())
    r2 = {k: v.cpu().numpy() for k, v in m.eval(Q).items()}
    compare(p, r2, oracle_mod.evaluate(p.X, p.y, p.Q, p.M, p.norm, mon=p.mon, w=p.w), FP32_TOL, "second add")
    m.set_M(2.0 * p.M)
    r3 = {k: v.cpu().numpy() for k, v in m.eval(Q).items()}
    p3 = W.Problem("m", p.X, p.y, p.Q, 2.0 * p.M, p.norm, p.mon, p.w)
    compare(p3, r3, oracle_mod.evaluate(p.X, p.y, p.Q, 2.0 * p.M, p.norm, mon=p.mon, w=p.w), FP32_TOL, "set_M")
    m.check()
    m.close()


def test_pruned_duplicates_and_constant_y(oracle_mod):
    """Many exactly equal values: duplicated points and a constant y with M = 0.  The chosen
    datum's FP64 bound equals the envelope."""
    p = W.random_problem(2300, 4_000, 2, 500, norm=W.NORM_L2)
    X = np.concatenate([p.X, p.X[:2000]])
    y = np.concatenate([p.y, p.y[:2000]])
    pd = W.Problem("dup", X, y, p.Q, p.M, p.norm, None, None)
    orc = oracle_mod.evaluate(X, y, p.Q, p.M, p.norm)
    compare(pd, gpu_eval(pd, variant=6), orc, FP32_TOL, "duplicates")
    pc = W.Problem("const", p.X, np.full(p.N, 0.5, np.float32), p.Q, 0.0, p.norm, None, None)
    r = gpu_eval(pc, variant=6)
    assert np.all(r["hi"] == 0.5) and np.all(r["lo"] == 0.5) and np.all(r["idx_up"] >= 0)


def test_pruned_full_size_benchmark_workload(oracle_mod):
    """The benchmark workload (N = 1e5, Q = 1e6, monotone d = 4) at full size, all three
    norms, on 1,000 sampled queries per norm, plus lo <= g <= hi everywhere; the scan
    evaluates a small share of the (row, chunk) pairs."""
    from paper_2606_04670_b300.lipfit import LipFit
    rng = np.random.default_rng(5)
    for norm in (1, 2, 3):
        p = W.monotone_d4(norm=norm)
        m = LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), p.M, norm=norm, mon=p.mon)
        m.set_tuning(0, 0, 6)
        r = {k: v.cpu().numpy() for k, v in m.eval(torch.as_tensor(p.Q).cuda()).items()}
        ev, tot = m.last_scan_work()
        st = m.last_scan_stats()
        m.check()
        m.close()
        assert 0 < ev < 0.5 * tot, (norm, ev, tot)
        # the same counts, the tiles copied out of blocks x tiles, and the (warp, chunk)
        # pairs past the warp-box test: at most 16 chunks a tile, 4 warps a block
        assert st[:2] == [ev, tot] and 0 < st[2] <= st[3] and 0 < st[4] <= 16 * 4 * st[2], st
        assert np.all(r["lo"] <= r["g"]) and np.all(r["g"] <= r["hi"])
        idx = np.sort(rng.choice(p.nq, 1_000, replace=False))
        ps = W.Problem("s", p.X, p.y, p.Q[idx], p.M, norm, p.mon, None)
        orc = oracle_mod.evaluate(p.X, p.y, ps.Q, p.M, norm, mon=p.mon)
        compare(ps, {k: v[idx] for k, v in r.items()}, orc, FP32_TOL, f"full L{norm}")


def test_pruned_autotune_and_tuning_report():
    from paper_2606_04670_b300 import lipfit as L
    p = W.random_problem(2400, 3_000, 4, 2_000, norm=W.NORM_L2, masked=True)
    m = L.LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), p.M, norm=p.norm, mon=p.mon)
    m.set_tuning(0, 0, 7)
    assert m.tuning()["variant"] == 7 and m.tuning()["queries_per_thread"] == 8
    m.eval(torch.as_tensor(p.Q).cuda())
    assert m.last_scan_work()[1] > 0 and m.tuning()["last_splits"] == 1
    m.set_tuning(0, 0, 1)
    m.eval(torch.as_tensor(p.Q).cuda())
    assert m.last_scan_work() == (-1, -1)
    assert m.last_scan_stats() == [-1, -1, -1, -1, -1]
    assert L.lip_set_tuning(m.h, 0, 0, 8) == L.LIP_ERR_ARG
    m.close()
    # d = 17 has no pruned instantiation (nor has d = 9..16 with constrained coordinates):
    # 6 / 7 run as 0 / 1
    p = W.random_problem(2401, 1_000, 17, 300, norm=W.NORM_L1)
    m = L.LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), p.M, norm=p.norm)
    m.set_tuning(0, 0, 6)
    m.eval(torch.as_tensor(p.Q).cuda())
    assert m.last_scan_work() == (-1, -1)
    m.close()


@pytest.mark.parametrize("case", ("cluster_d16", "monotone_d5_L1"))
def test_pruned_cyclic_order(oracle_mod, case):
    """More than 1,024 super-chunks (N > 262,144 data): the sweep runs in cyclic order from
    the block's start chunk instead of sorting the super-chunks.  The clustered d = 16 workload at full size (N = Q = 1e6, as the benchmark
    runs it) on 400 sampled queries, and a monotone, weighted d = 5 problem under L1 on all
    of its queries, against the FP64 oracle."""
    from paper_2606_04670_b300.lipfit import LipFit
    if case == "cluster_d16":
        p = W.cluster_d16()
        idx = np.sort(np.random.default_rng(23).choice(p.nq, 400, replace=False))
    else:
        p = W.random_problem(2402, 300_000, 5, 3_000, norm=W.NORM_L1, masked=True, weighted=True, decreasing=True)
        idx = np.arange(p.nq)
    m = LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), p.M, norm=p.norm, mon=p.mon, w=p.w)
    m.set_tuning(0, 0, 6)
    r = {k: v.cpu().numpy() for k, v in m.eval(torch.as_tensor(p.Q).cuda()).items()}
    ev, tot = m.last_scan_work()
    m.check()
    m.close()
    assert 0 < ev < 0.5 * tot, (ev, tot)
    assert np.all(r["lo"] <= r["g"]) and np.all(r["g"] <= r["hi"])
    ps = W.Problem("s", p.X, p.y, p.Q[idx], p.M, p.norm, p.mon, p.w)
    orc = oracle_mod.evaluate(p.X, p.y, ps.Q, p.M, p.norm, mon=p.mon, w=p.w)
    compare(ps, {k: v[idx] for k, v in r.items()}, orc, FP32_TOL, case)
