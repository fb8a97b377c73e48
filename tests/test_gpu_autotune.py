"""The autotuner picks a launch shape by timing and never changes results."""
import numpy as np
import pytest

from paper_2606_04670_b300 import workloads as W

pytestmark = pytest.mark.gpu


def test_tune_eval_keeps_results_and_caches(tmp_path):
    import torch

    from paper_2606_04670_b300 import autotune as AT
    from paper_2606_04670_b300.lipfit import LipFit
    p = W.monotone_d4(norm=W.NORM_L2, n_data=20_000, n_query=50_000)
    m = LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), p.M, norm=p.norm, mon=p.mon)
    Q = torch.as_tensor(p.Q).cuda()
    ref = {k: v.cpu().numpy() for k, v in m.eval(Q).items()}
    cache = {}
    # variants 0 / 1 (queries per thread) with tiles and splits never change a result; the
    # FMA-pipe square-root variants 2-5 are checked against the oracle in test_gpu_eval
    rec = AT.tune_eval(m, Q, tiles=(8, 32), splits=(0, 1, 4), variants=(0, 1), cache=cache, reps=2)
    assert not rec["cached"] and rec["ms"] <= rec["default_ms"] + 1e-9 and rec["candidates"] == 12
    assert m.tuning()["tile_groups"] == rec["tile_groups"]
    got = {k: v.cpu().numpy() for k, v in m.eval(Q).items()}
    for k in ref:
        np.testing.assert_array_equal(got[k], ref[k])
    path = str(tmp_path / "cache.json")
    AT.save_cache(cache, path)
    again = AT.tune_eval(m, Q, cache=AT.load_cache(path))
    assert again["cached"] and again["tile_groups"] == rec["tile_groups"]
    m.close()


def test_tune_batch_returns_options():
    import torch

    from paper_2606_04670_b300 import autotune as AT
    plan = W.batch_plan(n_sets=12, n_max=4000, q_min=100, q_max=1500)
    sets = []
    for bs in plan:
        X, y, Q, f = W.batch_set_data(bs)
        sets.append(dict(X=torch.as_tensor(X), y=torch.as_tensor(y), Q=torch.as_tensor(Q).cuda(), M=bs.M,
                         norm=bs.norm, mon=bs.mon))
    rec = AT.tune_batch(sets, tiles=(16, 32), items=(4, 8), cache={}, reps=1)
    assert rec["tile_groups"] in (16, 32) and rec["items_per_block"] in (4, 8) and rec["candidates"] == 4


def test_c_abi_autotune_keeps_results():
    """lip_autotune (the library's own tuner) applies a launch shape and changes no result."""
    import torch

    from paper_2606_04670_b300 import lipfit as L
    from paper_2606_04670_b300.lipfit import LipFit
    for prec, p in (("fp32", W.monotone_d4(norm=W.NORM_L1, n_data=8_000, n_query=20_000)),
                    ("fp64", W.random_problem(7, 3_000, 3, 2_000, norm=2, dtype=np.float64))):
        dt = torch.float64 if prec == "fp64" else torch.float32
        m = LipFit(torch.as_tensor(p.X).to("cuda", dt), torch.as_tensor(p.y).to("cuda", dt), p.M, norm=p.norm,
                   mon=p.mon, precision=prec)
        Q = torch.as_tensor(p.Q).to("cuda", dt)
        ref = {k: v.cpu().numpy() for k, v in m.eval(Q).items()}
        s, tg, sp, v, ms = L.lip_autotune(m.h, Q.data_ptr(), Q.shape[0], 2, torch.cuda.current_stream().cuda_stream)
        assert s == L.LIP_OK, L.last_error()
        assert tg in (8, 16, 32, 64) and ms > 0
        t = m.tuning()
        assert (t["tile_groups"], t["splits"]) == (tg, sp)
        got = {k: v.cpu().numpy() for k, v in m.eval(Q).items()}
        for k in ref:
            np.testing.assert_array_equal(got[k], ref[k])
        m.close()


def test_tune_eval_sweeps_the_square_root_variants(oracle_mod):
    """FP32 handles sweep all eight variants by default (the pruned ones, 6 and 7, take one
    split candidate: they scan all the data in one launch); the tuned evaluation still
    matches the oracle within the FP32 tolerance."""
    import torch

    from paper_2606_04670_b300 import autotune as AT
    from paper_2606_04670_b300.lipfit import LipFit
    from parity import FP32_TOL, compare
    p = W.monotone_d4(norm=W.NORM_L2, n_data=12_000, n_query=30_000)
    m = LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), p.M, norm=p.norm, mon=p.mon)
    Q = torch.as_tensor(p.Q).cuda()
    rec = AT.tune_eval(m, Q, tiles=(32,), splits=(0, 4), cache={}, reps=2)
    assert rec["candidates"] == 6 * 2 + 2 and 0 <= rec["variant"] < 8
    got = {k: v.cpu().numpy() for k, v in m.eval(Q).items()}
    m.close()
    sub = np.arange(0, p.nq, 15)
    ps = p.sub_queries(p.nq)
    ps.Q = p.Q[sub]
    orc = oracle_mod.evaluate(p.X, p.y, ps.Q, p.M, p.norm, mon=p.mon)
    compare(ps, {k: v[sub] for k, v in got.items()}, orc, FP32_TOL, "tuned")
