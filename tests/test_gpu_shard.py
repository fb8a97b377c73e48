"""The multi-GPU kernels on one GPU: the ranks of a data-sharded evaluation and of the
shared estimate are emulated in one process (each "rank" a handle on its slice of the data,
run one after the other; the all-reduces become element-wise minima and maxima here).  The
merged results must equal lip_eval / lip_estimate_M on one handle holding all the data, bit
for bit, and the FP64 oracle within the FP32 tolerance."""
import numpy as np
import pytest

from paper_2606_04670_b300 import shard as S
from paper_2606_04670_b300 import workloads as W
from parity import FP32_TOL, compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _handles(p, bounds, precision="fp32"):
    from paper_2606_04670_b300.lipfit import LipFit
    out = []
    for b, e in bounds:
        X = torch.as_tensor(p.X[b:e]).cuda()
        y = torch.as_tensor(p.y[b:e]).cuda()
        if e > b:
            m = LipFit(X, y, p.M, norm=p.norm, mon=p.mon, w=p.w, precision=precision)
        else:       # a rank without data: an empty handle
            m = LipFit(M=p.M, norm=p.norm, mon=p.mon, w=p.w, precision=precision, capacity=16, d=p.d)
        out.append((S.DeviceShard(m, b), m))
    return out


def _sharded_eval(shards, Q):
    keys = [sh.scan(Q) for sh, _ in shards]
    ku = torch.stack([k[0] for k in keys]).min(0).values
    kl = torch.stack([k[1] for k in keys]).min(0).values
    vals = [sh.reeval(Q, ku, kl) for sh, _ in shards]
    hi = torch.stack([v[0] for v in vals]).min(0).values
    lo = torch.stack([v[1] for v in vals]).max(0).values
    return shards[0][0].finish(ku, kl, hi, lo)


@pytest.mark.parametrize("norm", [W.NORM_L1, W.NORM_L2, W.NORM_LINF])
def test_data_sharded_eval_equals_single_handle(oracle_mod, norm):
    from paper_2606_04670_b300.lipfit import LipFit
    p = W.monotone_d4(norm=norm, n_data=20_011, n_query=3_001)
    Q = torch.as_tensor(p.Q).clone()
    Q[5, 2] = float("nan")
    Q = Q.cuda()
    full = LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), p.M, norm=norm, mon=p.mon)
    ref = {k: v.cpu().numpy() for k, v in full.eval(Q).items()}
    full.close()
    for bounds in ([S.shard_range(p.N, r, 3) for r in range(3)], [(0, 7_777), (7_777, 7_777), (7_777, 20_011)]):
        shards = _handles(p, bounds)
        got = {k: v.cpu().numpy() for k, v in _sharded_eval(shards, Q).items()}
        for k in ref:
            np.testing.assert_array_equal(got[k], ref[k], err_msg=f"{k} {bounds}")
        for _, m in shards:
            m.check()
            m.close()
    # and the oracle (finite queries)
    ok = np.isfinite(Q.cpu().numpy()).all(1)
    ps = p.sub_queries(p.nq)
    ps.Q = p.Q[ok]
    orc = oracle_mod.evaluate(p.X, p.y, ps.Q, p.M, norm, mon=p.mon)
    compare(ps, {k: v[ok] for k, v in ref.items()}, orc, FP32_TOL, f"sharded {norm}")


def test_data_sharded_on_tensor_core_handles_uses_the_fp32_scan():
    """Tensor-core handles take the plain FP32 scan in a data-sharded evaluation: the
    results are those of an FP32 handle on all the data."""
    from paper_2606_04670_b300.lipfit import LipFit
    p = W.random_problem(960, 9_000, 16, 1_000, norm=W.NORM_L2)
    Q = torch.as_tensor(p.Q).cuda()
    full = LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), p.M, norm=p.norm)
    ref = {k: v.cpu().numpy() for k, v in full.eval(Q).items()}
    full.close()
    shards = _handles(p, [S.shard_range(p.N, r, 2) for r in range(2)], precision="tc_bf16")
    got = {k: v.cpu().numpy() for k, v in _sharded_eval(shards, Q).items()}
    for k in ref:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
    for _, m in shards:
        m.close()


@pytest.mark.parametrize("norm", [W.NORM_L1, W.NORM_L2, W.NORM_LINF])
@pytest.mark.parametrize("nparts", [1, 2, 3, 7])
def test_estimate_parts_equal_the_estimate(norm, nparts):
    from paper_2606_04670_b300.lipfit import LipFit
    p = W.random_problem(970 + norm, 5_000, 3, 1, norm=norm, weighted=True)
    m = LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), 1.0, norm=norm, w=p.w)
    M, i, j = m.lipschitz_constant()
    best = [0.0, -1.0, -1.0, -1.0]
    for part in range(nparts):
        c = m.estimate_M_part(part, nparts)
        assert c[1] < 0 or (0 <= c[1] < c[2] < p.N)
        if S._better(c, best):
            best = c
    assert (best[0], int(best[1]), int(best[2])) == (M, i, j)
    m.close()


def test_shard_argument_errors():
    from paper_2606_04670_b300 import lipfit as L
    p = W.random_problem(980, 300, 2, 10, norm=W.NORM_L2, dtype=np.float64)
    m = L.LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), p.M, precision="fp64")
    with pytest.raises(L.LipError) as e:
        m.shard_scan(torch.as_tensor(p.Q).cuda(), 0)
    assert e.value.status == L.LIP_ERR_UNSUPPORTED
    m.close()
    p = W.random_problem(981, 300, 2, 10, norm=W.NORM_L2)
    m = L.LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), p.M)
    with pytest.raises(L.LipError) as e:
        m.shard_scan(torch.as_tensor(p.Q).cuda(), (1 << 31) - 100)
    assert e.value.status == L.LIP_ERR_ARG
    for part, nparts in ((0, 0), (2, 2), (-1, 3)):
        assert L.lip_estimate_M_part(m.h, part, nparts)[0] == L.LIP_ERR_ARG
    m.close()
