"""k > 1 neighbours (lip_eval_k) against the FP64 oracle.  Needs a CUDA device."""
import numpy as np
import pytest

from paper_2606_04670_b300 import workloads as W
from parity import FP32_TOL, diam

pytestmark = pytest.mark.gpu


def _run(p, k, wk, precision="fp32"):
    import torch

    from paper_2606_04670_b300.lipfit import LipFit
    dt = torch.float64 if precision == "fp64" else torch.float32
    m = LipFit(torch.as_tensor(p.X).to("cuda", dt), torch.as_tensor(p.y).to("cuda", dt), p.M, norm=p.norm,
               mon=p.mon, w=p.w, precision=precision)
    r = {key: v.cpu().numpy() for key, v in m.eval_k(torch.as_tensor(p.Q).to("cuda", dt), k, wk).items()}
    m.close()
    return r


def _clear(oracle_mod, p, k, tol):
    """Queries whose k + 1 smallest upper bounds (oracle, one-hot weights) differ by > tol."""
    vals = []
    for j in range(k + 1):
        e = np.zeros(k + 1)
        e[j] = 1.0
        vals.append(oracle_mod.evaluate_k(p.X, p.y, p.Q, p.M, k + 1, e, p.norm, mon=p.mon, w=p.w).hi)
    v = np.stack(vals, 1)
    return (np.diff(v, axis=1) > tol).all(1)


@pytest.mark.parametrize("norm", (1, 2, 3))
@pytest.mark.parametrize("d,masked,weighted,k", [(1, False, False, 2), (3, True, False, 3), (5, True, True, 5),
                                                 (12, True, True, 8), (4, False, True, 1), (16, False, False, 4)])
def test_eval_k_vs_oracle(oracle_mod, norm, d, masked, weighted, k):
    p = W.random_problem(1000 + d, 2_345, d, 301, norm=norm, masked=masked, weighted=weighted, decreasing=masked)
    wk = np.random.default_rng(k).random(k)
    wk /= wk.sum()
    r = _run(p, k, wk)
    o = oracle_mod.evaluate_k(p.X, p.y, p.Q, p.M, k, wk, norm, mon=p.mon, w=p.w)
    tol = FP32_TOL * p.M * diam(p.X, p.Q, norm, p.w)
    for key in ("hi", "lo", "g"):
        err = np.abs(r[key].astype(np.float64) - o[key])
        assert err.max() <= tol, (key, err.max(), tol)
    # the selected indices (in bound order) agree wherever the oracle's k + 1 best upper
    # bounds are separated by more than the tolerance
    ok = _clear(oracle_mod, p, k, tol)
    assert r["idx_up"].shape == (p.nq, k)
    bad = ok & ~(r["idx_up"] == o.idx_up).all(1)
    assert not bad.any(), np.nonzero(bad)[0][:5]


def test_eval_k_one_equals_eval(oracle_mod):
    import torch

    from paper_2606_04670_b300.lipfit import LipFit
    p = W.monotone_d4(norm=W.NORM_L1, n_data=7_001, n_query=999)
    m = LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), p.M, norm=p.norm, mon=p.mon)
    Q = torch.as_tensor(p.Q).cuda()
    a = {k: v.cpu().numpy() for k, v in m.eval(Q).items()}
    b = {k: v.cpu().numpy() for k, v in m.eval_k(Q, 1, [1.0]).items()}
    m.close()
    tol = FP32_TOL * p.M * diam(p.X, p.Q, p.norm)
    for key in ("hi", "lo", "g"):
        assert np.abs(a[key] - b[key]).max() <= tol
    assert (a["idx_up"] == b["idx_up"][:, 0]).mean() > 0.99


def test_eval_k_fewer_points_than_k_and_args():
    import torch

    from paper_2606_04670_b300.lipfit import LipError, LipFit
    p = W.random_problem(1100, 3, 2, 5)
    m = LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), p.M)
    r = m.eval_k(torch.as_tensor(p.Q).cuda(), 4, [0.25] * 4)
    assert torch.isnan(r["g"]).all() and (r["idx_up"] == -1).all()
    r = m.eval_k(torch.as_tensor(p.Q).cuda(), 3, [0.5, 0.3, 0.2])
    assert torch.isfinite(r["g"]).all() and (r["idx_up"] >= 0).all()
    with pytest.raises(LipError):
        m.eval_k(torch.as_tensor(p.Q).cuda(), 9, [0.1] * 9)
    with pytest.raises(LipError):
        m.eval_k(torch.as_tensor(p.Q).cuda(), 2, [0.5, -0.5])
    m.close()
