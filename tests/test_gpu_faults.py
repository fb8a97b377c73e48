"""Failure detection without a device fault.

* A bounded device wait that runs out: the exact scan is told to leave out one data tile's
  bulk copy, so its wait on that tile's barrier gives up after a short limit.  The kernel
  records the timeout, waits for the copies it did issue and returns; lip_check reports
  LIP_ERR_TIMEOUT and the handle evaluates correctly afterwards.
* Device allocation failure: lip_debug_fail_alloc makes the n-th allocation report
  out-of-memory (host side, no cudaMalloc), for every allocation the calls make in turn.
  The calls return LIP_ERR_OOM, leak nothing and leave the handle as it was."""
import ctypes

import numpy as np
import pytest

from paper_2606_04670_b300 import workloads as W
from parity import FP32_TOL, compare

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2606_04670_b300 import lipfit as L
    return L


def _eval(m, Q):
    r = m.eval(Q)
    return {k: v.cpu().numpy() for k, v in r.items()}


@pytest.mark.parametrize("skip_tile", [0, 2])
def test_scan_wait_runs_out_and_handle_recovers(oracle_mod, skip_tile):
    import torch
    L = _lib()
    p = W.monotone_d4(norm=W.NORM_L2, n_data=20_011, n_query=3_001)
    m = L.LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), p.M, norm=p.norm, mon=p.mon)
    m.set_tuning(8, 4, 0)              # 4 data splits of about 20 tiles each: every block has tile 2
    Q = torch.as_tensor(p.Q).cuda()
    assert L.lip_debug_scan_fault(m.h, 20_000, skip_tile) == L.LIP_OK
    r = _eval(m, Q)
    torch.cuda.synchronize()
    assert L.lip_check(m.h, torch.cuda.current_stream().cuda_stream) == L.LIP_ERR_TIMEOUT
    # every block gave up before finishing its share: no value and no index survives
    assert np.all(np.isnan(r["g"])) and np.all(r["idx_up"] == -1) and np.all(r["idx_lo"] == -1)
    # the status is cleared by lip_check, and evaluation works again
    assert L.lip_debug_scan_fault(m.h, 0, -1) == L.LIP_OK
    r = _eval(m, Q)
    m.check()
    orc = oracle_mod.evaluate(p.X, p.y, p.Q, p.M, p.norm, mon=p.mon)
    compare(p, r, orc, FP32_TOL, "after the timeout")
    m.close()


def test_scan_fault_argument_checks():
    L = _lib()
    assert L.lip_debug_scan_fault(None, 0, -1) == L.LIP_ERR_ARG
    assert L.lip_debug_fail_alloc(-1) == L.LIP_ERR_ARG
    assert L.lip_debug_fail_alloc(0) == L.LIP_OK


def _free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _fit(L, X, y, N, d, M, params):
    import torch
    s, h = L.lip_fit(X.data_ptr(), y.data_ptr(), N, d, M, params, torch.cuda.current_stream().cuda_stream)
    return s, h


@pytest.mark.parametrize("precision", ["fp32", "fp64", "tc_tf32"])
def test_fit_allocation_failures(precision):
    import torch
    L = _lib()
    dt = torch.float64 if precision == "fp64" else torch.float32
    p = W.random_problem(950, 5_000, 6, 700, norm=W.NORM_L2)
    X, y = torch.as_tensor(p.X).to("cuda", dt), torch.as_tensor(p.y).to("cuda", dt)
    params, keep = L.make_params(p.norm, precision)
    # one complete round first, so lazily loaded kernels are resident before measuring
    s, h = _fit(L, X, y, p.N, p.d, p.M, params)
    assert s == L.LIP_OK
    L.lip_free(h)
    failures = 0
    for n in range(1, 40):
        before = _free_bytes()
        assert L.lip_debug_fail_alloc(n) == L.LIP_OK
        s, h = _fit(L, X, y, p.N, p.d, p.M, params)
        L.lip_debug_fail_alloc(0)
        if s == L.LIP_OK:
            L.lip_free(h)
            break
        assert s == L.LIP_ERR_OOM, (n, s, L.last_error())
        assert not h.value and "out of device memory" in L.last_error()
        assert _free_bytes() == before, f"allocation {n}: device memory leaked"
        failures += 1
    assert 4 <= failures < 39


@pytest.mark.parametrize("precision", ["fp32", "fp64", "tc_bf16"])
def test_eval_and_estimate_allocation_failures(oracle_mod, precision):
    """Scratch growth in lip_eval and lip_estimate_M fails: LIP_ERR_OOM, the handle keeps its
    data and gives the oracle's results once allocations work again."""
    import torch
    L = _lib()
    dt = torch.float64 if precision == "fp64" else torch.float32
    p = W.random_problem(951, 3_000, 5, 2_000, norm=W.NORM_L2)
    m = L.LipFit(torch.as_tensor(p.X).to("cuda", dt), torch.as_tensor(p.y).to("cuda", dt), p.M, norm=p.norm,
                 precision=precision)
    Q = torch.as_tensor(p.Q).to("cuda", dt)
    small = Q[:64].contiguous()
    _eval(m, small)                    # scratch sized for 64 queries; the full call must grow it
    m.check()
    outs = {k: torch.empty(p.nq, dtype=dt, device="cuda") for k in ("g", "lo", "hi")}
    idx = {k: torch.empty(p.nq, dtype=torch.int32, device="cuda") for k in ("idx_up", "idx_lo")}
    st = torch.cuda.current_stream().cuda_stream
    failures = 0
    for n in range(1, 20):
        L.lip_debug_fail_alloc(n)
        s = L.lip_eval(m.h, Q.data_ptr(), p.nq, outs["g"].data_ptr(), outs["lo"].data_ptr(), outs["hi"].data_ptr(),
                       idx["idx_up"].data_ptr(), idx["idx_lo"].data_ptr(), st)
        L.lip_debug_fail_alloc(0)
        if s == L.LIP_OK:
            break
        assert s == L.LIP_ERR_OOM, (n, s, L.last_error())
        assert L.lip_size(m.h) == p.N
        failures += 1
    assert failures >= 1
    torch.cuda.synchronize()
    m.check()
    orc = oracle_mod.evaluate(p.X, p.y, p.Q, p.M, p.norm)
    got = {k: v.cpu().numpy() for k, v in {**outs, **idx}.items()}
    compare(p, got, orc, FP32_TOL, f"eval after OOM ({precision})")
    # the estimate's scratch
    L.lip_debug_fail_alloc(1)
    s, M, i, j = L.lip_estimate_M(m.h, st)
    L.lip_debug_fail_alloc(0)
    assert s == L.LIP_ERR_OOM and L.lip_size(m.h) == p.N
    s, M, i, j = L.lip_estimate_M(m.h, st)
    Mo, io, jo = oracle_mod.estimate_M(p.X, p.y, p.norm)
    assert s == L.LIP_OK and abs(M - Mo) <= 1e-5 * Mo and (i, j) == (io, jo)
    m.close()


def test_batch_and_local_allocation_failures():
    import torch
    L = _lib()
    p = W.random_problem(952, 2_000, 3, 100, norm=W.NORM_L1)
    X, y, Q = (torch.as_tensor(a).cuda() for a in (p.X, p.y, p.Q))
    m = L.LipFit(X, y, p.M, norm=p.norm)
    L.lip_debug_fail_alloc(1)
    with pytest.raises(L.LipError) as e:
        m.compute_local_lipschitz(8, 500, 1)
    L.lip_debug_fail_alloc(0)
    assert e.value.status == L.LIP_ERR_OOM
    with pytest.raises(L.LipError) as e:      # no table was made
        m.eval_local(Q)
    assert e.value.status == L.LIP_ERR_STATE
    m.compute_local_lipschitz(8, 500, 1)
    m.eval_local(Q)
    m.close()
    outs = [{k: torch.empty(p.nq, device="cuda") for k in ("g", "lo", "hi")}]
    outs[0].update({k: torch.empty(p.nq, device="cuda", dtype=torch.int32) for k in ("idx_up", "idx_lo")})
    sets = [dict(X=X, y=y, Q=Q, M=p.M, norm=p.norm, mon=None)]
    L.LipBatch(sets, outputs=outs).close()          # kernels resident before measuring
    before = _free_bytes()
    for n in (1, 3):
        L.lip_debug_fail_alloc(n)
        with pytest.raises(L.LipError) as e:
            L.LipBatch(sets, outputs=outs)
        L.lip_debug_fail_alloc(0)
        assert e.value.status == L.LIP_ERR_OOM and _free_bytes() == before
