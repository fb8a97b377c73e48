"""lip_estimate_M_noalloc, the estimate for callers that cannot allocate device memory
(for example a plugin whose host application's allocator already holds the GPU's
memory).  It must give what lip_estimate_M gives on the same data, call after call,
even though every call reuses the library's one fixed working array.  This file is
collected last on purpose, so that a failure here comes after every other test ran."""
import ctypes

import numpy as np
import pytest

from paper_2606_04670_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _via_handle(p):
    import torch

    from paper_2606_04670_b300.lipfit import LipFit
    m = LipFit(torch.as_tensor(p.X).cuda(), torch.as_tensor(p.y).cuda(), 1.0, norm=p.norm, w=p.w)
    M, i, j = m.lipschitz_constant()
    m.close()
    return M, i, j


def _via_noalloc(p, out):
    import torch

    from paper_2606_04670_b300 import lipfit as L
    X = torch.as_tensor(p.X).cuda()
    y = torch.as_tensor(p.y).cuda()
    w = None if p.w is None else np.ascontiguousarray(p.w, np.float64)
    s = L.lip_estimate_M_noalloc(X.data_ptr(), y.data_ptr(), p.N, p.d, p.norm,
                                 None if w is None else w.ctypes.data, out.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
    assert s == L.LIP_OK, L.last_error()
    torch.cuda.synchronize()
    M, i, j = out.cpu().tolist()
    return M, int(i), int(j)


def test_noalloc_matches_estimate_M_on_consecutive_calls():
    import torch
    out = torch.full((3,), -7.0, dtype=torch.float64, device="cuda")
    # a large call, then a smaller one on the same working array (stale contents must
    # not leak into the second), then the large one again
    cases = [W.random_problem(900, 30_001, 5, 1, norm=W.NORM_L2, weighted=True),
             W.random_problem(901, 1_234, 3, 1, norm=W.NORM_L1),
             W.random_problem(900, 30_001, 5, 1, norm=W.NORM_L2, weighted=True),
             W.random_problem(902, 777, 16, 1, norm=W.NORM_LINF, weighted=True)]
    for p in cases:
        M0, i0, j0 = _via_handle(p)
        M1, i1, j1 = _via_noalloc(p, out)
        assert abs(M1 - M0) <= 1e-5 * M0, (p.name, M1, M0)
        assert (i1, j1) == (i0, j0)


def test_noalloc_at_its_exact_capacity():
    """N = LIP_NOALLOC_N_MAX at d = LIP_D_MAX fills the fixed array's layout and its
    candidate records to the last byte; the result must still equal lip_estimate_M's, and
    the pair must be the FP64 oracle's maximum on a row sample."""
    import torch

    from paper_2606_04670_b300 import lipfit as L
    out = torch.full((3,), -7.0, dtype=torch.float64, device="cuda")
    n = L.LIP_NOALLOC_N_MAX
    for seed, d, norm in ((903, 16, W.NORM_L2), (904, 3, W.NORM_LINF)):
        p = W.random_problem(seed, n, d, 1, norm=norm, weighted=True)
        M0, i0, j0 = _via_handle(p)
        for _ in range(2):
            M1, i1, j1 = _via_noalloc(p, out)
            assert abs(M1 - M0) <= 1e-5 * M0, (d, M1, M0)
            assert (i1, j1) == (i0, j0)
        # the returned pair's exact ratio is the returned M (FP64 re-evaluation)
        Z = p.X.astype(np.float64) * np.asarray(p.w)[None, :]
        t = np.abs(Z[i1] - Z[j1])
        dist = {W.NORM_L1: t.sum(), W.NORM_L2: np.sqrt((t * t).sum()), W.NORM_LINF: t.max()}[norm]
        assert abs(M1 - abs(float(p.y[i1]) - float(p.y[j1])) / dist) <= 1e-12 * M1


def test_noalloc_constant_values():
    """Constant y at distinct points gives M = 0 with a real pair (the lowest), like the
    handle path; repeated points with equal y give -1 / -1."""
    import torch
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    p = W.random_problem(905, 700, 4, 1, norm=W.NORM_L2)
    p = W.Problem(p.name, p.X, np.full_like(p.y, 0.75), p.Q, p.M, p.norm, p.mon, p.w, None)
    assert _via_noalloc(p, out) == _via_handle(p) == (0.0, 0, 1)
    X = np.tile(p.X[:1], (5, 1))
    q = W.Problem(p.name, X, np.full(5, 0.75, np.float32), p.Q, p.M, p.norm, None, None, None)
    assert _via_noalloc(q, out) == (0.0, -1, -1)


def test_noalloc_rejects_sizes_beyond_its_capacity():
    import torch

    from paper_2606_04670_b300 import lipfit as L
    n = L.LIP_NOALLOC_N_MAX + 1
    X = torch.zeros(n, 2, device="cuda")
    y = torch.zeros(n, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    s = L.lip_estimate_M_noalloc(X.data_ptr(), y.data_ptr(), n, 2, L.LIP_L2, None, out.data_ptr(), 0)
    assert s == L.LIP_ERR_ARG and "capacity" in L.last_error()
    # a single point: no pair, M = 0 and indices -1
    s = L.lip_estimate_M_noalloc(X.data_ptr(), y.data_ptr(), 1, 2, L.LIP_L2, None, out.data_ptr(), 0)
    assert s == L.LIP_OK
    torch.cuda.synchronize()
    assert out.cpu().tolist() == [0.0, -1.0, -1.0]
