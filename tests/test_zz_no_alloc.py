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
