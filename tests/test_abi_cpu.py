"""The C ABI without a GPU: the library loads, exports every function the header
declares, and rejects bad arguments on the host before touching the device."""
import ctypes

import numpy as np
import pytest

from paper_2606_04670_b300 import lipfit as L


def test_exports_every_declared_symbol():
    names = L.header_symbols()
    assert len(names) >= 20
    lib = ctypes.CDLL(L.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_version():
    for s in range(10):
        assert L.status_string(s) and L.status_string(s) != "unknown status"
    assert L.status_string(99) == "unknown status"
    assert "sm_103a" in L.lip_version()


def _arr(*shape):
    return np.zeros(shape, np.float32)


@pytest.mark.parametrize("kw,status", [
    ({"N": 0}, L.LIP_ERR_ARG),
    ({"N": 1 << 31}, L.LIP_ERR_ARG),
    ({"d": 0}, L.LIP_ERR_ARG),
    ({"d": 33}, L.LIP_ERR_ARG),
    ({"M": -1.0}, L.LIP_ERR_ARG),
    ({"M": float("nan")}, L.LIP_ERR_ARG),
    ({"M": float("inf")}, L.LIP_ERR_ARG),
    ({"norm": 4}, L.LIP_ERR_ARG),
    ({"precision": 9}, L.LIP_ERR_ARG),
    ({"mon": [2, 0]}, L.LIP_ERR_ARG),
    ({"w": [1.0, 0.0]}, L.LIP_ERR_ARG),
    ({"w": [1.0, float("nan")]}, L.LIP_ERR_ARG),
    ({"norm": L.LIP_L1, "precision": L.LIP_TC_BF16}, L.LIP_ERR_UNSUPPORTED),
    ({"norm": L.LIP_LINF, "precision": L.LIP_TC_TF32}, L.LIP_ERR_UNSUPPORTED),
    ({"norm": L.LIP_L1, "precision": L.LIP_TC_FP16}, L.LIP_ERR_UNSUPPORTED),
    ({"precision": 5}, L.LIP_ERR_ARG),
    ({"nullX": True}, L.LIP_ERR_ARG),
])
def test_fit_argument_errors(kw, status):
    X, y = _arr(8, 2), _arr(8)
    p, keep = L.make_params(kw.get("norm", L.LIP_L2), kw.get("precision", L.LIP_FP32), kw.get("mon"), kw.get("w"))
    s, h = L.lip_fit(None if kw.get("nullX") else X.ctypes.data, y.ctypes.data, kw.get("N", 8), kw.get("d", 2),
                     kw.get("M", 1.0), p)
    assert s == status, L.last_error()
    assert not h.value
    assert L.last_error()


def test_null_handle_calls():
    assert L.lip_eval(None, None, 1, None, None, None, None, None) == L.LIP_ERR_ARG
    assert L.lip_add(None, None, None, 1) == L.LIP_ERR_ARG
    assert L.lip_add_host(None, None, None, 1) == L.LIP_ERR_ARG
    assert L.lip_add_async(None, None, None, 1) == L.LIP_ERR_ARG
    assert L.lip_add_host_async(None, None, None, 1) == L.LIP_ERR_ARG
    assert L.lip_set_tc_window(None, 0) == L.LIP_ERR_ARG
    assert L.lip_set_estimate_full(None, 1) == L.LIP_ERR_ARG
    assert L.lip_set_estimate_full(None, 3) == L.LIP_ERR_ARG
    assert L._lib.lip_last_estimate_work(None, None) == L.LIP_ERR_ARG
    assert L._lib.lip_last_scan_stats(None, None) == L.LIP_ERR_ARG
    assert L.lip_eval_host_async(None, None, 0, None, None, None, None, None) == L.LIP_ERR_ARG
    assert L.lip_clear(None) == L.LIP_ERR_ARG
    assert L.lip_set_M(None, 1.0) == L.LIP_ERR_ARG
    assert L.lip_estimate_M(None)[0] == L.LIP_ERR_ARG
    assert L.lip_estimate_M_async(None) == L.LIP_ERR_ARG
    assert L.lip_estimate_M_result(None)[0] == L.LIP_ERR_ARG
    assert L.lip_backward(None, None, 0, None, None, None, None, None, None) == L.LIP_ERR_ARG
    assert L.lip_backward(None, None, 0, None, None, None, None, None, None, 1) == L.LIP_ERR_ARG
    assert L.lip_eval_batched(None) == L.LIP_ERR_ARG
    assert L.lip_autotune(None, None, 1)[0] == L.LIP_ERR_ARG
    assert isinstance(L.lip_last_error_detail(), str)
    assert L.lip_check(None) == L.LIP_ERR_ARG
    assert L.lip_set_tuning(None, 0, 0, 0) == L.LIP_ERR_ARG
    assert L.lip_get_tuning(None)[0] == L.LIP_ERR_ARG
    assert L.lip_set_timing_events(None, None, None) == L.LIP_ERR_ARG
    assert L.lip_size(None) == -1
    L.lip_free(None)
    assert L.lip_kernel_launches() >= 0


def test_reserve_argument_errors():
    p, keep = L.make_params()
    assert L.lip_reserve(0, 2, 1.0, p)[0] == L.LIP_ERR_ARG
    assert L.lip_reserve(10, 0, 1.0, p)[0] == L.LIP_ERR_ARG
    assert L.lip_reserve(10, 2, -2.0, p)[0] == L.LIP_ERR_ARG


def test_valid_call_without_device_reports_no_device():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    X, y = _arr(8, 2), _arr(8)
    p, keep = L.make_params()
    s, h = L.lip_fit(X.ctypes.data, y.ctypes.data, 8, 2, 1.0, p)
    assert s in (L.LIP_ERR_NO_DEVICE, L.LIP_ERR_CUDA) and not h.value


def test_batch_argument_errors():
    arr = (L.lip_batch_set * 2)()
    ok = L.lip_batch_set(1, 1, 10, 3, L.LIP_L2, 1.0, None, None, 1, 5, None, None, None, None, None, 0, 0)
    arr[0] = ok
    arr[1] = L.lip_batch_set(1, 1, 10, 33, L.LIP_L2, 1.0, None, None, 1, 5, None, None, None, None, None, 0, 0)
    s, h = L.lip_batch_create(arr)
    assert s == L.LIP_ERR_ARG and "set 1" in L.last_error() and not h.value
    arr[1] = L.lip_batch_set(1, 1, 10, 3, L.LIP_L2, -1.0, None, None, 1, 5, None, None, None, None, None, 0, 0)
    assert L.lip_batch_create(arr)[0] == L.LIP_ERR_ARG
    arr[1] = L.lip_batch_set(1, 1, 10, 3, L.LIP_L2, 1.0, None, None, None, 5, None, None, None, None, None, 0, 0)
    assert L.lip_batch_create(arr)[0] == L.LIP_ERR_ARG          # queries but Q is NULL
    arr[1] = L.lip_batch_set(1, 1, 10, 3, L.LIP_L2, 1.0, None, None, 1, 5, None, None, None, None, None, 12, 0)
    assert L.lip_batch_create(arr)[0] == L.LIP_ERR_ARG          # tile size
    opt = L.lip_batch_options(7, 0, 0, 0)
    arr[1] = ok
    assert L.lip_batch_create(arr, opt)[0] == L.LIP_ERR_ARG
    assert L.lip_batch_eval(None) == L.LIP_ERR_ARG
    assert L.lip_batch_info(None)[0] == L.LIP_ERR_ARG
    assert L.lip_batch_check(None) == L.LIP_ERR_ARG
    L.lip_batch_free(None)


def test_tensor_core_precision_rules():
    X, y = _arr(8, 2), _arr(8)
    for norm, prec, mon in [(L.LIP_L1, L.LIP_TC_TF32, None), (L.LIP_L2, L.LIP_TC_TF32, [1, 0]),
                            (L.LIP_L1, L.LIP_TC_BF16, None), (L.LIP_L2, L.LIP_TC_BF16, [0, -1]),
                            (L.LIP_LINF, L.LIP_TC_FP16, None), (L.LIP_L2, L.LIP_TC_FP16, [1, 1])]:
        p, keep = L.make_params(norm, prec, mon, None)
        s, h = L.lip_fit(X.ctypes.data, y.ctypes.data, 8, 2, 1.0, p)
        assert s == L.LIP_ERR_UNSUPPORTED and not h.value, L.last_error()


def test_eval_k_argument_errors():
    wk = np.array([0.5, 0.5])
    assert L.lip_eval_k(None, None, 1, 2, wk.ctypes.data, None, None, None, None, None) == L.LIP_ERR_ARG


def test_local_lipschitz_argument_errors():
    assert L.lip_local_fit(None, 8, 100, 1) == L.LIP_ERR_ARG
    kn = np.array([0.5, 1.0])
    assert L.lip_local_fit_knots(None, kn.ctypes.data, 2) == L.LIP_ERR_ARG
    assert L.lip_local_knots(None)[0] == L.LIP_ERR_ARG
    assert L.lip_local_table(None, None, None, None) == L.LIP_ERR_ARG
    assert L.lip_local_stats(None)[0] == L.LIP_ERR_ARG
    assert L.lip_eval_local(None, None, 1, None, None, None, None, None) == L.LIP_ERR_ARG
    assert L.LIP_LOCAL_KNOTS_MAX == 31 and L.LIP_LOCAL_SAMPLE_MAX == 1 << 20
    assert L.status_string(L.LIP_ERR_STATE) == "call out of order"


def test_smoothing_argument_errors():
    eps = np.zeros(4)
    assert L.lip_smooth_objective(None, 1.0, 10.0, eps.ctypes.data, None)[0] == L.LIP_ERR_ARG
    assert L.lip_smooth(None, 1.0, 10.0, 10, 5, 1e-6, None)[0] == L.LIP_ERR_ARG
