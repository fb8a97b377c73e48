"""FP64 CPU oracle for optimal Lipschitz interpolation (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package.  It is the checker the CUDA library is compared against:
it shares no code with the library (different language, no common header or
table) and never calls it.  ``build()`` compiles ``lipfit_oracle.c`` with gcc into
``oracle/_build/``; the functions below are numpy front ends to it.

Passages followed (all in the C file's header): Sec. 3 Eq. (upperlower) and
Eq. (eq:g) for the envelopes and midpoint, Sec. 4.1 Eq. (distmon) for the
monotone distance, Sec. 5 for the Lipschitz-constant estimate and the k > 1
neighbours, Sec. 4.3 for the local Lipschitz constants, Sec. 4.4 Eq. (optim) for the
penalty smoothing, and Table 1
("differentiable almost everywhere") for the gradient.

``Oracle(path)`` binds any build of the same C source; the tests use it to check
that deliberately broken copies of the source fail the pins.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "lipfit_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liblipfit_oracle.so")

NORM_L1, NORM_L2, NORM_LINF = 1, 2, 3


def compile_source(src: str, out: str) -> str:
    """gcc -O2, no fast-math, no FMA contraction: plain IEEE double arithmetic."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fno-fast-math", "-pthread", src, "-o", tmp, "-lm"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(SOURCE):
        compile_source(SOURCE, _LIB_PATH)
    return _LIB_PATH


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _mon(mon, d):
    if mon is None:
        return None
    m = np.ascontiguousarray(mon, dtype=np.int8)
    assert m.shape == (d,)
    return m


def default_threads() -> int:
    return os.cpu_count() or 1


class EvalResult(dict):
    """hi, lo, g, idx_up, idx_lo, gap_up, gap_lo (all numpy arrays)."""

    def __getattr__(self, k):
        return self[k]


class Oracle:
    """numpy front end to one compiled copy of the oracle's C source."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.oracle_eval.argtypes = [P, P, i64, i32, f64, i32, P, P, P, i64, P, P, P, P, P, P, P, i32]
        lib.oracle_estimate_M.argtypes = [P, P, i64, i32, i32, P, P, P, P, i32]
        lib.oracle_estimate_M_rows.argtypes = [P, P, i64, i32, i32, P, i64, i64, P, P, P]
        lib.oracle_grad.argtypes = [P, P, i64, i32, f64, i32, P, P, P, i64, P, P, P, P, P, P]
        lib.oracle_eval_k.argtypes = [P, P, i64, i32, f64, i32, P, P, P, i64, i32, P, P, P, P, P, P, i32]
        u64 = ctypes.c_uint64
        lib.oracle_splitmix64.argtypes = [u64, u64]
        lib.oracle_splitmix64.restype = u64
        lib.oracle_local_knots.argtypes = [P, i64, i32, i32, P, P, u64, i64, i32, P, P, P]
        lib.oracle_local_table.argtypes = [P, P, i64, i32, i32, P, P, P, i32, P, P, P, i32]
        lib.oracle_local_table_rows.argtypes = [P, P, i64, i32, i32, P, P, P, i32, P, i64, P, P, P, i32]
        lib.oracle_eval_local.argtypes = [P, P, i64, i32, i32, P, P, P, i32, P, P, P, P, i64, f64, f64, P, P, P, P, P,
                                          P, P, P, P, i32]
        lib.oracle_local_terms.argtypes = [P, P, i64, i32, i32, P, P, P, i32, P, P, P, P, i64, P, i32, f64, P]
        lib.oracle_eval_local_k.argtypes = [P, P, i64, i32, i32, P, P, P, i32, P, P, P, P, i64, i32, P, P, P, P, P, P,
                                            i32]
        lib.oracle_eval_local_k.restype = ctypes.c_int
        lib.oracle_smooth_objective.argtypes = [P, P, i64, i32, f64, i32, P, P, f64, P, P, P, P, P]
        lib.oracle_smooth.argtypes = [P, P, i64, i32, f64, i32, P, P, f64, i32, i32, f64, P, P, P]
        lib.oracle_smooth_objective.restype = ctypes.c_int
        lib.oracle_smooth_grad_rows.argtypes = [P, P, i64, i32, f64, i32, P, P, f64, P, P, i64, P]
        lib.oracle_smooth_grad_rows.restype = ctypes.c_int
        lib.oracle_smooth.restype = ctypes.c_int
        for fn in (lib.oracle_eval, lib.oracle_estimate_M, lib.oracle_estimate_M_rows, lib.oracle_grad,
                   lib.oracle_eval_k, lib.oracle_local_knots, lib.oracle_local_table, lib.oracle_local_table_rows,
                   lib.oracle_eval_local,
                   lib.oracle_local_terms):
            fn.restype = ctypes.c_int
        self.lib = lib

    def evaluate(self, X, y, Q, M: float, norm: int = NORM_L2, mon=None, w=None,
                 nthreads: Optional[int] = None) -> EvalResult:
        """H_up, H_lo, g and the argmin/argmax data indices for each query row of Q."""
        X, y, Q, w = _f64(X), _f64(y), _f64(Q), _f64(w)
        N, d = X.shape
        nq = Q.shape[0]
        mon = _mon(mon, d)
        out = {k: np.empty(nq) for k in ("hi", "lo", "g", "gap_up", "gap_lo")}
        iu = np.empty(nq, np.int64)
        il = np.empty(nq, np.int64)
        rc = self.lib.oracle_eval(_ptr(X), _ptr(y), N, d, float(M), int(norm), _ptr(mon), _ptr(w),
                                  _ptr(Q), nq, _ptr(out["hi"]), _ptr(out["lo"]), _ptr(out["g"]),
                                  _ptr(iu), _ptr(il), _ptr(out["gap_up"]), _ptr(out["gap_lo"]),
                                  nthreads or default_threads())
        if rc != 0:
            raise ValueError("oracle_eval: bad arguments")
        return EvalResult(idx_up=iu, idx_lo=il, **out)

    def evaluate_k(self, X, y, Q, M: float, k: int, wk, norm: int = NORM_L2, mon=None, w=None,
                   nthreads: Optional[int] = None) -> EvalResult:
        """k > 1 neighbours: weighted sums of the k best upper / lower bounds (Sec. 5)."""
        X, y, Q, w = _f64(X), _f64(y), _f64(Q), _f64(w)
        wk = _f64(wk)
        N, d = X.shape
        nq = Q.shape[0]
        mon = _mon(mon, d)
        out = {key: np.empty(nq) for key in ("hi", "lo", "g")}
        iu = np.empty((nq, k), np.int64)
        il = np.empty((nq, k), np.int64)
        rc = self.lib.oracle_eval_k(_ptr(X), _ptr(y), N, d, float(M), int(norm), _ptr(mon), _ptr(w), _ptr(Q), nq,
                                    int(k), _ptr(wk), _ptr(out["hi"]), _ptr(out["lo"]), _ptr(out["g"]), _ptr(iu),
                                    _ptr(il), nthreads or default_threads())
        if rc != 0:
            raise ValueError("oracle_eval_k: bad arguments")
        return EvalResult(idx_up=iu, idx_lo=il, **out)

    def estimate_M(self, X, y, norm: int = NORM_L2, w=None, nthreads: Optional[int] = None):
        """(M_est, i, j): max over i<j of |y_i-y_j| / dist(x_i,x_j), lowest (i,j) on ties."""
        X, y, w = _f64(X), _f64(y), _f64(w)
        N, d = X.shape
        M, i, j = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
        rc = self.lib.oracle_estimate_M(_ptr(X), _ptr(y), N, d, int(norm), _ptr(w), ctypes.byref(M),
                                        ctypes.byref(i), ctypes.byref(j), nthreads or default_threads())
        if rc != 0:
            raise ValueError("oracle_estimate_M: bad arguments")
        return M.value, i.value, j.value

    def estimate_M_rows(self, X, y, i0: int, i1: int, norm: int = NORM_L2, w=None):
        """Single-threaded M_est restricted to rows i in [i0, i1) (pairs i<j)."""
        X, y, w = _f64(X), _f64(y), _f64(w)
        N, d = X.shape
        M, i, j = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
        self.lib.oracle_estimate_M_rows(_ptr(X), _ptr(y), N, d, int(norm), _ptr(w), int(i0), int(i1),
                                        ctypes.byref(M), ctypes.byref(i), ctypes.byref(j))
        return M.value, i.value, j.value

    def gradient(self, X, y, Q, M: float, idx_up, idx_lo, gbar=None, norm: int = NORM_L2,
                 mon=None, w=None):
        """(grad_Q [nq,d], grad_y [N], grad_M) of sum_q gbar_q g(q) at the given argmin/argmax."""
        X, y, Q, w = _f64(X), _f64(y), _f64(Q), _f64(w)
        N, d = X.shape
        nq = Q.shape[0]
        mon = _mon(mon, d)
        iu = np.ascontiguousarray(idx_up, np.int64)
        il = np.ascontiguousarray(idx_lo, np.int64)
        gb = _f64(gbar) if gbar is not None else None
        gQ = np.zeros((nq, d))
        gy = np.zeros(N)
        gM = ctypes.c_double()
        rc = self.lib.oracle_grad(_ptr(X), _ptr(y), N, d, float(M), int(norm), _ptr(mon), _ptr(w),
                                  _ptr(Q), nq, _ptr(iu), _ptr(il), _ptr(gb), _ptr(gQ), _ptr(gy),
                                  ctypes.byref(gM))
        if rc != 0:
            raise ValueError("oracle_grad: bad arguments")
        return gQ, gy, gM.value

    # ------------------------------------------------------- local Lipschitz (Sec. 4.3)
    def splitmix64(self, seed: int, c: int) -> int:
        """Output number c (0-based) of SplitMix64 seeded with `seed`."""
        return int(self.lib.oracle_splitmix64(seed & (2**64 - 1), c & (2**64 - 1)))

    def local_knots(self, X, m: int, S: int, seed: int, norm: int = NORM_L2, w=None, mon=None):
        """(knots, pairs [S,2], dist [S]): quantile knots from S sampled pairs (with monotone
        coordinates, the upper-side distance dist_up(x^a, x^b) of pair (a, b))."""
        X, w = _f64(X), _f64(w)
        N, d = X.shape
        mon = _mon(mon, d)
        knots = np.empty(max(m, 1))
        pairs = np.empty((S, 2), np.int64)
        dist = np.empty(S)
        n = self.lib.oracle_local_knots(_ptr(X), N, d, int(norm), _ptr(w), _ptr(mon), seed & (2**64 - 1), int(S), int(m),
                                        _ptr(knots), _ptr(pairs), _ptr(dist))
        if n < 0:
            raise ValueError("oracle_local_knots: bad arguments")
        return knots[:n].copy(), pairs, dist

    def local_table(self, X, y, knots, norm: int = NORM_L2, w=None, nthreads: Optional[int] = None, mon=None):
        """(d1 [N], F [N], Mtab [N, m+1]) for the given knots."""
        X, y, w = _f64(X), _f64(y), _f64(w)
        T = _f64(np.asarray(knots, np.float64).reshape(-1))
        N, d = X.shape
        mon = _mon(mon, d)
        m = T.shape[0]
        d1, F = np.empty(N), np.empty(N)
        Mtab = np.empty((N, m + 1))
        rc = self.lib.oracle_local_table(_ptr(X), _ptr(y), N, d, int(norm), _ptr(w), _ptr(mon), _ptr(T), m, _ptr(d1), _ptr(F),
                                         _ptr(Mtab), nthreads or default_threads())
        if rc != 0:
            raise ValueError("oracle_local_table: bad arguments")
        return d1, F, Mtab

    def local_table_rows(self, X, y, knots, rows, norm: int = NORM_L2, w=None, nthreads: Optional[int] = None,
                         mon=None):
        """(d1, F, Mtab) of the data rows[i] only (row i of each output)."""
        X, y, w = _f64(X), _f64(y), _f64(w)
        T = _f64(np.asarray(knots, np.float64).reshape(-1))
        rows = np.ascontiguousarray(rows, np.int64)
        N, d = X.shape
        mon = _mon(mon, d)
        m, n = T.shape[0], rows.shape[0]
        d1, F = np.empty(n), np.empty(n)
        Mtab = np.empty((n, m + 1))
        rc = self.lib.oracle_local_table_rows(_ptr(X), _ptr(y), N, d, int(norm), _ptr(w), _ptr(mon), _ptr(T), m,
                                              _ptr(rows), n,
                                              _ptr(d1), _ptr(F), _ptr(Mtab), nthreads or default_threads())
        if rc != 0:
            raise ValueError("oracle_local_table_rows: bad arguments")
        return d1, F, Mtab

    def evaluate_local(self, X, y, Q, knots, table, norm: int = NORM_L2, w=None, eta: float = 0.0,
                       tau: float = 0.0, nthreads: Optional[int] = None, mon=None) -> EvalResult:
        """Envelopes with M replaced by M_k(dist).  eta > 0 (a distance error) and tau >= 0
        (a bound-value error) add hi_plus / lo_minus, the envelopes with every constant at
        M_k(t + eta), and the amb_up / amb_lo flags: some datum that an evaluation with
        those errors could pick has an exact value more than tau from the envelope."""
        X, y, Q, w = _f64(X), _f64(y), _f64(Q), _f64(w)
        T = _f64(np.asarray(knots, np.float64).reshape(-1))
        d1, F, Mtab = (_f64(a) for a in table)
        N, d = X.shape
        nq = Q.shape[0]
        out = {k: np.empty(nq) for k in ("hi", "lo", "g")}
        iu, il = np.empty(nq, np.int64), np.empty(nq, np.int64)
        au, al = np.zeros(nq, np.int8), np.zeros(nq, np.int8)
        hp, lm = np.full(nq, np.nan), np.full(nq, np.nan)
        mon = _mon(mon, d)
        rc = self.lib.oracle_eval_local(_ptr(X), _ptr(y), N, d, int(norm), _ptr(w), _ptr(mon), _ptr(T), T.shape[0],
                                        _ptr(d1),
                                        _ptr(F), _ptr(Mtab), _ptr(Q), nq, float(eta), float(tau), _ptr(out["hi"]),
                                        _ptr(out["lo"]), _ptr(out["g"]), _ptr(iu), _ptr(il), _ptr(au), _ptr(al),
                                        _ptr(hp), _ptr(lm), nthreads or default_threads())
        if rc != 0:
            raise ValueError("oracle_eval_local: bad arguments")
        return EvalResult(idx_up=iu, idx_lo=il, amb_up=au.astype(bool), amb_lo=al.astype(bool), hi_plus=hp,
                          lo_minus=lm, **out)

    def evaluate_local_k(self, X, y, Q, knots, table, k: int, wk, norm: int = NORM_L2, w=None,
                         nthreads: Optional[int] = None, mon=None) -> EvalResult:
        """k > 1 neighbours with the local constants: weighted sums of the k best bounds."""
        X, y, Q, w, wk = _f64(X), _f64(y), _f64(Q), _f64(w), _f64(wk)
        T = _f64(np.asarray(knots, np.float64).reshape(-1))
        d1, F, Mtab = (_f64(a) for a in table)
        N, d = X.shape
        nq = Q.shape[0]
        out = {key: np.empty(nq) for key in ("hi", "lo", "g")}
        iu, il = np.empty((nq, k), np.int64), np.empty((nq, k), np.int64)
        mon = _mon(mon, d)
        rc = self.lib.oracle_eval_local_k(_ptr(X), _ptr(y), N, d, int(norm), _ptr(w), _ptr(mon), _ptr(T), T.shape[0],
                                          _ptr(d1),
                                          _ptr(F), _ptr(Mtab), _ptr(Q), nq, int(k), _ptr(wk), _ptr(out["hi"]),
                                          _ptr(out["lo"]), _ptr(out["g"]), _ptr(iu), _ptr(il),
                                          nthreads or default_threads())
        if rc != 0:
            raise ValueError("oracle_eval_local_k: bad arguments")
        return EvalResult(idx_up=iu, idx_lo=il, **out)

    def local_terms(self, X, y, Q, knots, table, idx, side: int, norm: int = NORM_L2, w=None, shift: float = 0.0,
                    mon=None):
        """y_k + M_k(t + shift) t (side +1) or y_k - M_k(t + shift) t (side -1) for k = idx[q],
        t = dist(q, x^k) (with monotone coordinates dist_up for side +1, dist_lo for -1); NaN
        where idx[q] is not a datum."""
        X, y, Q, w = _f64(X), _f64(y), _f64(Q), _f64(w)
        T = _f64(np.asarray(knots, np.float64).reshape(-1))
        d1, F, Mtab = (_f64(a) for a in table)
        N, d = X.shape
        nq = Q.shape[0]
        ix = np.ascontiguousarray(idx, np.int64)
        out = np.empty(nq)
        mon = _mon(mon, d)
        rc = self.lib.oracle_local_terms(_ptr(X), _ptr(y), N, d, int(norm), _ptr(w), _ptr(mon), _ptr(T), T.shape[0],
                                         _ptr(d1),
                                         _ptr(F), _ptr(Mtab), _ptr(Q), nq, _ptr(ix), int(side), float(shift),
                                         _ptr(out))
        if rc != 0:
            raise ValueError("oracle_local_terms: bad arguments")
        return out

    # ----------------------------------------------------- penalty smoothing (Sec. 4.4)
    def smooth_objective(self, X, y, eps, M: float, p: float, norm: int = NORM_L2, mon=None, w=None):
        """(Phi, grad [N], S1, S2) of Eq. (optim) at eps; S1 and S2 are its two penalty sums."""
        X, y, w, eps = _f64(X), _f64(y), _f64(w), _f64(eps)
        N, d = X.shape
        mon = _mon(mon, d)
        f, s1, s2 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        g = np.empty(N)
        rc = self.lib.oracle_smooth_objective(_ptr(X), _ptr(y), N, d, float(M), int(norm), _ptr(mon), _ptr(w),
                                              float(p), _ptr(eps), ctypes.byref(f), _ptr(g), ctypes.byref(s1),
                                              ctypes.byref(s2))
        if rc != 0:
            raise ValueError("oracle_smooth_objective: bad arguments")
        return f.value, g, s1.value, s2.value

    def smooth_grad_rows(self, X, y, eps, rows, M: float, p: float, norm: int = NORM_L2, mon=None, w=None):
        """dPhi/deps_j for j in rows (O(N) per row)."""
        X, y, w, eps = _f64(X), _f64(y), _f64(w), _f64(eps)
        N, d = X.shape
        mon = _mon(mon, d)
        rows = np.ascontiguousarray(rows, np.int64)
        out = np.empty(rows.shape[0])
        rc = self.lib.oracle_smooth_grad_rows(_ptr(X), _ptr(y), N, d, float(M), int(norm), _ptr(mon), _ptr(w),
                                              float(p), _ptr(eps), _ptr(rows), rows.shape[0], _ptr(out))
        if rc != 0:
            raise ValueError("oracle_smooth_grad_rows: bad arguments")
        return out

    def smooth(self, X, y, M: float, p: float, norm: int = NORM_L2, mon=None, w=None, max_iter: int = 500,
               hist: int = 10, gtol: float = 1e-10):
        """(eps [N], Phi, iterations): the L-BFGS minimiser of Eq. (optim) from eps = 0."""
        X, y, w = _f64(X), _f64(y), _f64(w)
        N, d = X.shape
        mon = _mon(mon, d)
        eps = np.empty(N)
        f, it = ctypes.c_double(), ctypes.c_int()
        rc = self.lib.oracle_smooth(_ptr(X), _ptr(y), N, d, float(M), int(norm), _ptr(mon), _ptr(w), float(p),
                                    int(max_iter), int(hist), float(gtol), _ptr(eps), ctypes.byref(f),
                                    ctypes.byref(it))
        if rc != 0:
            raise ValueError("oracle_smooth: bad arguments")
        return eps, f.value, it.value


_default: Optional[Oracle] = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle(build())
    return _default


def evaluate(*a, **k) -> EvalResult:
    return default().evaluate(*a, **k)


def estimate_M(*a, **k):
    return default().estimate_M(*a, **k)


def evaluate_k(*a, **k):
    return default().evaluate_k(*a, **k)


def estimate_M_rows(*a, **k):
    return default().estimate_M_rows(*a, **k)


def gradient(*a, **k):
    return default().gradient(*a, **k)


def splitmix64(*a, **k):
    return default().splitmix64(*a, **k)


def local_knots(*a, **k):
    return default().local_knots(*a, **k)


def local_table(*a, **k):
    return default().local_table(*a, **k)


def evaluate_local(*a, **k):
    return default().evaluate_local(*a, **k)


def local_terms(*a, **k):
    return default().local_terms(*a, **k)


def local_table_rows(*a, **k):
    return default().local_table_rows(*a, **k)


def smooth_objective(*a, **k):
    return default().smooth_objective(*a, **k)


def smooth(*a, **k):
    return default().smooth(*a, **k)


def smooth_grad_rows(*a, **k):
    return default().smooth_grad_rows(*a, **k)


def evaluate_local_k(*a, **k):
    return default().evaluate_local_k(*a, **k)
