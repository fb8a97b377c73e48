"""Seeded synthetic workloads shaped like the paper's use cases.

This module only draws inputs: scattered data X (N x d), responses y = f(X) for a
test function f with a known Lipschitz bound M, query points Q, and the method's
parameters (norm, monotonicity vector, norm weights).  It contains none of the
method's arithmetic (no distances, no envelopes), so the FP64 oracle and the CUDA
path can both consume it without sharing code.

Every generator uses ``numpy.random.default_rng(seed)`` with
``seed = 20260604 * 10 + workload_id`` and independent child streams (``spawn``)
for the data, the queries and the parameters.

Workloads (all coordinates in [0,1]^d unless stated):

* ``plain_d2``      d=2, N=1000, Q=10000, y = sin(3x1)+cos(2x2)+0.5 x1 x2, M=4.5, L2.
* ``monotone_d4``   d=4, N=1e5, Q=1e6, y = sum_i a_i log(1+4x_i) + 0.3 sin(2 pi x3),
                    a_i ~ U(0.5,1.5), increasing in x1,x2 (mon=[1,1,0,0]); L1/L2/Linf.
* ``cluster_d16``   d=16, N=1e6, Q=1e6, 32-cluster Gaussian mixture (sigma 0.05,
                    clipped), y = ||x-c||_2 + 0.1 sum sin(5 x_i), c = 0.5, M = 3, L2.
* ``grad_d8``       d=8, N=2e5, Q=262144, y = sum_i w_i tanh(2x_i-1), w ~ U(0,1),
                    increasing in x1..x4, M = 2||w||_2, L2.
* ``batch_4096``    4096 independent sets, N log-uniform in [64,65536], d uniform in
                    {2..10}, Q log-uniform in [1e3,1e5], random masks (p=0.5), L1/L2
                    mixed, y = sum_i alpha_i softplus(beta_i (x_i - tau_i)).
* ``toy_d3``        the paper's toy example shape (Sec. 5): d=3, N=1000, Q=1000,
                    increasing in every coordinate.

The Lipschitz bounds are closed forms of sup ||grad f||_* in the dual norm of the
evaluation norm (L1 <-> Linf, L2 <-> L2), taken at the point where every partial
derivative is largest.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np

SEED_BASE = 20260604 * 10

NORM_L1, NORM_L2, NORM_LINF = 1, 2, 3
NORM_NAMES = {NORM_L1: "L1", NORM_L2: "L2", NORM_LINF: "Linf"}


@dataclasses.dataclass
class Problem:
    """One fitting problem: data, queries, and the method's parameters."""

    name: str
    X: np.ndarray              # [N, d] row-major
    y: np.ndarray              # [N]
    Q: np.ndarray              # [nq, d]
    M: float                   # Lipschitz constant for the evaluation norm
    norm: int                  # NORM_L1 / NORM_L2 / NORM_LINF
    mon: Optional[np.ndarray]  # int8 [d] in {-1,0,1} or None
    w: Optional[np.ndarray]    # float [d] > 0 (norm weights) or None
    f: Optional[object] = None  # callable: f(X float64 [n,d]) -> float64 [n]
    M_by_norm: Optional[Dict[int, float]] = None

    @property
    def N(self) -> int:
        return int(self.X.shape[0])

    @property
    def d(self) -> int:
        return int(self.X.shape[1])

    @property
    def nq(self) -> int:
        return int(self.Q.shape[0])

    def with_norm(self, norm: int) -> "Problem":
        M = self.M_by_norm[norm] if self.M_by_norm else self.M
        return dataclasses.replace(self, norm=norm, M=M)

    def sub_queries(self, n: int) -> "Problem":
        return dataclasses.replace(self, Q=self.Q[:n])


def _rngs(workload_id: int, n: int = 3):
    return np.random.default_rng(SEED_BASE + workload_id).spawn(n)


# --------------------------------------------------------------------------- f's

def f_plain_d2(X):
    X = np.asarray(X, np.float64)
    return np.sin(3 * X[:, 0]) + np.cos(2 * X[:, 1]) + 0.5 * X[:, 0] * X[:, 1]


def _f_monotone_d4(a):
    def f(X):
        X = np.asarray(X, np.float64)
        return (a[None, :] * np.log1p(4.0 * X)).sum(1) + 0.3 * np.sin(2 * math.pi * X[:, 2])
    return f


def _f_cluster_d16(X):
    X = np.asarray(X, np.float64)
    return np.linalg.norm(X - 0.5, axis=1) + 0.1 * np.sin(5.0 * X).sum(1)


def _f_grad_d8(w):
    def f(X):
        X = np.asarray(X, np.float64)
        return (w[None, :] * np.tanh(2.0 * X - 1.0)).sum(1)
    return f


def _softplus(z):
    return np.logaddexp(0.0, z)


def _f_softplus(alpha, beta, tau):
    def f(X):
        X = np.asarray(X, np.float64)
        return (alpha[None, :] * _softplus(beta[None, :] * (X - tau[None, :]))).sum(1)
    return f


def _f_toy_d3(X):
    X = np.asarray(X, np.float64)
    return X[:, 0] + X[:, 1] ** 2 + 0.5 * (1.0 - np.cos(X[:, 2]))


# --------------------------------------------------------------------- workloads

def _f_local_d4(X):
    X = np.asarray(X, np.float64)
    return np.tanh(10.0 * (X[:, 0] - 0.5)) + 0.2 * X[:, 1] + 0.1 * np.sin(3.0 * X[:, 2]) + 0.05 * X[:, 3]


def _as(x, dtype):
    return np.ascontiguousarray(x, dtype=dtype)


def plain_d2(dtype=np.float32, n_data=1000, n_query=10_000) -> Problem:
    """d=2 plain method, L2, M=4.5 (sup ||grad f||_2 <= sqrt(3.5^2+2.5^2) = 4.30)."""
    rx, rq, _ = _rngs(1)
    X = _as(rx.random((n_data, 2)), dtype)
    Q = _as(rq.random((n_query, 2)), dtype)
    y = _as(f_plain_d2(X), dtype)
    return Problem("plain_d2", X, y, Q, 4.5, NORM_L2, None, None, f_plain_d2)


def monotone_d4(norm=NORM_L2, n_data=100_000, n_query=1_000_000, dtype=np.float32, query_block=0) -> Problem:
    """query_block b > 0 draws another n_query queries from an independent stream (block b of
    a larger query set shared out over several GPUs); the data are the same."""
    rx, rq, rp = _rngs(2)
    if query_block > 0:
        rq = _rngs(2, 3 + query_block)[2 + query_block]
    a = rp.uniform(0.5, 1.5, size=4)
    X = _as(rx.random((n_data, 4)), dtype)
    Q = _as(rq.random((n_query, 4)), dtype)
    f = _f_monotone_d4(a)
    y = _as(f(X), dtype)
    s = 4.0 * a.copy()
    s[2] += 0.6 * math.pi                  # 0.3 * 2 pi * cos(0)
    Ms = {NORM_L1: float(s.max()), NORM_L2: float(np.linalg.norm(s)), NORM_LINF: float(s.sum())}
    mon = np.array([1, 1, 0, 0], np.int8)
    return Problem("monotone_d4", X, y, Q, Ms[norm], norm, mon, None, f, Ms)


def cluster_d16(n_data=1_000_000, n_query=1_000_000, dtype=np.float32) -> Problem:
    rx, rq, rp = _rngs(3)
    centres = rp.random((32, 16))

    def draw(r, n):
        lab = r.integers(0, 32, size=n)
        pts = centres[lab] + 0.05 * r.standard_normal((n, 16))
        return np.clip(pts, 0.0, 1.0)

    X = _as(draw(rx, n_data), dtype)
    Q = _as(draw(rq, n_query), dtype)
    y = _as(_f_cluster_d16(X), dtype)
    return Problem("cluster_d16", X, y, Q, 3.0, NORM_L2, None, None, _f_cluster_d16)


def grad_d8(n_data=200_000, n_query=262_144, dtype=np.float32) -> Problem:
    rx, rq, rp = _rngs(4)
    w = rp.random(8)
    X = _as(rx.random((n_data, 8)), dtype)
    Q = _as(rq.random((n_query, 8)), dtype)
    f = _f_grad_d8(w)
    y = _as(f(X), dtype)
    mon = np.array([1, 1, 1, 1, 0, 0, 0, 0], np.int8)
    return Problem("grad_d8", X, y, Q, float(2.0 * np.linalg.norm(w)), NORM_L2, mon, None, f)


def toy_d3(n_data=1000, n_query=1000, dtype=np.float32) -> Problem:
    rx, rq, _ = _rngs(6)
    X = _as(rx.random((n_data, 3)), dtype)
    Q = _as(rq.random((n_query, 3)), dtype)
    y = _as(_f_toy_d3(X), dtype)
    # grad = (1, 2 x2, 0.5 sin x3) <= (1, 2, 0.43) -> ||.||_2 <= 2.28
    return Problem("toy_d3", X, y, Q, 2.3, NORM_L2, np.ones(3, np.int8), None, _f_toy_d3)


def local_d4(n_data=100_000, n_query=1_000_000, dtype=np.float32) -> Problem:
    """A function whose slope differs across the domain (Sec. 4.3's motivation for local
    constants): a steep tanh step across x1 = 0.5 (slope up to 10) on gentle terms (slopes
    0.2, 0.3, 0.05).  L2, no monotonicity; grad norm <= sqrt(100 + 0.04 + 0.09 + 0.0025)."""
    rx, rq, _ = _rngs(7)
    X = _as(rx.random((n_data, 4)), dtype)
    Q = _as(rq.random((n_query, 4)), dtype)
    y = _as(_f_local_d4(X), dtype)
    return Problem("local_d4", X, y, Q, 10.01, NORM_L2, None, None, _f_local_d4)


SMOOTH_M = 3.5      # >= sup |grad f|_2 of smooth_d4's f (sqrt(pi^2 + 1 + 1 + 0.04) = 3.45)
SMOOTH_P = 100.0    # penalty weight p of Eq. (optim) used with it


def _f_smooth_d4(X):
    X = np.asarray(X, np.float64)
    return 0.5 * np.sin(2 * math.pi * X[:, 0]) + X[:, 1] + 0.5 * X[:, 2] ** 2 + 0.2 * X[:, 3]


def smooth_d4(n_data=100_000, n_query=10_000, noise=0.05, dtype=np.float32) -> Problem:
    """Noisy samples of a smooth function (Sec. 4.4's use: data that violate the Lipschitz
    condition only through noise): f plus N(0, noise^2), L2, no monotonicity."""
    rx, rq, rn = _rngs(8)
    X = _as(rx.random((n_data, 4)), dtype)
    Q = _as(rq.random((n_query, 4)), dtype)
    y = _as(_f_smooth_d4(X) + noise * rn.standard_normal(n_data), dtype)
    return Problem("smooth_d4", X, y, Q, SMOOTH_M, NORM_L2, None, None, _f_smooth_d4)


@dataclasses.dataclass
class BatchSet:
    """The sizes and parameters of one set of the batched workload (data drawn lazily)."""

    index: int
    N: int
    d: int
    nq: int
    norm: int
    mon: np.ndarray
    alpha: np.ndarray
    beta: np.ndarray
    tau: np.ndarray
    M: float
    seed: int


def batch_plan(n_sets=4096, n_min=64, n_max=65536, q_min=1000, q_max=100_000) -> List[BatchSet]:
    """Sizes and parameters of the batched workload, drawn from one parameter stream."""
    _, _, rp = _rngs(5)
    out = []
    for s in range(n_sets):
        N = int(round(math.exp(rp.uniform(math.log(n_min), math.log(n_max)))))
        d = int(rp.integers(2, 11))
        nq = int(round(math.exp(rp.uniform(math.log(q_min), math.log(q_max)))))
        mon = (rp.random(d) < 0.5).astype(np.int8)
        norm = NORM_L1 if rp.random() < 0.5 else NORM_L2
        beta = rp.uniform(1.0, 8.0, size=d)
        tau = rp.uniform(0.0, 1.0, size=d)
        alpha = np.where(mon == 1, rp.uniform(0.5, 1.5, size=d), rp.uniform(-1.5, 1.5, size=d))
        m = np.abs(alpha) * beta
        M = float(m.max() if norm == NORM_L1 else np.linalg.norm(m))
        out.append(BatchSet(s, N, d, nq, norm, mon, alpha, beta, tau, M, SEED_BASE + 5000 + s))
    return out


def batch_set_data(bs: BatchSet, dtype=np.float32, nq: Optional[int] = None):
    """X, y, Q of one batched set (each set has its own seed, so any subset can be drawn)."""
    rx, rq = np.random.default_rng(bs.seed).spawn(2)
    X = _as(rx.random((bs.N, bs.d)), dtype)
    Q = _as(rq.random((bs.nq if nq is None else min(nq, bs.nq), bs.d)), dtype)
    f = _f_softplus(bs.alpha, bs.beta, bs.tau)
    y = _as(f(X), dtype)
    return X, y, Q, f


def random_problem(seed, N, d, nq, norm=NORM_L2, masked=False, weighted=False,
                   decreasing=False, dtype=np.float32, M=None) -> Problem:
    """Small random problem for parity tests: a smooth test function with known M."""
    r = np.random.default_rng(SEED_BASE + 100 + seed)
    X = _as(r.random((N, d)), dtype)
    Q = _as(r.random((nq, d)), dtype)
    c = r.uniform(0.2, 1.0, size=d)
    mon = None
    if masked:
        mon = (r.random(d) < 0.5).astype(np.int8)
        if decreasing:
            mon = np.where(r.random(d) < 0.5, -mon, mon).astype(np.int8)
    sgn = np.ones(d) if mon is None else np.where(mon < 0, -1.0, 1.0)
    w = _as(r.uniform(0.5, 2.0, size=d), np.float64) if weighted else None

    def f(Z):
        Z = np.asarray(Z, np.float64)
        return (sgn * c * Z).sum(1) + 0.1 * np.sin(Z[:, 0])

    y = _as(f(X), dtype)
    g = np.abs(c)
    g[0] += 0.1                         # |d/dz0 of 0.1 sin z0| <= 0.1 < c_0: monotone kept
    if w is not None:
        g = g / w                       # |f(a)-f(b)| <= sum g_i |a_i-b_i| = sum (g_i/w_i) w_i|.|
    Ms = {NORM_L1: float(g.max()), NORM_L2: float(np.linalg.norm(g)), NORM_LINF: float(g.sum())}
    Mv = Ms[norm] if M is None else float(M)
    return Problem(f"random{seed}", X, y, Q, Mv, norm, mon, w, f, Ms)


WORKLOADS = {
    "plain_d2": plain_d2,
    "monotone_d4": monotone_d4,
    "cluster_d16": cluster_d16,
    "grad_d8": grad_d8,
    "toy_d3": toy_d3,
    "local_d4": local_d4,
    "smooth_d4": smooth_d4,
}
