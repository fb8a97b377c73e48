"""The multi-GPU exchange steps with 2 and 3 gloo ranks on the CPU.

The per-rank steps run through host-side stand-ins built on the FP64 oracle (each rank's
slice of the data, its extrema packed into keys as the library packs them); the exchange
code under test is the package's own (``paper_2606_04670_b300.shard``): the all-reduce of
packed keys and of the owners' exact values for data-sharded evaluation, the gather of
query-sharded outputs, and the block-cyclic estimate.  Each merged result is compared with
the oracle on the full data, element by element."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2606_04670_b300 import shard as S
from paper_2606_04670_b300 import workloads as W

TILE = 512          # the estimate's tile of points (tile pairs are the block-cyclic unit)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _ord32(v):
    """Order-preserving unsigned 32-bit image of float32 values (sign flipped for
    positives, all bits flipped for negatives)."""
    u = np.asarray(v, np.float32).view(np.uint32).astype(np.int64)
    return np.where(u & 0x80000000, (~u) & 0xFFFFFFFF, u | 0x80000000)


def _pack(v, idx):
    return (_ord32(v) << 31) | np.asarray(idx, np.int64)


class OracleShard:
    """The per-rank steps on the host: this rank's data X[base:base+n] evaluated by the
    oracle, keys from the FP32 rounding of its extrema, FP64 re-evaluation of the winners
    this rank holds."""

    def __init__(self, o, p, base, end):
        self.o, self.p, self.base = o, p, base
        self.X, self.y = p.X[base:end], p.y[base:end]

    def scan(self, Q):
        n = len(self.y)
        nq = len(Q)
        if n == 0:
            k = torch.full((nq,), S.NO_KEY, dtype=torch.int64)
            return k, k.clone()
        r = self.o.evaluate(self.X, self.y, Q, self.p.M, self.p.norm, mon=self.p.mon, w=self.p.w)
        ku = _pack(r.hi.astype(np.float32), r.idx_up + self.base)
        kl = _pack(-r.lo.astype(np.float32), r.idx_lo + self.base)
        bad = ~np.isfinite(Q).all(1)
        ku[bad] = S.NO_KEY
        kl[bad] = S.NO_KEY
        return torch.as_tensor(ku), torch.as_tensor(kl)

    def _exact(self, Q, keys, side):
        out = np.full(len(Q), np.inf * side)
        for q, k in enumerate(keys.tolist()):
            if k == S.NO_KEY:
                continue
            j = (k & 0x7FFFFFFF) - self.base
            if 0 <= j < len(self.y):
                r = self.o.evaluate(self.X[j:j + 1], self.y[j:j + 1], Q[q:q + 1], self.p.M, self.p.norm,
                                    mon=self.p.mon, w=self.p.w)
                out[q] = r.hi[0] if side > 0 else r.lo[0]
        return torch.as_tensor(out)

    def reeval(self, Q, key_up, key_lo):
        return self._exact(Q, key_up, +1), self._exact(Q, key_lo, -1)

    def finish(self, key_up, key_lo, hi64, lo64):
        ku, kl = key_up.numpy(), key_lo.numpy()
        none = (ku == S.NO_KEY) | (kl == S.NO_KEY)
        hi = np.where(none, np.nan, hi64.numpy())
        lo = np.where(none, np.nan, lo64.numpy())
        return {"g": (0.5 * (hi + lo)).astype(np.float32), "hi": hi.astype(np.float32), "lo": lo.astype(np.float32),
                "idx_up": np.where(none, -1, ku & 0x7FFFFFFF), "idx_lo": np.where(none, -1, kl & 0x7FFFFFFF)}


class OracleEstimateShard:
    """lip_estimate_M_part on the host: the tile pairs (I, J >= I) with (I nb + J) mod nparts
    = part, each pair's ratio in FP64; the key is that ratio."""

    def __init__(self, p):
        self.p = p

    def estimate_part(self, part, nparts):
        from scipy.spatial.distance import cdist
        X = self.p.X.astype(np.float64) * (1.0 if self.p.w is None else np.asarray(self.p.w))
        y = self.p.y.astype(np.float64)
        N = len(y)
        nb = (N + TILE - 1) // TILE
        metric = {1: "cityblock", 2: "euclidean", 3: "chebyshev"}[self.p.norm]
        best = [0.0, -1.0, -1.0, -1.0]
        for I in range(nb):
            for J in range(I, nb):
                if (I * nb + J) % nparts != part:
                    continue
                a = np.arange(I * TILE, min(N, (I + 1) * TILE))
                b = np.arange(J * TILE, min(N, (J + 1) * TILE))
                D = cdist(X[a], X[b], metric)
                dy = np.abs(y[a][:, None] - y[b][None, :])
                with np.errstate(divide="ignore", invalid="ignore"):
                    R = dy / D
                ok = (a[:, None] < b[None, :]) & ~np.isnan(R)
                if not ok.any():
                    continue
                R = np.where(ok, R, -1.0)
                k = np.argmax(R)
                i, j = a[k // len(b)], b[k % len(b)]
                cand = [float(R.flat[k]), float(i), float(j), float(R.flat[k])]
                if S._better(cand, best):
                    best = cand
        return best


def _init(rank, world, port):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    return dist


def _worker(rank, world, port, out):
    import oracle
    dist = _init(rank, world, port)
    o = oracle.default()
    res = {}
    for case, p in enumerate(_problems()):
        # data-sharded evaluation; the last case gives rank 0 no data at all
        if case == 3:
            base, end = (0, 0) if rank == 0 else S.shard_range(p.N, rank - 1, world - 1)
        else:
            base, end = S.shard_range(p.N, rank, world)
        got = S.eval_data_sharded(OracleShard(o, p, base, end), p.Q)
        res[f"data{case}"] = {k: np.asarray(v) for k, v in got.items()}
        # query-sharded evaluation (all data on every rank), gathered on rank 0
        qb, qe = S.shard_range(p.nq, rank, world)
        r = o.evaluate(p.X, p.y, p.Q[qb:qe], p.M, p.norm, mon=p.mon, w=p.w)
        mine = {k: torch.as_tensor(np.asarray(r[k])) for k in ("g", "hi", "lo", "idx_up", "idx_lo")}
        counts = [S.shard_range(p.nq, q, world)[1] - S.shard_range(p.nq, q, world)[0] for q in range(world)]
        full = S.gather_outputs(mine, counts, dst=0)
        if rank == 0:
            res[f"query{case}"] = {k: v.numpy() for k, v in full.items()}
        else:
            assert full is None
        # the shared estimate
        res[f"est{case}"] = S.estimate_M_sharded(OracleEstimateShard(p))
    out[rank] = res
    dist.destroy_process_group()


def _problems():
    out = []
    for seed, (N, d, norm, masked, weighted) in enumerate([(1500, 3, 2, True, False), (1300, 2, 1, True, True),
                                                            (1100, 4, 3, False, True), (1800, 2, 2, False, False)]):
        p = W.random_problem(800 + seed, N, d, 60, norm=norm, masked=masked, weighted=weighted, decreasing=masked,
                             dtype=np.float32)
        if seed == 0:
            p.Q[7, 1] = np.nan                 # a non-finite query: NaN and -1 everywhere
        out.append(p)
    return out


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_exchange_matches_oracle(world, oracle_mod):
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    o = oracle_mod.default()
    for case, p in enumerate(_problems()):
        ref = o.evaluate(p.X, p.y, p.Q, p.M, p.norm, mon=p.mon, w=p.w)
        finite = np.isfinite(p.Q).all(1)
        scale = 1e-6 * (np.abs(p.y).max() + p.M)
        for r in range(world):
            got = res[r][f"data{case}"]
            for k in ("hi", "lo", "g"):
                assert np.all(np.isnan(got[k][~finite]))
                err = np.abs(got[k][finite].astype(np.float64) - ref[k][finite])
                assert err.max() <= scale, (world, case, r, k, err.max())
            for k, gk in (("idx_up", "gap_up"), ("idx_lo", "gap_lo")):
                assert np.all(got[k][~finite] == -1)
                clear = finite & (ref[gk] > scale)
                assert np.array_equal(got[k][clear], ref[k][clear]), (world, case, r, k)
            # every rank holds the same merged result
            for k in got:
                np.testing.assert_array_equal(got[k], res[0][f"data{case}"][k])
        q = res[0][f"query{case}"]
        for k in ("g", "hi", "lo", "idx_up", "idx_lo"):
            np.testing.assert_array_equal(q[k], np.asarray(ref[k]))
        M, i, j = o.estimate_M(p.X, p.y, p.norm, w=p.w)
        for r in range(world):
            Ms, is_, js = res[r][f"est{case}"]
            assert abs(Ms - M) <= 1e-12 * M and (is_, js) == (i, j), (world, case, r, Ms, M, is_, js, i, j)


def test_shard_range_covers_every_item_once():
    for n in (0, 1, 7, 1000, 10**6 + 3):
        for world in (1, 2, 3, 8):
            spans = [S.shard_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [e - b for b, e in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        S.shard_range(10, 2, 2)


def test_key_packing_orders_like_the_merge():
    """Smaller value first, then the lower index; negative, zero and infinite values; the
    no-candidate key above all."""
    v = np.array([-np.inf, -3.5, -1e-30, -0.0, 0.0, 1e-30, 2.0, 2.0, np.inf], np.float32)
    idx = np.array([5, 4, 9, 2, 1, 0, 3, 8, 0])
    k = _pack(v, idx)
    # listed in increasing (value, index) order; -0.0 and 0.0 compare equal as floats and
    # the packing puts -0.0 first
    assert list(np.argsort(k, kind="stable")) == list(range(len(v)))
    assert k.max() < S.NO_KEY and k.min() >= 0
