// Exact scan with chunk bounds (lip_set_tuning variants 6 and 7): the same values and
// extrema as scan_exact_kernel, over the data in spatial order, skipping every 16-point
// chunk that provably cannot lower H_up nor raise H_lo of any query of a row.
//
// The data are laid out in the spatial order of their points (a Hilbert order), so a
// chunk's points are close together; each chunk carries its bounding box in the layout's
// coordinates (already scaled by M w, mirrored where decreasing) and the range of its
// values.  From a query q and the box, the kernel forms the smallest distance any point
// of the chunk can have on each side, with the same FP32 operations in the same order as
// the per-pair code (group_values): a per-coordinate difference of smaller magnitude
// (q minus the box's nearest face, or 0 inside), squared and accumulated exactly as a
// pair is.  IEEE rounding is monotone, so every pair's FP32 distance is at least the
// box's, and:
//   L1, Linf: every pair's FP32 upper value y + d is at least ylo + d_box (rounded), and
//     every lower value at most yhi - d_box, so the chunk is skipped for a query when
//     ylo + d_box >= mu and yhi - d_box <= ml (mu, ml the running extrema);
//   L2: the square root is sqrt.approx (relative error far below 2^-21), so the test is
//     taken on squares: the upper side is skipped when ylo >= mu or
//     s_box > (mu - ylo)^2 (1 + 2^-17) (and s_box >= FLT_MIN, so that the flush to zero of
//     sqrt.approx.ftz cannot apply), which gives y + sqrt~(s) >= mu for every pair; the
//     lower side mirrors it with (yhi - ml).
// A skipped chunk holds no value below mu (above ml), so it can neither change the
// running extrema nor the chunk where they were reached: the results are those of an
// unpruned scan over the same order.  A warp holds R rows of 32 consecutive queries of the
// spatial order (one query per lane and row); it evaluates a chunk for each row in which
// any query needs it (queries in spatial order make a row's needs coherent).
//
// Processing order: 64-group super-chunks (16 chunks, so the order is the same for every
// tile size), nearest first from the centroid of the block's queries (below); with too
// many super-chunks to sort, cyclically from the one whose box centre is nearest.  Among data with
// exactly equal FP32 values the earliest in this order wins, which can differ from the
// lowest index (the FP64 re-evaluation of the merge returns the chosen datum's exact
// value either way).
#pragma once

#include "launch.h"

namespace lip {

// True when the chunk with box (lo, hi, ylo, yhv) may lower mu or raise ml for query q.
template <int NORM, int C, int U>
__device__ __forceinline__ bool chunk_needed(const float2 (&q)[C + U], const float* lo, const float* hi, float ylo,
                                             float yhv, float mu, float ml) {
    constexpr int D = C + U;
    // per-coordinate differences of the box's nearest points, as the pair code forms them
    float t[D], tl[C > 0 ? C : 1];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const float qj = q[j].x;
        if (j < C) {
            t[j] = __fsub_rn(qj, hi[j]);            // the upper side's (q - x)_+ is smallest at x = hi
            tl[j] = __fsub_rn(qj, lo[j]);           // the lower side's (x - q)_+ is smallest at x = lo
        } else {
            t[j] = __fsub_rn(qj, fminf(fmaxf(qj, lo[j]), hi[j]));   // 0 inside the box
        }
    }
    bool skip_u, skip_l;
    if constexpr (NORM == LIP_L2) {
        float s0 = 0.f;
        if constexpr (U > 0) {
            s0 = __fmul_rn(t[C], t[C]);
#pragma unroll
            for (int j = C + 1; j < D; ++j) s0 = __fmaf_rn(t[j], t[j], s0);
        }
        float su = s0, sl = s0;
        if constexpr (C > 0) {
#pragma unroll
            for (int j = 0; j < C; ++j) {
                const float p = fmaxf(t[j], 0.f), n = fminf(tl[j], 0.f);
                if (j == 0 && U == 0) { su = __fmul_rn(p, p); sl = __fmul_rn(n, n); }
                else { su = __fmaf_rn(p, p, su); sl = __fmaf_rn(n, n, sl); }
            }
        }
        constexpr float GROW = 1.00000762939453125f;     // 1 + 2^-17
        constexpr float TINY = 1.17549435e-38f;          // FLT_MIN
        const float du = __fsub_rn(mu, ylo), dl = __fsub_rn(yhv, ml);
        skip_u = du <= 0.f || su > fmaxf(__fmul_rn(__fmul_rn(du, du), GROW), TINY);
        skip_l = dl <= 0.f || sl > fmaxf(__fmul_rn(__fmul_rn(dl, dl), GROW), TINY);
    } else if constexpr (NORM == LIP_L1) {
        float acc = 0.f;
        if constexpr (U >= 2) {
            acc = __fadd_rn(fabsf(t[C]), fabsf(t[C + 1]));
#pragma unroll
            for (int j = C + 2; j < D; ++j) acc = __fadd_rn(acc, fabsf(t[j]));
        } else if constexpr (U == 1) {
            acc = fabsf(t[C]);
        }
        // the lower side's distance (the direct form of group_values): the unconstrained sum
        // plus the negative parts (x - q)_+, smallest at x = lo
        float accl = acc;
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const float p = fmaxf(t[j], 0.f), n = fmaxf(-tl[j], 0.f);
            acc = (j == 0 && U == 0) ? p : __fadd_rn(acc, p);
            accl = (j == 0 && U == 0) ? n : __fadd_rn(accl, n);
        }
        skip_u = __fadd_rn(ylo, acc) >= mu;
        skip_l = __fsub_rn(yhv, accl) <= ml;
    } else {
        float uu = 0.f;
#pragma unroll
        for (int j = C; j < D; ++j) uu = fmaxf(uu, fabsf(t[j]));
        float du = uu, dl = uu;
#pragma unroll
        for (int j = 0; j < C; ++j) {
            du = fmaxf(du, t[j]);
            dl = fmaxf(dl, -tl[j]);
        }
        skip_u = __fadd_rn(ylo, du) >= mu;
        skip_l = __fsub_rn(yhv, dl) <= ml;
    }
    return !(skip_u && skip_l);
}

// True when the record (lo, hi, ylo, yhv) may lower mu_max or raise ml_min for some query
// of the box [qlo, qhi] (the warp's queries).  The per-coordinate differences are bounded
// for every query of the box at once: q - x >= qlo - hi and x - q >= lo - qhi, rounded the
// same way, so each magnitude the pair code forms is at least the one used here; the
// accumulation then mirrors chunk_needed, and with mu_max (ml_min) the loosest running
// bound of the warp a record that fails here fails chunk_needed for every query.
template <int NORM, int C, int U>
__device__ __forceinline__ bool box_needed(const float* qlo, const float* qhi, const float* lo, const float* hi,
                                           float ylo, float yhv, float mu_max, float ml_min) {
    constexpr int D = C + U;
    float a[D], b[D];                  // a: lower bound of q - x; b: lower bound of x - q
#pragma unroll
    for (int j = 0; j < D; ++j) {
        a[j] = __fsub_rn(qlo[j], hi[j]);
        b[j] = __fsub_rn(lo[j], qhi[j]);
    }
    bool skip_u, skip_l;
    if constexpr (NORM == LIP_L2) {
        float s0 = 0.f;
        if constexpr (U > 0) {
            const float g = fmaxf(fmaxf(a[C], b[C]), 0.f);
            s0 = __fmul_rn(g, g);
#pragma unroll
            for (int j = C + 1; j < D; ++j) {
                const float gj = fmaxf(fmaxf(a[j], b[j]), 0.f);
                s0 = __fmaf_rn(gj, gj, s0);
            }
        }
        float su = s0, sl = s0;
        if constexpr (C > 0) {
#pragma unroll
            for (int j = 0; j < C; ++j) {
                const float p = fmaxf(a[j], 0.f), n = fmaxf(b[j], 0.f);
                if (j == 0 && U == 0) { su = __fmul_rn(p, p); sl = __fmul_rn(n, n); }
                else { su = __fmaf_rn(p, p, su); sl = __fmaf_rn(n, n, sl); }
            }
        }
        constexpr float GROW = 1.00000762939453125f;     // 1 + 2^-17
        constexpr float TINY = 1.17549435e-38f;          // FLT_MIN
        const float du = __fsub_rn(mu_max, ylo), dl = __fsub_rn(yhv, ml_min);
        skip_u = du <= 0.f || su > fmaxf(__fmul_rn(__fmul_rn(du, du), GROW), TINY);
        skip_l = dl <= 0.f || sl > fmaxf(__fmul_rn(__fmul_rn(dl, dl), GROW), TINY);
    } else if constexpr (NORM == LIP_L1) {
        float acc = 0.f;
        if constexpr (U >= 2) {
            acc = __fadd_rn(fmaxf(fmaxf(a[C], b[C]), 0.f), fmaxf(fmaxf(a[C + 1], b[C + 1]), 0.f));
#pragma unroll
            for (int j = C + 2; j < D; ++j) acc = __fadd_rn(acc, fmaxf(fmaxf(a[j], b[j]), 0.f));
        } else if constexpr (U == 1) {
            acc = fmaxf(fmaxf(a[C], b[C]), 0.f);
        }
        float accl = acc;
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const float p = fmaxf(a[j], 0.f), n = fmaxf(b[j], 0.f);
            acc = (j == 0 && U == 0) ? p : __fadd_rn(acc, p);
            accl = (j == 0 && U == 0) ? n : __fadd_rn(accl, n);
        }
        skip_u = __fadd_rn(ylo, acc) >= mu_max;
        skip_l = __fsub_rn(yhv, accl) <= ml_min;
    } else {
        float uu = 0.f;
#pragma unroll
        for (int j = C; j < D; ++j) uu = fmaxf(uu, fmaxf(a[j], b[j]));
        float du = uu, dl = uu;
#pragma unroll
        for (int j = 0; j < C; ++j) {
            du = fmaxf(du, a[j]);
            dl = fmaxf(dl, b[j]);
        }
        skip_u = __fadd_rn(ylo, du) >= mu_max;
        skip_l = __fsub_rn(yhv, dl) <= ml_min;
    }
    return !(skip_u && skip_l);
}

constexpr int PRUNED_LEAD = 2;     // super-chunks streamed before the first window
constexpr int PRUNED_STAGES = 6;   // the pruned scan's ring of tiles
constexpr int PRUNED_WIN = 256;    // super-chunks per window
constexpr int PRUNED_SORT = 1024;  // most super-chunks put in nearest-first order per block

template <int NORM, int C, int U, int R>
__global__ void __launch_bounds__(SCAN_THREADS) scan_pruned_kernel(const PrunedParams PP) {
    using S = ExactShape<NORM, C, U, true>;        // the direct lower distance, no aux channel
    constexpr int D = S::D;
    constexpr int NCH = S::NCH;
    constexpr int NB4 = pruned_box_f4(D);
    constexpr int NW = SCAN_THREADS / 32;
    // PRUNED_STAGES * tile_groups * NCH data, then PRUNED_STAGES * RECS chunk records
    constexpr int RECS = TILE_GROUPS_MAX / PRUNED_CG;
    extern __shared__ __align__(128) float4 tiles[];
    __shared__ __align__(8) uint64_t bars[PRUNED_STAGES];
    __shared__ int fin[PRUNED_STAGES];           // warps done with the stage's current tile
    __shared__ int last_issued[PRUNED_STAGES];   // ring step of the stage's last copy, -1 none
    __shared__ float red_c[NW][D + 1];
    __shared__ float red_d[NW];
    __shared__ int red_k[NW];
    __shared__ int start_chunk;
    const ScanParams& P = PP.S;
    const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
    const int tg = P.tile_groups;
    const uint32_t tile_bytes = (uint32_t)tg * NCH * 16u;
    const float4* hot = static_cast<const float4*>(P.hot);
    const float* Q = static_cast<const float*>(P.Q);

    // the block's queries: a warp holds 32 R consecutive positions of the spatial order,
    // row r the 32 of them at warp * 32 R + 32 r (lane l: position qblock * 128 R +
    // warp * 32 R + 32 r + l), so a row's queries are neighbours and its decisions agree
    float2 qq[R][D];
    float sq[R];
    int64_t qidx[R];
    bool live[R];
    float csum[D + 1];
#pragma unroll
    for (int j = 0; j <= D; ++j) csum[j] = 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t pos = (int64_t)blockIdx.x * (SCAN_THREADS * R) + (int64_t)warp * 32 * R + 32 * r + lane;
        qidx[r] = pos < P.nq ? (int64_t)PP.qperm[pos] : -1;
        float s = 0.f;
        bool fin = qidx[r] >= 0;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            float v = 0.f;
            if (qidx[r] >= 0) v = (float)(P.scale[j] * (double)__ldg(Q + qidx[r] * P.d + P.perm[j]));
            qq[r][j] = make_float2(v, v);
            fin = fin && isfinite(v);
            if (j < C) s = s + v;
        }
        sq[r] = s;
        live[r] = fin;
        if (fin) {
#pragma unroll
            for (int j = 0; j < D; ++j) csum[j] += qq[r][j].x;
            csum[D] += 1.f;
        }
    }
    // the warp's query box (its finite queries), for the tests of whole records
    float qlo[D], qhi[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        float a = __int_as_float(0x7f800000), b = -__int_as_float(0x7f800000);
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (live[r]) {
                a = fminf(a, qq[r][j].x);
                b = fmaxf(b, qq[r][j].x);
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a = fminf(a, __shfl_xor_sync(0xffffffffu, a, o));
            b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, o));
        }
        qlo[j] = a;
        qhi[j] = b;
    }
    bool any_live = false;
#pragma unroll
    for (int r = 0; r < R; ++r) any_live = any_live || live[r];
    const bool wlive = __any_sync(0xffffffffu, any_live);
    // the start chunk: the box centre nearest the centroid of the block's finite queries
#pragma unroll
    for (int j = 0; j <= D; ++j)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) csum[j] += __shfl_xor_sync(0xffffffffu, csum[j], o);
    if (lane == 0)
#pragma unroll
        for (int j = 0; j <= D; ++j) red_c[warp][j] = csum[j];
    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < PRUNED_STAGES; ++s) {
            mbar_init(&bars[s], 1);
            fin[s] = 0;
            last_issued[s] = -1;
        }
        fence_mbar_init();
    }
    __syncthreads();
    float cen[D];
    float cnt = 0.f;
#pragma unroll
    for (int w = 0; w < NW; ++w) cnt += red_c[w][D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        float a = 0.f;
#pragma unroll
        for (int w = 0; w < NW; ++w) a += red_c[w][j];
        cen[j] = cnt > 0.f ? a / cnt : 0.f;
    }
    float bd = __int_as_float(0x7f800000);
    int bk = 0x7fffffff;
    // (only for the cyclic order, taken when the super-chunks are too many to sort)
    const int64_t nsearch = PP.nchunks / PRUNED_CPS <= PRUNED_SORT ? 0 : PP.nchunks;
    for (int64_t k = tid; k < nsearch; k += SCAN_THREADS) {
        const float* b = reinterpret_cast<const float*>(PP.box + k * NB4);
        if (!(b[2 * D] == b[2 * D])) continue;             // a chunk without data
        float dd = 0.f;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const float e = 0.5f * (b[j] + b[D + j]) - cen[j];
            dd = fmaf(e, e, dd);
        }
        if (dd < bd) { bd = dd; bk = (int)k; }               // k increases: the first stays on ties
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float od = __shfl_xor_sync(0xffffffffu, bd, o);
        const int ok = __shfl_xor_sync(0xffffffffu, bk, o);
        if (od < bd || (od == bd && ok < bk)) { bd = od; bk = ok; }
    }
    if (lane == 0) {
        red_d[warp] = bd;
        red_k[warp] = bk;
    }
    __syncthreads();
    if (tid == 0) {
        float d0 = red_d[0];
        int k0 = red_k[0];
        for (int w = 1; w < NW; ++w)
            if (red_d[w] < d0 || (red_d[w] == d0 && red_k[w] < k0)) { d0 = red_d[w]; k0 = red_k[w]; }
        start_chunk = k0 == 0x7fffffff ? 0 : (k0 / PRUNED_CPS) * PRUNED_CPS;   // a multiple of 64 groups
    }
    __syncthreads();

    // The sweep runs over super-chunks (PRUNED_CPS chunks, 64 groups).  Up to PRUNED_SORT of them it
    // takes them nearest first: by the distance from the centre of their box to the
    // centroid of the block's queries (ties by index), sorted in shared memory by a bitonic
    // network, so the running extrema approach their final values within the first few
    // and the rest are tested against nearly final bounds.  With more super-chunks it runs
    // in cyclic order from the start one.  The first PRUNED_LEAD are streamed as they are;
    // the rest go in windows of PRUNED_WIN, each reduced first to the super-chunks that
    // some warp of the block may still need (tested against the running bounds, which only
    // tighten afterwards, so a super-chunk left out then would be skipped later too).  Only
    // the listed tiles are copied to shared memory.
    const int nsuper = (int)(PP.nchunks / PRUNED_CPS);
    const int sup0 = start_chunk / PRUNED_CPS;
    const bool sorted = nsuper <= PRUNED_SORT;
    __shared__ float skey[PRUNED_SORT];
    __shared__ short sidx[PRUNED_SORT];
    if (sorted) {
        int n2 = 1;
        while (n2 < nsuper) n2 <<= 1;
        for (int s = tid; s < n2; s += SCAN_THREADS) {
            float dd = __int_as_float(0x7f800000);
            if (s < nsuper) {
                const float* b = reinterpret_cast<const float*>(PP.sbox + (int64_t)s * NB4);
                if (b[2 * D] == b[2 * D]) {                   // a super-chunk with data
                    dd = 0.f;
#pragma unroll
                    for (int j = 0; j < D; ++j) {
                        const float e = 0.5f * (b[j] + b[D + j]) - cen[j];
                        dd = fmaf(e, e, dd);
                    }
                }
            }
            skey[s] = dd;
            sidx[s] = (short)s;            // padding entries (s >= nsuper) sort last
        }
        __syncthreads();
        for (int k = 2; k <= n2; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = tid; i < n2; i += SCAN_THREADS) {
                    const int x = i ^ j;
                    if (x > i) {
                        const float ki = skey[i], kx = skey[x];
                        const int ii = sidx[i], ix = sidx[x];
                        const bool gt = ki > kx || (ki == kx && ii > ix);
                        if (gt == ((i & k) == 0)) {           // ascending where bit k of i is 0
                            skey[i] = kx;
                            skey[x] = ki;
                            sidx[i] = (short)ix;
                            sidx[x] = (short)ii;
                        }
                    }
                }
                __syncthreads();
            }
        }
    }
    // the super-chunk taken at place s of the sweep
    auto super_at = [&](int s) {
        if (sorted) return (int)sidx[s];
        int sp = sup0 + s;
        return sp >= nsuper ? sp - nsuper : sp;
    };
    const int tps = TILE_GROUPS_MAX / tg;             // tiles per super-chunk
    __shared__ int seq[PRUNED_WIN * (TILE_GROUPS_MAX / 8)];
    __shared__ unsigned wmask[PRUNED_WIN / 32];
    __shared__ int seq_len;
    // the stages' copies of the tile's chunk records follow the data stages
    float4* recs = tiles + (size_t)PRUNED_STAGES * tg * NCH;
    const uint32_t rec_bytes = (uint32_t)(tg / PRUNED_CG) * NB4 * 16u;
    auto issue = [&](int step, int tile) {            // one thread: the bulk copies of ring step `step`
        if (step == P.skip_tile) return;
        const int st = step % PRUNED_STAGES;
        last_issued[st] = step;
        mbar_expect_tx(&bars[st], tile_bytes + rec_bytes);
        bulk_g2s(tiles + (size_t)st * tg * NCH, hot + (size_t)tile * tg * NCH, tile_bytes, &bars[st]);
        bulk_g2s(recs + (size_t)st * RECS * NB4, PP.box + (size_t)tile * (tg / PRUNED_CG) * NB4, rec_bytes, &bars[st]);
    };
    auto load_rec = [&](const float4* rec, float (&b)[NB4 * 4]) {     // from shared memory
#pragma unroll
        for (int k = 0; k < NB4; ++k) {
            const float4 v = rec[k];
            b[4 * k] = v.x;
            b[4 * k + 1] = v.y;
            b[4 * k + 2] = v.z;
            b[4 * k + 3] = v.w;
        }
    };
    auto load_box = [&](const float4* rec, float (&b)[NB4 * 4]) {
#pragma unroll
        for (int k = 0; k < NB4; ++k) {
            const float4 v = __ldg(rec + k);
            b[4 * k] = v.x;
            b[4 * k + 1] = v.y;
            b[4 * k + 2] = v.z;
            b[4 * k + 3] = v.w;
        }
    };

    float mu[R], ml[R], pu[R], pl[R];
    int bu[R], bl[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        mu[r] = __int_as_float(0x7f800000);
        ml[r] = -__int_as_float(0x7f800000);
        pu[r] = mu[r];
        pl[r] = ml[r];
        bu[r] = -1;
        bl[r] = -1;
    }
    // bit r set when some query of row r of the warp may need the record b
    auto row_needs = [&](const float (&b)[NB4 * 4]) {
        unsigned rows = 0u;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const bool n = b[2 * D] == b[2 * D] && live[r] &&        // the record holds data
                           chunk_needed<NORM, C, U>(qq[r], b, b + D, b[2 * D], b[2 * D + 1], mu[r], ml[r]);
            if (__any_sync(0xffffffffu, n)) rows |= 1u << r;
        }
        return rows;
    };
    unsigned evaluated = 0, candidates = 0;
    // the warp's loosest running bounds (largest mu, smallest ml of its finite queries)
    auto warp_bounds = [&](float& mmax, float& mmin) {
        mmax = -__int_as_float(0x7f800000);
        mmin = __int_as_float(0x7f800000);
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (live[r]) {
                mmax = fmaxf(mmax, mu[r]);
                mmin = fminf(mmin, ml[r]);
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mmax = fmaxf(mmax, __shfl_xor_sync(0xffffffffu, mmax, o));
            mmin = fminf(mmin, __shfl_xor_sync(0xffffffffu, mmin, o));
        }
    };

    int step = 0;                   // tiles this block has taken from the ring
    bool ok = true;
    for (int s_begin = 0; ok && s_begin < nsuper;) {
        const bool lead = s_begin == 0;
        const int s_count = min(lead ? PRUNED_LEAD : PRUNED_WIN, nsuper - s_begin);
        if (lead) {
            if (tid == 0) {
                for (int i = 0; i < s_count * tps; ++i) seq[i] = super_at(i / tps) * tps + i % tps;
                seq_len = s_count * tps;
            }
        } else {
            if (tid < PRUNED_WIN / 32) wmask[tid] = 0u;
            __syncthreads();
            float mmax, mmin;
            warp_bounds(mmax, mmin);
            for (int i0 = 0; i0 < s_count; i0 += 32) {
                bool need8 = false;
                if (wlive && i0 + lane < s_count) {
                    const int sp = super_at(s_begin + i0 + lane);
                    float sb[NB4 * 4];
                    load_box(PP.sbox + (int64_t)sp * NB4, sb);
                    need8 = sb[2 * D] == sb[2 * D] &&
                            box_needed<NORM, C, U>(qlo, qhi, sb, sb + D, sb[2 * D], sb[2 * D + 1], mmax, mmin);
                }
                const unsigned bits = __ballot_sync(0xffffffffu, need8);
                if (lane == 0 && bits) atomicOr(&wmask[i0 >> 5], bits);
            }
            __syncthreads();
            if (tid == 0) {
                int n = 0;
                for (int i = 0; i < s_count; ++i) {
                    if (!((wmask[i >> 5] >> (i & 31)) & 1u)) continue;
                    const int sp = super_at(s_begin + i);
                    for (int k = 0; k < tps; ++k) seq[n++] = sp * tps + k;
                }
                seq_len = n;
            }
        }
        __syncthreads();
        const int len = seq_len;
        if (PP.work && tid == 0 && len) atomicAdd(PP.work + 1, (unsigned long long)len);
        if (tid == 0)
            for (int k = 0; k < PRUNED_STAGES && k < len; ++k) issue(step + k, seq[k]);
        // The warps take the batch's tiles independently: a warp waits for a tile's copies,
        // tests and evaluates its chunks, and counts itself out of the stage; the last warp
        // out of a stage refills it with the tile PRUNED_STAGES ahead, so a warp with little
        // to evaluate runs up to that far ahead of the others instead of waiting at a block
        // barrier after every tile.
        bool ok_w = true;
        for (int i = 0; i < len; ++i) {
            const int st = (step + i) % PRUNED_STAGES;
            const uint32_t par = (uint32_t)((step + i) / PRUNED_STAGES) & 1u;
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bars[st], par, P.err, P.wait_ns))) {
                ok_w = false;
                break;
            }
            const float4* tile = tiles + (size_t)st * tg * NCH;
            const float4* trec = recs + (size_t)st * RECS * NB4;
            const int64_t tg0 = (int64_t)seq[i] * tg;           // first group of the tile
            const int chunk0 = (int)(tg0 / PRUNED_CG), nck = tg / PRUNED_CG;
            // lane k tests chunk k of the tile against the warp's query box and loosest
            // bounds; only the chunks that pass get the per-query test
            float mmax, mmin;
            warp_bounds(mmax, mmin);
            bool cand = false;
            if (wlive && lane < nck) {
                float cb[NB4 * 4];
                load_rec(trec + lane * NB4, cb);
                cand = cb[2 * D] == cb[2 * D] &&
                       box_needed<NORM, C, U>(qlo, qhi, cb, cb + D, cb[2 * D], cb[2 * D + 1], mmax, mmin);
            }
            const unsigned cands = __ballot_sync(0xffffffffu, cand);
            candidates += __popc(cands);
            for (unsigned left = cands; left; left &= left - 1) {
                const int k = __ffs(left) - 1;
                const int chunk = chunk0 + k, c = k * PRUNED_CG;
                float bx[NB4 * 4];
                load_rec(trec + k * NB4, bx);
                const unsigned rows = row_needs(bx);
                if (!rows) continue;
                evaluated += __popc(rows);
#pragma unroll 2
                for (int gi = 0; gi < PRUNED_CG; ++gi) {
                    float4 x[NCH];
#pragma unroll
                    for (int ch = 0; ch < NCH; ++ch) x[ch] = tile[(c + gi) * NCH + ch];
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        if (!((rows >> r) & 1u)) continue;      // warp-uniform
                        float vu[4], vl[4];
                        group_values<NORM, C, U, true>(qq[r], x, vu, vl);
                        // the group's own extrema first: one link of each running chain per group
                        mu[r] = min3f(mu[r], min3f(vu[0], vu[1], vu[2]), vu[3]);
                        ml[r] = max3f(ml[r], max3f(vl[0], vl[1], vl[2]), vl[3]);
                    }
                }
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    bu[r] = (mu[r] < pu[r]) ? chunk : bu[r];
                    pu[r] = mu[r];
                    bl[r] = (ml[r] > pl[r]) ? chunk : bl[r];
                    pl[r] = ml[r];
                }
            }
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();                          // this warp's reads of the stage are done
                if (atomicAdd(&fin[st], 1) == NW - 1) {
                    fin[st] = 0;
                    if (i + PRUNED_STAGES < len) {
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        issue(step + i + PRUNED_STAGES, seq[i + PRUNED_STAGES]);
                    }
                }
            }
        }
        ok = __syncthreads_and(ok_w);
        if (!ok && tid == 0) {
            // as in scan_block: wait (bounded) for every copy still in flight
            for (int s2 = 0; s2 < PRUNED_STAGES; ++s2)
                if (last_issued[s2] >= 0)
                    mbar_wait_bounded(&bars[s2], (uint32_t)(last_issued[s2] / PRUNED_STAGES) & 1u, nullptr);
        }
        step += len;
        s_begin += s_count;
    }
    if (PP.work && lane == 0 && evaluated) atomicAdd(PP.work, (unsigned long long)evaluated);
    if (PP.work && lane == 0 && candidates) atomicAdd(PP.work + 2, (unsigned long long)candidates);
    PartialRec<float>* out = static_cast<PartialRec<float>*>(P.partial);
    if (!ok) {
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (qidx[r] >= 0)
                out[qidx[r]] = PartialRec<float>{__int_as_float(0x7fc00000), -1, __int_as_float(0x7fc00000), -1};
        return;
    }

    // the lowest position attaining each extremum inside its chunk, then its data index
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (qidx[r] < 0) continue;
        int iu = -1, il = -1;
#pragma unroll 1
        for (int side = 0; side < 2; ++side) {
            const int chunk = side == 0 ? bu[r] : bl[r];
            if (chunk < 0) continue;
#pragma unroll 1
            for (int gi = 0; gi < PRUNED_CG; ++gi) {
                const int64_t g = (int64_t)chunk * PRUNED_CG + gi;
                float4 x[NCH];
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) x[ch] = __ldg(hot + g * NCH + ch);
                float vu[4], vl[4];
                group_values<NORM, C, U, true>(qq[r], x, vu, vl);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if (side == 0 && iu < 0 && vu[e] == mu[r]) iu = PP.dperm[g * 4 + e];
                    if (side == 1 && il < 0 && vl[e] == ml[r]) il = PP.dperm[g * 4 + e];
                }
            }
        }
        const float lo_v = S::AUX ? ml[r] + sq[r] : ml[r];
        out[qidx[r]] = PartialRec<float>{mu[r], iu, lo_v, il};
    }
}

}  // namespace lip
