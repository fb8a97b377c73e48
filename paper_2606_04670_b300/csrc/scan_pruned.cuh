// Exact scan with chunk bounds (lip_set_tuning variants 6 and 7): the same values and
// extrema as scan_exact_kernel, over the data in spatial order, skipping every 32-point
// chunk that provably cannot lower H_up nor raise H_lo of any query of the warp.
//
// The data are laid out in the spatial order of their points (a Morton order), so a
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
// unpruned scan over the same order.  The warp evaluates a chunk when any of its queries
// needs it (queries in spatial order make the warp's needs coherent).
//
// Processing order: the block's queries (R per thread, in spatial order) pick a start
// chunk, the one whose box centre is nearest their centroid, rounded down to a multiple
// of 8 chunks (64 groups, so the order is the same for every tile size), and the sweep
// wraps around from there; the near chunks tighten mu and ml first.  Among data with
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
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const float p = fmaxf(t[j], 0.f);
            acc = (j == 0 && U == 0) ? p : __fadd_rn(acc, p);
        }
        // with constrained coordinates the lower side runs on the aux channel with the
        // same (upper) distance; without them both sides take the symmetric distance
        skip_u = __fadd_rn(ylo, acc) >= mu;
        skip_l = __fsub_rn(yhv, acc) <= ml;
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

template <int NORM, int C, int U, int R>
__global__ void __launch_bounds__(SCAN_THREADS) scan_pruned_kernel(const PrunedParams PP) {
    using S = ExactShape<NORM, C, U>;
    constexpr int D = S::D;
    constexpr int NCH = S::NCH;
    constexpr int NB4 = pruned_box_f4(D);
    constexpr int NW = SCAN_THREADS / 32;
    extern __shared__ __align__(128) float4 tiles[];   // SCAN_STAGES * tile_groups * NCH
    __shared__ __align__(8) uint64_t bars[SCAN_STAGES];
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

    // the block's queries: a warp holds 32 R consecutive positions of the spatial order
    // (lane l, row r: position qblock * 128 R + warp * 32 R + l R + r), so its queries are
    // neighbours and its chunk decisions agree
    float2 qq[R][D];
    float sq[R];
    int64_t qidx[R];
    bool live[R];
    float csum[D + 1];
#pragma unroll
    for (int j = 0; j <= D; ++j) csum[j] = 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t pos = (int64_t)blockIdx.x * (SCAN_THREADS * R) + (int64_t)warp * 32 * R + lane * R + r;
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
        for (int s = 0; s < SCAN_STAGES; ++s) mbar_init(&bars[s], 1);
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
    for (int64_t k = tid; k < PP.nchunks; k += SCAN_THREADS) {
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
        start_chunk = k0 == 0x7fffffff ? 0 : (k0 / 8) * 8;   // a multiple of 64 groups
    }
    __syncthreads();

    const int ntiles = (int)(P.ngroups / tg);
    const int t0 = (int)((int64_t)start_chunk * CHUNK_GROUPS / tg);
    auto tile_of = [&](int t) { const int u = t0 + t; return u >= ntiles ? u - ntiles : u; };
    if (tid == 0) {
        for (int s = 0; s < SCAN_STAGES && s < ntiles; ++s) {
            if (s == P.skip_tile) continue;
            mbar_expect_tx(&bars[s], tile_bytes);
            bulk_g2s(tiles + (size_t)s * tg * NCH, hot + (size_t)tile_of(s) * tg * NCH, tile_bytes, &bars[s]);
        }
    }

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
    unsigned evaluated = 0;
    bool super_need = false;        // the current 8 chunks (64 groups) may be needed

    int t = 0;
    bool ok = true;
    for (; t < ntiles; ++t) {
        const int s = t % SCAN_STAGES;
        const uint32_t par = (uint32_t)(t / SCAN_STAGES) & 1u;
        const bool got = mbar_wait_bounded(&bars[s], par, P.err, P.wait_ns);
        if (!__syncthreads_and(got)) { ok = false; break; }
        const float4* tile = tiles + (size_t)s * tg * NCH;
        const int64_t tg0 = (int64_t)tile_of(t) * tg;        // first group of the tile
        for (int c = 0; c < tg; c += CHUNK_GROUPS) {
            const int chunk = (int)((tg0 + c) / CHUNK_GROUPS);
            // the record of 8 chunks first: its box contains theirs and its value range
            // theirs, so where it rules a query out, each of the 8 would too
            if ((chunk & 7) == 0) {
                float sb[NB4 * 4];
#pragma unroll
                for (int k = 0; k < NB4; ++k) {
                    const float4 v = __ldg(PP.sbox + (int64_t)(chunk >> 3) * NB4 + k);
                    sb[4 * k] = v.x;
                    sb[4 * k + 1] = v.y;
                    sb[4 * k + 2] = v.z;
                    sb[4 * k + 3] = v.w;
                }
                bool need8 = false;
                if (sb[2 * D] == sb[2 * D]) {
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        need8 = need8 ||
                                (live[r] && chunk_needed<NORM, C, U>(qq[r], sb, sb + D, sb[2 * D], sb[2 * D + 1], mu[r], ml[r]));
                }
                super_need = __any_sync(0xffffffffu, need8);
            }
            if (!super_need) continue;
            float bx[NB4 * 4];
#pragma unroll
            for (int k = 0; k < NB4; ++k) {
                const float4 v = __ldg(PP.box + (int64_t)chunk * NB4 + k);
                bx[4 * k] = v.x;
                bx[4 * k + 1] = v.y;
                bx[4 * k + 2] = v.z;
                bx[4 * k + 3] = v.w;
            }
            const float ylo = bx[2 * D], yhv = bx[2 * D + 1];
            bool need = false;
            if (ylo == ylo) {                                 // the chunk holds data
#pragma unroll
                for (int r = 0; r < R; ++r)
                    need = need || (live[r] && chunk_needed<NORM, C, U>(qq[r], bx, bx + D, ylo, yhv, mu[r], ml[r]));
            }
            if (!__any_sync(0xffffffffu, need)) continue;
            ++evaluated;
#pragma unroll 2
            for (int gi = 0; gi < CHUNK_GROUPS; ++gi) {
                float4 x[NCH];
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) x[ch] = tile[(c + gi) * NCH + ch];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    float vu[4], vl[4];
                    group_values<NORM, C, U>(qq[r], x, vu, vl);
                    mu[r] = min3f(min3f(mu[r], vu[0], vu[1]), vu[2], vu[3]);
                    ml[r] = max3f(max3f(ml[r], vl[0], vl[1]), vl[2], vl[3]);
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
        __syncthreads();   // every thread is done with stage s
        if (tid == 0 && t + SCAN_STAGES < ntiles && t + SCAN_STAGES != P.skip_tile) {
            mbar_expect_tx(&bars[s], tile_bytes);
            bulk_g2s(tiles + (size_t)s * tg * NCH, hot + (size_t)tile_of(t + SCAN_STAGES) * tg * NCH, tile_bytes,
                     &bars[s]);
        }
    }
    if (PP.work && lane == 0 && evaluated) atomicAdd(PP.work, (unsigned long long)evaluated);
    PartialRec<float>* out = static_cast<PartialRec<float>*>(P.partial);
    if (!ok) {
        // as in scan_block: wait (bounded) for the copies still in flight, then give up
        if (tid == 0) {
            for (int u = t; u < ntiles && u < t + SCAN_STAGES; ++u)
                if (u != P.skip_tile) mbar_wait_bounded(&bars[u % SCAN_STAGES], (uint32_t)(u / SCAN_STAGES) & 1u, nullptr);
        }
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
            for (int gi = 0; gi < CHUNK_GROUPS; ++gi) {
                const int64_t g = (int64_t)chunk * CHUNK_GROUPS + gi;
                float4 x[NCH];
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) x[ch] = __ldg(hot + g * NCH + ch);
                float vu[4], vl[4];
                group_values<NORM, C, U>(qq[r], x, vu, vl);
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
