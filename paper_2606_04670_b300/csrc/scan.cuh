// All-pairs envelope scan: H_up(q) = min_k (y^k + M dist_up), H_lo(q) = max_k (y^k - M dist_lo)
// (Sec. 3, Eq. (upperlower); monotone distance of Sec. 4.1, Eq. (distmon)).
//
// Scan layout ("hot" copy, built by build_hot_kernel): data points in groups of 4,
// each group stored as NCH float4 channels [coord 0..D-1][y][aux?], coordinates
// permuted so the C constrained ones come first, mirrored for decreasing
// coordinates, and multiplied by M * w, so that dist on the scaled copy is
// M * dist.  Padding points have y = NaN; the three-input min/max ignore NaN, so
// they drop out without a length check in the hot loop.
//
// For L1 with constrained coordinates, dist_lo = dist_up - sum_{j<C} t_j, so the
// lower bound is (y - sum_{j<C} x_j) - dist_up + sum_{j<C} q_j: the aux channel
// holds y - sum_{j<C} x_j and the scan needs a single distance per pair.
#pragma once

#include "common.cuh"

namespace lip {

struct ScanParams {
    const void* Q;            // caller's queries [nq][d], element type of the handle
    int64_t nq;
    int d;                    // caller's dimension
    int C;                    // constrained coordinates (first C of the layout)
    int dl;                   // layout dimension (>= d for the generic kernel)
    int nch;                  // float4 (or double4) channels per group
    int perm[D_MAX];          // layout coordinate j <- caller coordinate perm[j]
    double scale[D_MAX];      // M * sign_j * w_j
    const void* hot;          // scan layout
    int64_t ngroups;          // groups to scan (multiple of TILE_GROUPS_MAX)
    int64_t groups_per_split; // multiple of tile_groups
    int tile_groups;          // groups per shared-memory tile (multiple of 8, <= 64)
    void* partial;            // PartialRec<T> [gridDim.y][nq]
    unsigned* err;            // device status word
    unsigned long long wait_ns = WAIT_LIMIT_NS;  // limit of the exact scan's bounded waits
    int skip_tile = -1;       // tests only: every block leaves out the bulk copy of its tile
                              // number skip_tile (its wait then runs out); -1 = none
};

// Per (split, query) result of a scan: approximate extremum values and their indices.
template <typename T>
struct PartialRec;
template <>
struct __align__(16) PartialRec<float> { float vu; int iu; float vl; int il; };
template <>
struct __align__(16) PartialRec<double> { double vu; double vl; int iu; int il; int pad0; int pad1; };

constexpr int SCAN_THREADS = 128;
constexpr int SCAN_STAGES = 3;
constexpr int CHUNK_GROUPS = 8;   // argmin/argmax are localised to 32-point chunks

// DIRECT: the lower distance is formed from the negative parts of the constrained
// differences instead of through the aux channel (used by the pruned scan, whose chunk
// bounds are tighter on the direct form; no aux channel then).
template <int NORM, int C, int U, bool DIRECT = false>
struct ExactShape {
    static constexpr int D = C + U;
    static constexpr bool AUX = !DIRECT && (NORM == LIP_L1 && C > 0);
    static constexpr int NCH = D + 1 + (AUX ? 1 : 0);
};

__device__ __forceinline__ float2 half_of(const float4& v, int h) {
    return h == 0 ? make_float2(v.x, v.y) : make_float2(v.z, v.w);
}

template <int K>
__device__ __forceinline__ float max_reduce(const float (&v)[K]) {
    static_assert(K >= 1, "");
    if constexpr (K == 1) {
        return v[0];
    } else {
        float m = (K == 2) ? max2f(v[0], v[1]) : max3f(v[0], v[1], v[2]);
#pragma unroll
        for (int i = 3; i < K; i += 2) m = (i + 1 < K) ? max3f(m, v[i], v[i + 1]) : max2f(m, v[i]);
        return m;
    }
}

// Bound values of the 4 points of one group for one query (qq: the query's scaled
// coordinates, each duplicated into both halves of a float2).  vu = y + M dist_up;
// vl = y - M dist_lo, except with AUX where vl = (y - Sx) - M dist_up (the caller adds
// sum_{j<C} q_j).  Exactly the same instruction sequence is used by the scan and by the
// rescan that recovers the index, so the values compare bitwise.  fs (L2 with constrained
// coordinates): the lower distances of the group's second pair of points take the FMA-pipe
// square root (sqrt_fma2) instead of the special-function unit, which the two roots per
// pair otherwise saturate.
template <int NORM, int C, int U, bool DIRECT = false>
__device__ __forceinline__ void group_values(const float2 (&qq)[C + U],
                                             const float4 (&x)[ExactShape<NORM, C, U, DIRECT>::NCH],
                                             float (&vu)[4], float (&vl)[4], bool fs = false) {
    constexpr int D = C + U;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float2 t[D];
#pragma unroll
        for (int j = 0; j < D; ++j) t[j] = sub2(qq[j], half_of(x[j], h));
        const float2 yv = half_of(x[D], h);
        float2 du, dl;
        if constexpr (NORM == LIP_L2) {
            float2 s0 = make_float2(0.f, 0.f);
            if constexpr (U > 0) {
                s0 = mul2(t[C], t[C]);
#pragma unroll
                for (int j = C + 1; j < D; ++j) s0 = fma2(t[j], t[j], s0);
            }
            if constexpr (C > 0) {
                float2 su, sl;
#pragma unroll
                for (int j = 0; j < C; ++j) {
                    // the positive and negative parts on the ALU pipe, next to the busier FMA pipe
                    const float2 p = make_float2(fmaxf(t[j].x, 0.f), fmaxf(t[j].y, 0.f));
                    const float2 n = make_float2(fminf(t[j].x, 0.f), fminf(t[j].y, 0.f));
                    if (j == 0 && U == 0) { su = mul2(p, p); sl = mul2(n, n); }
                    else if (j == 0) { su = fma2(p, p, s0); sl = fma2(n, n, s0); }
                    else { su = fma2(p, p, su); sl = fma2(n, n, sl); }
                }
                du = make_float2(sqrt_approx(su.x), sqrt_approx(su.y));
                dl = (fs && h == 1) ? sqrt_fma2(sl) : make_float2(sqrt_approx(sl.x), sqrt_approx(sl.y));
            } else {
                du = make_float2(sqrt_approx(s0.x), sqrt_approx(s0.y));
                dl = du;
            }
        } else if constexpr (NORM == LIP_L1) {
            float2 acc = make_float2(0.f, 0.f);
            // unconstrained: |t|, constrained: (t)_+ (upper); the lower comes from AUX, or
            // (DIRECT) from the same unconstrained sum plus the negative parts (-t)_+
            if constexpr (U >= 2) {
                acc = make_float2(fabsf(t[C].x) + fabsf(t[C + 1].x), fabsf(t[C].y) + fabsf(t[C + 1].y));
#pragma unroll
                for (int j = C + 2; j < D; ++j) acc = make_float2(acc.x + fabsf(t[j].x), acc.y + fabsf(t[j].y));
            } else if constexpr (U == 1) {
                acc = make_float2(fabsf(t[C].x), fabsf(t[C].y));
            }
            float2 accl = acc;
#pragma unroll
            for (int j = 0; j < C; ++j) {
                const float2 p = make_float2(fmaxf(t[j].x, 0.f), fmaxf(t[j].y, 0.f));
                if (j == 0 && U == 0) acc = p;
                else acc = add2(acc, p);
                if constexpr (DIRECT) {
                    const float2 n = make_float2(fmaxf(-t[j].x, 0.f), fmaxf(-t[j].y, 0.f));
                    if (j == 0 && U == 0) accl = n;
                    else accl = add2(accl, n);
                }
            }
            du = acc;
            dl = DIRECT ? accl : acc;
        } else {  // LINF
            float du_[2], dl_[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                float uu = 0.f;
                if constexpr (U > 0) {
                    float ab[U];
#pragma unroll
                    for (int j = 0; j < U; ++j) ab[j] = fabsf(e == 0 ? t[C + j].x : t[C + j].y);
                    uu = max_reduce<U>(ab);
                }
                if constexpr (C > 0) {
                    float pu[C + 1], pl[C + 1];
#pragma unroll
                    for (int j = 0; j < C; ++j) {
                        const float tj = e == 0 ? t[j].x : t[j].y;
                        pu[j] = tj;
                        pl[j] = -tj;
                    }
                    pu[C] = uu;   // uu >= 0 (0 when U == 0) supplies the max with 0
                    pl[C] = uu;
                    du_[e] = max_reduce<C + 1>(pu);
                    dl_[e] = max_reduce<C + 1>(pl);
                } else {
                    du_[e] = uu;
                    dl_[e] = uu;
                }
            }
            du = make_float2(du_[0], du_[1]);
            dl = make_float2(dl_[0], dl_[1]);
        }
        float2 v_up = add2(yv, du);
        float2 v_lo;
        if constexpr (ExactShape<NORM, C, U, DIRECT>::AUX) v_lo = sub2(half_of(x[D + 1], h), dl);
        else v_lo = sub2(yv, dl);
        vu[2 * h] = v_up.x;
        vu[2 * h + 1] = v_up.y;
        vl[2 * h] = v_lo.x;
        vl[2 * h + 1] = v_lo.y;
    }
}

// Load R queries into registers: layout coordinate j = scale[j] * q[perm[j]] (product in
// FP64, one rounding), duplicated into float2.  Out-of-range queries get zeros and are
// never stored; non-finite queries produce NaN bounds and index -1.
template <int D, int R>
__device__ __forceinline__ void load_queries(const ScanParams& P, int64_t qbase, float2 (&qq)[R][D], float (&sq)[R], int C) {
    const float* Q = static_cast<const float*>(P.Q);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t qi = qbase + (int64_t)r * SCAN_THREADS;
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            float v = 0.f;
            if (qi < P.nq) v = (float)(P.scale[j] * (double)__ldg(Q + qi * P.d + P.perm[j]));
            qq[r][j] = make_float2(v, v);
            if (j < C) s = s + v;
        }
        sq[r] = s;
    }
}

__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// One block's share of the scan: queries [qblock * 128 R, +128 R) against data split
// `split` of P.  Used by the one-launch-per-data-set kernel below and by the batched
// persistent kernel (which calls it once per work item and re-initialises the
// barriers between items: reinit = true invalidates them first).  FSR > 0: query rows
// r with r % FSR == FSR - 1 take group_values' FMA-pipe square roots (one in 4 FSR of the
// pair's roots).
template <int NORM, int C, int U, int R, int FSR = 0>
__device__ __forceinline__ void scan_block(const ScanParams& P, int64_t qblock, int split, float4* tiles,
                                           uint64_t* bars, bool reinit) {
    using S = ExactShape<NORM, C, U>;
    constexpr int D = S::D;
    constexpr int NCH = S::NCH;

    const int tg = P.tile_groups;
    const uint32_t tile_bytes = (uint32_t)tg * NCH * 16u;
    const float4* hot = static_cast<const float4*>(P.hot);

    const int64_t qbase = qblock * (SCAN_THREADS * R) + threadIdx.x;
    float2 qq[R][D];
    float sq[R];
    load_queries<D, R>(P, qbase, qq, sq, C);

    const int64_t g_begin = (int64_t)split * P.groups_per_split;
    int64_t g_end = g_begin + P.groups_per_split;
    if (g_end > P.ngroups) g_end = P.ngroups;
    const int ntiles = g_begin < g_end ? (int)((g_end - g_begin) / tg) : 0;

    if (threadIdx.x == 0) {
#pragma unroll
        for (int s = 0; s < SCAN_STAGES; ++s) {
            if (reinit) mbar_inval(&bars[s]);
            mbar_init(&bars[s], 1);
        }
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int s = 0; s < SCAN_STAGES && s < ntiles; ++s) {
            if (s == P.skip_tile) continue;
            mbar_expect_tx(&bars[s], tile_bytes);
            bulk_g2s(tiles + (size_t)s * tg * NCH, hot + (size_t)(g_begin + (int64_t)s * tg) * NCH, tile_bytes, &bars[s]);
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

    int t = 0;
    bool ok = true;
    for (; t < ntiles; ++t) {
        const int s = t % SCAN_STAGES;
        const uint32_t par = (uint32_t)(t / SCAN_STAGES) & 1u;
        const bool got = mbar_wait_bounded(&bars[s], par, P.err, P.wait_ns);
        if (!__syncthreads_and(got)) { ok = false; break; }
        const float4* tile = tiles + (size_t)s * tg * NCH;
        for (int c = 0; c < tg; c += CHUNK_GROUPS) {
#pragma unroll 2
            for (int gi = 0; gi < CHUNK_GROUPS; ++gi) {
                float4 x[NCH];
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) x[ch] = tile[(c + gi) * NCH + ch];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    float vu[4], vl[4];
                    group_values<NORM, C, U>(qq[r], x, vu, vl, FSR > 0 && r % FSR == FSR - 1);
                    // the group's own extrema first: one link of each running chain per group
                    mu[r] = min3f(mu[r], min3f(vu[0], vu[1], vu[2]), vu[3]);
                    ml[r] = max3f(ml[r], max3f(vl[0], vl[1], vl[2]), vl[3]);
                }
            }
            const int chunk = (int)((g_begin + (int64_t)t * tg + c) / CHUNK_GROUPS);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                bu[r] = (mu[r] < pu[r]) ? chunk : bu[r];
                pu[r] = mu[r];
                bl[r] = (ml[r] > pl[r]) ? chunk : bl[r];
                pl[r] = ml[r];
            }
        }
        __syncthreads();   // every thread is done with stage s
        if (threadIdx.x == 0 && t + SCAN_STAGES < ntiles && t + SCAN_STAGES != P.skip_tile) {
            mbar_expect_tx(&bars[s], tile_bytes);
            bulk_g2s(tiles + (size_t)s * tg * NCH, hot + (size_t)(g_begin + (int64_t)(t + SCAN_STAGES) * tg) * NCH,
                     tile_bytes, &bars[s]);
        }
    }
    if (!ok) {
        // A copy did not arrive in time: wait (bounded, with the default limit) for the
        // copies still in flight so none lands in shared memory after this block has
        // exited, then give up.  A tile left out on purpose has no copy to wait for.
        if (threadIdx.x == 0) {
            for (int u = t; u < ntiles && u < t + SCAN_STAGES; ++u)
                if (u != P.skip_tile) mbar_wait_bounded(&bars[u % SCAN_STAGES], (uint32_t)(u / SCAN_STAGES) & 1u, nullptr);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int64_t qi = qbase + (int64_t)r * SCAN_THREADS;
            if (qi < P.nq)
                static_cast<PartialRec<float>*>(P.partial)[(int64_t)split * P.nq + qi] =
                    PartialRec<float>{__int_as_float(0x7fc00000), -1, __int_as_float(0x7fc00000), -1};
        }
        return;
    }

    // Recover the lowest index attaining each extremum inside its chunk.
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t qi = qbase + (int64_t)r * SCAN_THREADS;
        if (qi >= P.nq) continue;
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
                group_values<NORM, C, U>(qq[r], x, vu, vl, FSR > 0 && r % FSR == FSR - 1);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if (side == 0 && iu < 0 && vu[e] == mu[r]) iu = (int)(g * 4 + e);
                    if (side == 1 && il < 0 && vl[e] == ml[r]) il = (int)(g * 4 + e);
                }
            }
        }
        const float lo_v = S::AUX ? ml[r] + sq[r] : ml[r];
        static_cast<PartialRec<float>*>(P.partial)[(int64_t)split * P.nq + qi] = PartialRec<float>{mu[r], iu, lo_v, il};
    }
}

template <int NORM, int C, int U, int R, int FSR = 0>
__global__ void __launch_bounds__(SCAN_THREADS)
scan_exact_kernel(const ScanParams P) {
    extern __shared__ __align__(128) float4 tiles[];   // SCAN_STAGES * tile_groups * NCH
    __shared__ __align__(8) uint64_t bars[SCAN_STAGES];
    scan_block<NORM, C, U, R, FSR>(P, blockIdx.x, blockIdx.y, tiles, bars, false);
}

// ------------------------------------------------------------------ generic scan
// Any (d <= D_MAX, C) and FP32 or FP64: coordinates padded to DP with zeros (2, 4, 8, 12,
// 16, 24 or 32); the
// monotone parts come from per-coordinate clamps (0 for constrained coordinates,
// +-Inf otherwise).  Plain global loads, index tracked per pair.  Used for FP64
// handles and for FP32 shapes without an exact instantiation.
template <typename T>
struct Vec4 { using type = float4; };
template <>
struct Vec4<double> { using type = double4; };

template <typename T, int NORM, int DP, int R>
__global__ void __launch_bounds__(SCAN_THREADS)
scan_generic_kernel(const ScanParams P) {
    using V4 = typename Vec4<T>::type;
    const V4* hot = static_cast<const V4*>(P.hot);
    const T* Q = static_cast<const T*>(P.Q);
    const int nch = P.nch;
    const int64_t qbase = (int64_t)blockIdx.x * (SCAN_THREADS * R) + threadIdx.x;
    const T inf = (T)INFINITY;
    T q[R][DP];
    T lo_clamp[DP], hi_clamp[DP];
#pragma unroll
    for (int j = 0; j < DP; ++j) {
        lo_clamp[j] = j < P.C ? (T)0 : -inf;
        hi_clamp[j] = j < P.C ? (T)0 : inf;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t qi = qbase + (int64_t)r * SCAN_THREADS;
#pragma unroll
        for (int j = 0; j < DP; ++j)
            q[r][j] = (qi < P.nq && j < P.dl && j < P.d) ? (T)(P.scale[j] * (double)Q[qi * P.d + P.perm[j]]) : (T)0;
    }
    T mu[R], ml[R];
    int iu[R], il[R];
#pragma unroll
    for (int r = 0; r < R; ++r) { mu[r] = inf; ml[r] = -inf; iu[r] = -1; il[r] = -1; }

    const int64_t g_begin = (int64_t)blockIdx.y * P.groups_per_split;
    int64_t g_end = g_begin + P.groups_per_split;
    if (g_end > P.ngroups) g_end = P.ngroups;
    for (int64_t g = g_begin; g < g_end; ++g) {
        T x[DP + 1][4];
#pragma unroll
        for (int ch = 0; ch <= DP; ++ch) {
            const V4 v = hot[g * nch + ch];
            x[ch][0] = v.x; x[ch][1] = v.y; x[ch][2] = v.z; x[ch][3] = v.w;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                T au = 0, al = 0;
#pragma unroll
                for (int j = 0; j < DP; ++j) {
                    const T tj = q[r][j] - x[j][e];
                    const T u = fabs(tj > lo_clamp[j] ? tj : lo_clamp[j]);
                    const T l = fabs(tj < hi_clamp[j] ? tj : hi_clamp[j]);
                    if (NORM == LIP_L1) { au += u; al += l; }
                    else if (NORM == LIP_L2) { au += u * u; al += l * l; }
                    else { au = u > au ? u : au; al = l > al ? l : al; }
                }
                if (NORM == LIP_L2) { au = sqrt(au); al = sqrt(al); }
                const T vu = x[DP][e] + au;
                const T vl = x[DP][e] - al;
                if (vu < mu[r]) { mu[r] = vu; iu[r] = (int)(g * 4 + e); }
                if (vl > ml[r]) { ml[r] = vl; il[r] = (int)(g * 4 + e); }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t qi = qbase + (int64_t)r * SCAN_THREADS;
        if (qi < P.nq) {
            PartialRec<T> rec{};
            rec.vu = mu[r]; rec.iu = iu[r]; rec.vl = ml[r]; rec.il = il[r];
            static_cast<PartialRec<T>*>(P.partial)[(int64_t)blockIdx.y * P.nq + qi] = rec;
        }
    }
}

// ------------------------------------------------------------------ split merge

struct MergeParams {
    const void* Q;
    int64_t nq;
    int d;
    int nsplit;
    double M;
    int norm;
    int8_t mon[D_MAX];   // caller's coordinate order
    double w[D_MAX];
    const void* X0;      // caller's data copy [N][d]
    const void* y0;
    const void* partial; // PartialRec<T> [nsplit][nq]
    void *g, *lo, *hi;
    int32_t *idx_up, *idx_lo;
};

// A float widened to double exactly from its IEEE-754 fields on the integer pipe
// (normal: exponent rebias by 1023 - 127 and the mantissa moved up 29 bits; subnormal:
// normalised from its leading bit; zeros, infinities and NaN kept), which leaves the
// FP64 pipe, the merge's bound, to the arithmetic.  to_f64 of a double is itself.
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned long long s = (unsigned long long)(u >> 31) << 63;
    const unsigned e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    unsigned long long bits;
    if (e == 0xffu) bits = s | (0x7ffull << 52) | ((unsigned long long)m << 29);
    else if (e != 0u) bits = s | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)m << 29);
    else if (m == 0u) bits = s;
    else {
        const int p = 31 - __clz((int)m);                 // the leading bit, 0..22
        bits = s | ((unsigned long long)(p + 874) << 52) | (((unsigned long long)m << (52 - p)) & 0xfffffffffffffull);
    }
    return __longlong_as_double((long long)bits);
}

// dist_up (side > 0) or dist_lo (side < 0) in FP64 in the caller's coordinates.
template <typename T>
__device__ __forceinline__ double dist_fp64(const MergeParams& P, const T* q, const T* x, int side) {
    double acc = 0.0;
    for (int i = 0; i < P.d; ++i) {
        double t = to_f64(q[i]) - to_f64(x[i]);
        if (P.mon[i] < 0) t = -t;
        if (P.w[i] != 1.0) t *= P.w[i];                 // a product by 1 is exact: skip it
        double v;
        if (P.mon[i] != 0) v = side > 0 ? (t > 0 ? t : 0.0) : (t < 0 ? -t : 0.0);
        else v = fabs(t);
        if (P.norm == LIP_L1) acc += v;
        else if (P.norm == LIP_L2) acc += v * v;
        else acc = v > acc ? v : acc;
    }
    return P.norm == LIP_L2 ? sqrt(acc) : acc;
}

// Picks the best split record (lowest split, hence lowest index, on exact ties), then
// re-evaluates both winners in FP64 from the caller's data and writes g, lo, hi, idx.
template <typename T>
__device__ __forceinline__ void merge_one(const MergeParams& P, int64_t qi) {
    T bu = 0, bl = 0;
    int iu = -1, il = -1;
    const PartialRec<T>* part = static_cast<const PartialRec<T>*>(P.partial);
    for (int s = 0; s < P.nsplit; ++s) {
        const PartialRec<T> r = part[(int64_t)s * P.nq + qi];
        if (r.iu >= 0 && (iu < 0 || r.vu < bu)) { bu = r.vu; iu = r.iu; }
        if (r.il >= 0 && (il < 0 || r.vl > bl)) { bl = r.vl; il = r.il; }
    }
    const T* q = static_cast<const T*>(P.Q) + qi * P.d;
    bool finite = true;
    for (int i = 0; i < P.d; ++i) finite = finite && isfinite(q[i]);
    double hi, lo;
    if (!finite || iu < 0 || il < 0) {
        hi = lo = __longlong_as_double(0x7ff8000000000000ll);
        iu = il = -1;
    } else {
        const T* X0 = static_cast<const T*>(P.X0);
        const T* y0 = static_cast<const T*>(P.y0);
        hi = to_f64(y0[iu]) + P.M * dist_fp64<T>(P, q, X0 + (int64_t)iu * P.d, +1);
        lo = to_f64(y0[il]) - P.M * dist_fp64<T>(P, q, X0 + (int64_t)il * P.d, -1);
    }
    if (P.g) static_cast<T*>(P.g)[qi] = (T)(0.5 * (hi + lo));
    if (P.lo) static_cast<T*>(P.lo)[qi] = (T)lo;
    if (P.hi) static_cast<T*>(P.hi)[qi] = (T)hi;
    if (P.idx_up) P.idx_up[qi] = iu;
    if (P.idx_lo) P.idx_lo[qi] = il;
}

template <typename T>
__global__ void merge_kernel(const MergeParams P) {
    const int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (qi < P.nq) merge_one<T>(P, qi);
}

// -------------------------------------------------------------- layout builder

struct HotParams {
    const void* X0;      // caller's data [*][d]
    const void* y0;
    int64_t k0, k1;      // points to (re)build
    int d, C, dl, nch, aux;
    int perm[D_MAX];
    double scale[D_MAX];
    void* hot;
    unsigned* err;       // ERRBIT_NONFINITE if any value is not finite
    const int* gather = nullptr;   // layout position k holds data point gather[k] (nullptr: k)
};

template <typename T>
__global__ void build_hot_kernel(const HotParams P) {
    const int64_t k = P.k0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P.k1) return;
    const int64_t src = P.gather ? (int64_t)P.gather[k] : k;
    const T* x = static_cast<const T*>(P.X0) + src * P.d;
    const T yv = static_cast<const T*>(P.y0)[src];
    T* hot = static_cast<T*>(P.hot);
    const int64_t base = (k / GROUP) * (int64_t)P.nch * GROUP + (k % GROUP);
    bool finite = isfinite((double)yv);
    T sx = 0;
    for (int j = 0; j < P.dl; ++j) {
        T v = 0;
        if (j < P.d) {
            const T raw = x[P.perm[j]];
            finite = finite && isfinite((double)raw);
            v = (T)(P.scale[j] * (double)raw);
        }
        hot[base + (int64_t)j * GROUP] = v;
        if (j < P.C) sx = sx + v;
    }
    hot[base + (int64_t)P.dl * GROUP] = yv;
    if (P.aux) hot[base + (int64_t)(P.dl + 1) * GROUP] = yv - sx;
    if (!finite) atomicOr(P.err, ERRBIT_NONFINITE);
}

// Marks points [k0, k1) as padding: coordinates 0, y (channel dl) and aux = NaN.
template <typename T>
__global__ void pad_hot_kernel(void* hot_, int64_t k0, int64_t k1, int nch, int dl) {
    const int64_t k = k0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= k1) return;
    T* hot = static_cast<T*>(hot_);
    const int64_t base = (k / GROUP) * (int64_t)nch * GROUP + (k % GROUP);
    for (int ch = 0; ch < nch; ++ch) hot[base + (int64_t)ch * GROUP] = ch < dl ? (T)0 : (T)NAN;
}

}  // namespace lip

namespace lip {

// Queries held per thread by the exact kernel, by dimension (registers: 2 * R * D for
// the duplicated query coordinates).
__host__ __device__ constexpr int rows_for_dim(int D) { return D <= 4 ? 8 : (D <= 10 ? 4 : 2); }

// Launch variants of the exact kernel (chosen by lip_set_tuning / the autotuner):
// variant 0 holds rows_for_dim(D) queries per thread, variant 1 half as many (fewer
// registers, more resident warps, more shared-memory broadcasts per pair).  Variants 2-5
// (L2 scans with constrained coordinates, the two square roots per pair) are 0 and 1 with
// one in eight (2, 3) or one in sixteen (4, 5) of the roots on the FMA pipe; other shapes
// take them as 0 and 1.
constexpr int SCAN_VARIANTS = 6;
// Variants 6 and 7: the pruned scan (scan_pruned.cuh) with half / all of rows_for_dim.
constexpr int SCAN_VARIANTS_ALL = 8;
__host__ __device__ constexpr int rows_for_variant(int D, int v) {
    return (v & 1) == 0 ? rows_for_dim(D) : (rows_for_dim(D) / 2 > 0 ? rows_for_dim(D) / 2 : 1);
}
__host__ __device__ constexpr int fsr_for_variant(int v) { return v >= 4 ? 4 : (v >= 2 ? 2 : 0); }
// Shapes with the FMA-pipe square-root variants: L2 with 1..6 coordinates, some constrained.
__host__ __device__ constexpr bool fma_sqrt_shape(int norm, int C, int U) {
    return norm == LIP_L2 && C >= 1 && C + U <= 6;
}

// Exact instantiations: every (C, U) with 1 <= C + U <= 10, and unconstrained D up to 16
// (EXACT_DMAX).  Wider shapes (up to D_MAX = 32) take the generic kernel: the exact body
// holds a whole group's channels and the duplicated query coordinates in registers, which
// does not fit beyond 16 coordinates.
constexpr int EXACT_DMAX = 16;
__host__ __device__ constexpr bool exact_shape_available(int C, int U) {
    return (C + U >= 1 && C + U <= 10 && C >= 0 && U >= 0) || (C == 0 && U >= 11 && U <= EXACT_DMAX);
}

// Layout dimension of the generic kernel for d coordinates (zero-padded).
__host__ __device__ constexpr int generic_dim(int d) {
    return d <= 2 ? 2 : (d <= 4 ? 4 : (d <= 8 ? 8 : (d <= 12 ? 12 : (d <= 16 ? 16 : (d <= 24 ? 24 : 32)))));
}
// Queries per thread of the generic kernel (each holds DP coordinates in registers).
__host__ __device__ constexpr int generic_rows(int DP) { return DP <= 16 ? 2 : 1; }

using ScanLaunchFn = cudaError_t (*)(const ScanParams&, int gx, int gy, cudaStream_t);

struct ScanKernelInfo {
    ScanLaunchFn launch = nullptr;
    const void* kernel = nullptr;   // for occupancy queries
    int rows = 0;                   // queries per thread
    int nch = 0;                    // channels per group
};

ScanKernelInfo scan_exact_info(int norm, int C, int U, int variant = 0);
ScanKernelInfo scan_generic_info(int elem_bytes, int norm, int dl);

}  // namespace lip
