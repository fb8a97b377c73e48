// Tensor-core form of the unmasked L2 envelope scan (LIP_TC_TF32 and LIP_TC_BF16).
//
// Squared distance as products: with q^ = M w (q - c), x^ = M w (x - c) (c = the centre
// of the data's bounding box; distances do not depend on it),
//     s(q, x) = |q^|^2 + |x^|^2 - 2 q^.x^ = a . b + n_a . n_b,
//     a = -2 q^, b = x^ (K = d padded to 8 or 16),
//     n_a = [1, .., 1, pieces of |q^|^2],  n_b = [pieces of |x^|^2, 1, .., 1]
// (the norm block: one more MMA of 32 bytes of K, so the two norms no longer widen K).
// Every operand is split v = hi + lo with hi the value truncated to TF32 and lo the FP32
// remainder, and a . b runs as three tcgen05.mma kind::tf32 passes a_hi.b_hi + a_hi.b_lo +
// a_lo.b_hi accumulating in FP32 in TMEM; the norm block holds the norms' hi and lo.
//
// BF16 (LIP_TC_BF16): K = 16, every operand split into three bf16 pieces v = h + m + l (each
// the bf16 rounding of the remainder; |v - h - m - l| <= 2^-24 |v|), and a . b =
// hh + hm + mh + hl + lh + mm (products of bf16 pieces are exact in FP32) runs as six
// tcgen05.mma kind::f16 passes with both operands bf16; the norm block holds h, m, l.
//
// Error bound used to prune (conservative, per query): |s~ - s| <= eps = C (|q^| + R)^2,
// R = max_k |x^_k|.  Every term of the products is bounded by S = sum_j |a_j b_j| + |x^|^2
// + |q^|^2 <= (|q^| + R)^2:
//   * TF32: 3 * 2^-20 S for the dropped and truncated split terms (the norms' lo pieces are
//     truncated to TF32 too), plus (3K + 4) * 2^-23 S for FP32 accumulation of 3K + 4
//     products (52 at K = 16);
//   * BF16: 2^-22 S for the dropped products and the representation error, plus
//     (6K + 6) * 2^-23 S (102 products at K = 16);
//   * the FP32 rounding of the inputs and of the two norms: <= 2^-23 (|q^| + R)^2 + 2^-24 S.
// Together at most 9.3e-6 (TF32) and 1.3e-5 (BF16) times (|q^| + R)^2; C = 1.3e-5 and
// 1.7e-5.
// Then |sqrt(s~+) - sqrt(s)| <= eps / sqrt(max(s~+, eps)); for a 32-point chunk the
// smallest s~ in it bounds every pair.  With the FP32 evaluation error of the bounds,
//   delta_c = 1.001 eps rsqrt(max(min_chunk s~, eps)) + 2^-19 (max|y| + |q^| + R).
// A chunk can hold the exact argmin only if min_chunk v~ - delta_c <= U, where
// U = min over chunks of (min_chunk v~ + delta_c) is an upper bound of H_up; the same
// holds mirrored for H_lo.  Candidate chunks are kept per query (8 per list, one list
// per column slice), then rescreened from the caller's data: one warp per query
// evaluates each candidate chunk in FP32 and re-evaluates in FP64 only the points within
// the FP32 error bound of the chunk's extremum, so the result is the FP64 argmin/argmax.
// A query whose list overflows is recomputed by the plain FP32 scan.
//
// Kernel: one CTA per 128-query tile, 18 warps.  Warp 0 streams 256-point data tiles
// (pre-tiled operand pieces, norm block and y, one 1-D bulk copy each) into a 4-stage ring; warp 1
// owns TMEM (512 columns = two 128 x 256 FP32 accumulators) and issues the MMAs; warps
// 2..17 are the epilogue: each reads one 32-lane quarter of the accumulator rows (one
// query per thread) over a quarter of the columns with tcgen05.ld, tests each 32-column
// chunk's smallest s~ against the running bounds and, only where the chunk
// may hold an extremum, takes sqrt(|s~|), forms y +- sqrt and keeps the chunk extrema and
// candidate lists.  Every wait is bounded.
// (sqrt(|s~|) needs no clamp: s~ < 0 only when s < eps, and then both roots are below
// sqrt(eps), which delta already covers.)
#include <cstdio>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "launch.h"

namespace lip {

constexpr int TC_M = 128;
constexpr int TC_N = 256;
constexpr int TC_STAGES = 4;
constexpr int TC_CAP = 8;
// Epilogue warps: 4 lane quarters x PARTS column slices (PARTS = 2 or 4, a launch variant);
// each (query, bound) keeps one candidate list per column slice.
constexpr int TC_MAX_PARTS = 4;
__host__ __device__ constexpr int tc_threads(int parts) { return 32 * (2 + 4 * parts); }
// Operand formats: the TF32 two-piece split, the BF16 three-piece split and the FP16
// two-piece split (tc_fmt in launch.h).
constexpr float TC_C_EPS_TF32 = 1.3e-5f;   // TF32 split (bound 9.3e-6)
constexpr float TC_C_EPS_BF16 = 1.7e-5f;   // BF16 three-piece split (bound 1.3e-5)
constexpr float TC_C_EPS_FP16 = 1.0e-5f;   // FP16 two-piece split (bound 7.2e-6)
// The error bound of |s~ - s| / (|q^| + R)^2 as a function of K (the derivation's terms:
// the split's dropped products, K-proportional FP32 accumulation, the input roundings).
__host__ __device__ constexpr double tc_eps_bound(int fmt, int K) {
    return fmt == TC_BF16 ? 0x1p-22 + (6.0 * K + 6.0) * 0x1p-23 + 0x1p-23 + 0x1p-24
         : fmt == TC_FP16 ? 3 * 0x1p-22 + (3.0 * K + 2.0) * 0x1p-23 + 0x1p-24 + 0x1p-23 + 0x1p-24
                          : 3 * 0x1p-20 + (3.0 * K + 4.0) * 0x1p-23 + 0x1p-23 + 0x1p-24;
}
// The constant used for eps: the K = 16 constant above (about 1.4 times its bound), and for
// wider K (d above 16) the same constant scaled by the bound's growth with K.
__host__ __device__ constexpr float tc_c_eps(int fmt, int K) {
    const float c16 = fmt == TC_BF16 ? TC_C_EPS_BF16 : (fmt == TC_FP16 ? TC_C_EPS_FP16 : TC_C_EPS_TF32);
    return K <= 16 ? c16 : (float)(c16 * (tc_eps_bound(fmt, K) / tc_eps_bound(fmt, 16)));
}

struct TcRec {      // candidate list of one (query, bound, column quarter)
    float U;        // upper bound of H_up (bound 0) or lower bound of H_lo (bound 1)
    int n;          // entries, -1 = overflow
    int id[TC_CAP];
    float L[TC_CAP];
};

// Operand geometry per format: TF32 keeps 2 pieces of 4-byte elements with K a multiple
// of 8; BF16 keeps 3 pieces and FP16 2 pieces of 2-byte elements with K a multiple of 16.
// Either way one MMA consumes 32 bytes of K per row (two 8-row x 16-byte core matrices).
__host__ __device__ constexpr int tc_k_for_dim(int d, int fmt) {
    return fmt == TC_TF32 ? ((d + 7) / 8) * 8 : ((d + 15) / 16) * 16;
}
__host__ __device__ constexpr int tc_pieces(int fmt) { return fmt == TC_BF16 ? 3 : 2; }
__host__ __device__ constexpr int tc_esz(int fmt) { return fmt == TC_TF32 ? 4 : 2; }
// piece products per pair: TF32 and FP16 hi.hi + hi.lo + lo.hi; BF16 hh + hm + mh + hl + lh + mm
__host__ __device__ constexpr int tc_npass(int fmt) { return fmt == TC_BF16 ? 6 : 3; }
__host__ __device__ constexpr uint32_t tc_sbo_bytes(int row_bytes) { return (uint32_t)(row_bytes / 16) * 128u; }
// The norm block: one more K-major operand of 32 bytes per row (one MMA's K), holding the
// pieces of |x^|^2 against ones (B) and ones against the pieces of |q^|^2 (A).
constexpr int TC_NORM_ROW = 32;
constexpr int TC_CHUNKS = TC_N / 32;       // 32-point chunks per tile
// a data tile: the pieces, the norm block, y of its 256 points, then (min y, max y) of each
// chunk (NaN when it holds no datum)
__host__ __device__ constexpr int tc_tile_bytes(int K, int fmt) {
    return tc_pieces(fmt) * TC_N * K * tc_esz(fmt) + TC_N * TC_NORM_ROW + TC_N * 4 + TC_CHUNKS * 8;
}
// a tile's slot in the shared-memory ring (1024-byte aligned operands in every stage)
__host__ __device__ constexpr int tc_stage_bytes(int K, int fmt) { return (tc_tile_bytes(K, fmt) + 1023) / 1024 * 1024; }
__host__ __device__ constexpr int tc_a_bytes(int K, int fmt) {
    return tc_pieces(fmt) * TC_M * K * tc_esz(fmt) + TC_M * TC_NORM_ROW;
}
// Stages of the data-tile ring: TC_STAGES where they fit in the 227 KB of shared memory next
// to the A operand (every K up to 16, and FP16 at 32); fewer for the widest tiles (TF32 at
// K = 24 and BF16 at 32 keep 3, TF32 at 32 keeps 2).
constexpr int TC_SMEM_BYTES = 227 * 1024 - 1024;    // a margin for the static barriers
__host__ __device__ constexpr int tc_stages(int K, int fmt) {
    return (TC_SMEM_BYTES - tc_a_bytes(K, fmt)) / tc_stage_bytes(K, fmt) < TC_STAGES
               ? (TC_SMEM_BYTES - tc_a_bytes(K, fmt)) / tc_stage_bytes(K, fmt)
               : TC_STAGES;
}

// byte offset of the element at row r, byte kb along K, in a canonical no-swizzle K-major
// operand whose rows hold row_bytes of K (core matrices of 8 rows x 16 bytes)
__host__ __device__ inline uint32_t tc_off(int r, int kb, int row_bytes) {
    return (uint32_t)(r / 8) * tc_sbo_bytes(row_bytes) + (uint32_t)(kb / 16) * 128u + (uint32_t)(r % 8) * 16u +
           (uint32_t)(kb % 16);
}

// Writes the pieces of v at (r, k) of a piece-major operand block (piece p at p * piece_bytes).
template <int FMT>
__device__ __forceinline__ void tc_store_pieces(char* base, int piece_bytes, int r, int k, int K, float v) {
    if (FMT == TC_FP16) {
        const __half h = __float2half_rn(v);
        const __half l = __float2half_rn(v - __half2float(h));
        const uint32_t off = tc_off(r, k * 2, K * 2);
        *reinterpret_cast<__half*>(base + off) = h;
        *reinterpret_cast<__half*>(base + piece_bytes + off) = l;
    } else if (FMT == TC_BF16) {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        const float r1 = v - __bfloat162float(h);
        const __nv_bfloat16 m = __float2bfloat16_rn(r1);
        const float r2 = r1 - __bfloat162float(m);
        const __nv_bfloat16 l = __float2bfloat16_rn(r2);
        const uint32_t off = tc_off(r, k * 2, K * 2);
        *reinterpret_cast<__nv_bfloat16*>(base + off) = h;
        *reinterpret_cast<__nv_bfloat16*>(base + piece_bytes + off) = m;
        *reinterpret_cast<__nv_bfloat16*>(base + 2 * piece_bytes + off) = l;
    } else {
        const float hi = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);   // truncated to TF32
        const uint32_t off = tc_off(r, k * 4, K * 4);
        *reinterpret_cast<float*>(base + off) = hi;
        *reinterpret_cast<float*>(base + piece_bytes + off) = v - hi;
    }
}

// Writes row r of a norm block.  B rows (ones_first false): the pieces of nv, then ones
// matching the A side's norm pieces.  A rows (ones_first true): ones matching the B side's
// pieces, then the pieces of nv.  The rest of the row is zero.  TF32: 2 pieces of 4 bytes
// (hi truncated, FP32 remainder); BF16: 3 pieces of 2 bytes.  FP16: 2 pieces of 2 bytes,
// and only |x^|^2 goes through the block (|q^|^2 would leave the f16 range for distant
// queries; the epilogue adds it), so A rows are [1, 1, 0, ..].
template <int FMT>
__device__ __forceinline__ void tc_store_norm(char* base, int r, float nv, bool ones_first) {
    constexpr int np = tc_pieces(FMT), per = TC_NORM_ROW / tc_esz(FMT);
    constexpr int nq = FMT == TC_FP16 ? 0 : np;          // pieces of the A side's norm
    float pc[3] = {0.f, 0.f, 0.f};
    if (FMT == TC_BF16) {
        const __nv_bfloat16 h = __float2bfloat16_rn(nv);
        const float r1 = nv - __bfloat162float(h);
        const __nv_bfloat16 m = __float2bfloat16_rn(r1);
        const float r2 = r1 - __bfloat162float(m);
        pc[0] = __bfloat162float(h);
        pc[1] = __bfloat162float(m);
        pc[2] = __bfloat162float(__float2bfloat16_rn(r2));
    } else if (FMT == TC_FP16) {
        pc[0] = __half2float(__float2half_rn(nv));
        pc[1] = __half2float(__float2half_rn(nv - pc[0]));
    } else {
        pc[0] = __uint_as_float(__float_as_uint(nv) & 0xFFFFE000u);
        pc[1] = nv - pc[0];
    }
    for (int k = 0; k < per; ++k) {
        float v = 0.f;
        if (ones_first) {
            if (k < np) v = 1.f;
            else if (k < np + nq) v = pc[k - np];
        } else {
            if (k < np) v = pc[k];
            else if (k < np + nq) v = 1.f;
        }
        const uint32_t off = tc_off(r, k * tc_esz(FMT), TC_NORM_ROW);
        if (FMT == TC_BF16) *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(v);
        else if (FMT == TC_FP16) *reinterpret_cast<__half*>(base + off) = __float2half_rn(v);
        else *reinterpret_cast<float*>(base + off) = v;
    }
}

// --------------------------------------------------------------- data preparation

struct TcPrepParams {
    const float* X0;      // caller's data [N][d]
    const float* y0;
    int64_t N;
    int d, K;
    double scale[D_MAX];  // M * w_j (caller's coordinate order; unmasked, so no mirroring)
    const float2* bounds; // [d] (min, max) of the data's finite coordinates (the centre is their midpoint)
    unsigned* maxbits;    // [2]: float bits of R and of max|y|
    char* tiles;          // [ntiles][tile_bytes]
    int64_t ntiles;
    const int* perm;      // [N] position -> data index (tiles are in position order)
    float* Xs;            // [N][d] position-ordered copy of the data
    float* ys;            // [N]
};

// The centre of the scaled coordinates: the midpoint of the data's bounding box, the same
// double for the data and the query pieces.
__device__ __forceinline__ double tc_centre(const float2 b, double scale) {
    return scale * 0.5 * ((double)b.x + (double)b.y);
}

// FP16 operands are scaled by 2^k (exactly, a power of two) with k chosen from the box's
// half-diagonal Rb >= max |x^|: Rb 2^k lies in [64, 128), so every centred data coordinate
// stays below 128 and |x^|^2 below 2^14 in the f16 range; queries up to 2^14 per coordinate
// fit (-2 q^ <= 2^15).  k = 0 for a box of one point.
constexpr float TC_F16_QMAX = 16384.f;
__device__ __forceinline__ int tc_f16_shift(const float2* bounds, const double* scale, int d) {
    double r2 = 0.0;
    for (int j = 0; j < d; ++j) {
        const double h = 0.5 * scale[j] * ((double)bounds[j].y - (double)bounds[j].x);
        r2 += h * h;
    }
    if (!(r2 > 0.0)) return 0;
    int e;
    frexp(sqrt(r2), &e);                   // Rb = m 2^e, m in [0.5, 1): Rb 2^(7 - e) in [64, 128)
    const int k = 7 - e;
    return k < -60 ? -60 : (k > 60 ? 60 : k);
}

// One thread per (padded) position: the row of the B pieces, of the norm block and y of
// the datum at that position, in the tile layout, and the position-ordered copy of its
// row.  A padding position has zero rows (s~ = 0) and y = NaN.
template <int FMT>
__global__ void tc_build_b_kernel(const TcPrepParams P) {
    __shared__ double f_s;                 // FP16: the operand scale 2^k, once per block
    __shared__ double c_s[D_MAX];          // the centre, once per block
    if (FMT == TC_FP16 && threadIdx.x == 0) f_s = ldexp(1.0, tc_f16_shift(P.bounds, P.scale, P.d));
    if (threadIdx.x < P.d) c_s[threadIdx.x] = tc_centre(P.bounds[threadIdx.x], P.scale[threadIdx.x]);
    __syncthreads();
    const double f = FMT == TC_FP16 ? f_s : 1.0;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P.ntiles * TC_N) return;
    const int64_t t = k / TC_N;
    const int r = (int)(k % TC_N);
    char* tile = P.tiles + t * (int64_t)tc_tile_bytes(P.K, FMT);
    const int piece = TC_N * P.K * tc_esz(FMT);
    char* norm = tile + tc_pieces(FMT) * piece;
    float* yv = reinterpret_cast<float*>(norm + TC_N * TC_NORM_ROW);
    float b[D_MAX];
    for (int j = 0; j < P.K; ++j) b[j] = 0.f;
    float yy = __int_as_float(0x7fc00000);
    bool real = false;
    unsigned rbits = 0u, ybits = 0u;
    if (k < P.N) {
        const int64_t src = P.perm[k];
        double n2 = 0.0;
        for (int j = 0; j < P.d; ++j) {
            const float x = P.X0[src * P.d + j];
            P.Xs[k * P.d + j] = x;
            const float xh = (float)(P.scale[j] * (double)x - c_s[j]);
            b[j] = (float)((double)xh * f);
            n2 += (double)xh * (double)xh;
        }
        tc_store_norm<FMT>(norm, r, (float)(n2 * f * f), false);
        real = true;
        yy = P.y0[src];
        P.ys[k] = yy;
        rbits = __float_as_uint((float)sqrt(n2));
        ybits = __float_as_uint(fabsf(yy));
    }
    // R and max |y|: one atomic per warp (non-negative floats order as their bits)
    const unsigned act = __activemask();
    rbits = __reduce_max_sync(act, rbits);
    ybits = __reduce_max_sync(act, ybits);
    if (threadIdx.x % 32 == __ffs(act) - 1) {
        atomicMax(&P.maxbits[0], rbits);
        atomicMax(&P.maxbits[1], ybits);
    }
    for (int j = 0; j < P.K; ++j) tc_store_pieces<FMT>(tile, piece, r, j, P.K, b[j]);
    if (!real)
        for (int kb = 0; kb < TC_NORM_ROW; kb += 4) *reinterpret_cast<float*>(norm + tc_off(r, kb, TC_NORM_ROW)) = 0.f;
    yv[r] = yy;
}

// (min y, max y) of each 32-position chunk (NaN if it holds no datum), the epilogue's chunk
// bounds, written at the end of the chunk's tile.
__global__ void tc_chunk_bounds_kernel(const float* ys, int64_t N, int64_t nchunks, char* tiles, int tile_bytes) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nchunks) return;
    float2* cb = reinterpret_cast<float2*>(tiles + (c / TC_CHUNKS) * (int64_t)tile_bytes + tile_bytes - TC_CHUNKS * 8) +
                 c % TC_CHUNKS;
    const float nan = __int_as_float(0x7fc00000);
    float lo = nan, hi = nan;
    for (int64_t k = c * 32; k < c * 32 + 32 && k < N; ++k) {
        lo = fminf(lo, ys[k]);        // NaN operands are ignored
        hi = fmaxf(hi, ys[k]);
    }
    *cb = make_float2(lo, hi);
}

struct TcQueryParams {
    const float* Q;        // caller's queries [nq][d]
    const int* qperm;      // [nq] position -> query index (tiles are in position order)
    int64_t nq;
    int d, K;
    double scale[D_MAX];
    const float2* bounds;  // [d] the data's bounding box (the centre is its midpoint)
    int64_t N;
    const unsigned* maxbits;
    char* atiles;          // [nqt][a_bytes]: the A pieces
    float4* qc;            // [nq] per-query constants of the scan (below)
};

// Per-query constants of the scan, one float4: x = eps, y = eps_v (the error bounds), and
// for FP16 z = |q^|^2 (added in the epilogue) and w = 2^-2k (the products' unscaling; w < 0
// marks a query outside the f16 range, which goes through the fallback).  TF32 and BF16:
// z = 0, w = 1.

// One thread per (padded) query: its row of the A pieces and its constants.
template <int FMT>
__global__ void tc_build_a_kernel(const TcQueryParams P) {
    __shared__ int ks_s;                   // FP16: the operand scale's exponent, once per block
    __shared__ double c_s[D_MAX];          // the centre, once per block
    if (FMT == TC_FP16 && threadIdx.x == 0) ks_s = tc_f16_shift(P.bounds, P.scale, P.d);
    if (threadIdx.x < P.d) c_s[threadIdx.x] = tc_centre(P.bounds[threadIdx.x], P.scale[threadIdx.x]);
    __syncthreads();
    const int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nqp = (P.nq + TC_M - 1) / TC_M * TC_M;
    if (qi >= nqp) return;
    const int64_t t = qi / TC_M;
    const int r = (int)(qi % TC_M);
    char* at = P.atiles + t * (int64_t)tc_a_bytes(P.K, FMT);
    const int piece = TC_M * P.K * tc_esz(FMT);
    float a[D_MAX];
    for (int j = 0; j < P.K; ++j) a[j] = 0.f;
    char* norm = at + tc_pieces(FMT) * piece;
    bool real = false;
    if (qi < P.nq) {
        const int64_t src = P.qperm[qi];
        const int ks = FMT == TC_FP16 ? ks_s : 0;
        const double f = ldexp(1.0, ks);
        double n2 = 0.0;
        bool inside = true;
        for (int j = 0; j < P.d; ++j) {
            const float qh = (float)(P.scale[j] * (double)P.Q[src * P.d + j] - c_s[j]);
            const float qs = (float)((double)qh * f);
            if (FMT == TC_FP16 && fabsf(qs) > TC_F16_QMAX) inside = false;   // also +-inf; NaN stays
            a[j] = -2.f * qs;
            n2 += (double)qh * (double)qh;
        }
        const double R = (double)__uint_as_float(P.maxbits[0]);
        const double Y = (double)__uint_as_float(P.maxbits[1]);
        const double nq = sqrt(n2);
        const float eps = (float)((double)tc_c_eps(FMT, P.K) * (nq + R) * (nq + R));
        const float epsv = (float)(ldexp(1.0, -19) * (Y + nq + R));
        const float usc = (float)ldexp(1.0, -2 * ks);
        P.qc[qi] = make_float4(eps, epsv, FMT == TC_FP16 ? (float)n2 : 0.f, inside ? usc : -usc);
        if (!inside)
            for (int j = 0; j < P.K; ++j) a[j] = 0.f;
        tc_store_norm<FMT>(norm, r, (float)n2, true);
        real = true;
    }
    for (int j = 0; j < P.K; ++j) tc_store_pieces<FMT>(at, piece, r, j, P.K, a[j]);
    if (!real)
        for (int kb = 0; kb < TC_NORM_ROW; kb += 4) *reinterpret_cast<float*>(norm + tc_off(r, kb, TC_NORM_ROW)) = 0.f;
}

// --------------------------------------------------------------- tcgen05 helpers

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, int row_bytes) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;                      // leading (K-direction) byte offset
    d |= (uint64_t)((tc_sbo_bytes(row_bytes) >> 4) & 0x3FFFu) << 32;   // stride between 8-row groups
    d |= (uint64_t)1 << 46;                                 // descriptor version of sm_100
    return d;                                               // no swizzle, base offset 0
}

template <int FMT>
__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    if (FMT != TC_TF32)   // both operands bf16, or both f16 (the instruction descriptor says which)
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                     ::"r"(dtmem), "l"(da), "l"(db), "r"(idesc), "r"(acc) : "memory");
    else
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                     ::"r"(dtmem), "l"(da), "l"(db), "r"(idesc), "r"(acc) : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                   "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// Two adjacent 32-column loads issued back to back, then one wait.
__device__ __forceinline__ void tmem_ld32x2(uint32_t taddr, float (&v)[2][32]) {
    uint32_t r[64];
#define LIP_TMEM_LD32(OFF, BASE)                                                                                   \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"    \
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                         \
                 : "=r"(r[BASE + 0]), "=r"(r[BASE + 1]), "=r"(r[BASE + 2]), "=r"(r[BASE + 3]), "=r"(r[BASE + 4]),    \
                   "=r"(r[BASE + 5]), "=r"(r[BASE + 6]), "=r"(r[BASE + 7]), "=r"(r[BASE + 8]), "=r"(r[BASE + 9]),    \
                   "=r"(r[BASE + 10]), "=r"(r[BASE + 11]), "=r"(r[BASE + 12]), "=r"(r[BASE + 13]),                  \
                   "=r"(r[BASE + 14]), "=r"(r[BASE + 15]), "=r"(r[BASE + 16]), "=r"(r[BASE + 17]),                  \
                   "=r"(r[BASE + 18]), "=r"(r[BASE + 19]), "=r"(r[BASE + 20]), "=r"(r[BASE + 21]),                  \
                   "=r"(r[BASE + 22]), "=r"(r[BASE + 23]), "=r"(r[BASE + 24]), "=r"(r[BASE + 25]),                  \
                   "=r"(r[BASE + 26]), "=r"(r[BASE + 27]), "=r"(r[BASE + 28]), "=r"(r[BASE + 29]),                  \
                   "=r"(r[BASE + 30]), "=r"(r[BASE + 31])                                                            \
                 : "r"(taddr + (OFF)))
    LIP_TMEM_LD32(0, 0);
    LIP_TMEM_LD32(32, 32);
#undef LIP_TMEM_LD32
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        v[0][j] = __uint_as_float(r[j]);
        v[1][j] = __uint_as_float(r[32 + j]);
    }
}

__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

struct TcScanParams {
    const char* atiles;
    const char* btiles;
    const float4* qc;      // [nq] per-query constants (eps, eps_v, FP16: |q^|^2 and 2^-2k)
    int64_t nq;
    int64_t ntiles;
    TcRec* rec;            // [nq positions][2 bounds][TC_MAX_PARTS column slices]
    unsigned* err;
    int64_t nqt;           // query tiles; CTA c takes tiles c, c + grid, ... (one per round)
    // Soft lockstep of the CTAs of a round (lag > 0): arrive[round][c] counts the CTAs whose
    // producer has reached data chunk c (ctiles tiles each) of that round; a producer waits,
    // for at most THROTTLE_NS, until every CTA of its round has reached chunk c - lag.
    int* arrive;           // [rounds][nch], zeroed before the launch
    int nch;
    int ctiles;
    int lag;
    int wave;              // SMs: query tile qt belongs to round qt / wave (its sweep direction)
};

constexpr unsigned long long TC_THROTTLE_NS = 2000000;     // 2 ms, then the CTA stops waiting

// The soft lockstep's wait: true when *cnt >= need; false (stop waiting for the rest of the
// kernel) after TC_THROTTLE_NS.  Only the order of the data tiles' L2 reuse depends on it,
// never a result.
__device__ __forceinline__ bool tc_throttle(const int* cnt, int need) {
    if (*reinterpret_cast<const volatile int*>(cnt) >= need) return true;
    const unsigned long long t0 = globaltimer();
    for (;;) {
        __nanosleep(256);
        if (*reinterpret_cast<const volatile int*>(cnt) >= need) return true;
        if (globaltimer() - t0 > TC_THROTTLE_NS) return false;
    }
}

// Candidate list append with compaction when full (entries that can no longer qualify
// are dropped; the bound only tightens).  upper = true for H_up (keep L <= U).
__device__ __forceinline__ void tc_append(TcRec* R, int& n, int id, float L, float bound, bool upper) {
    if (n < 0) return;
    if (n == TC_CAP) {
        int m = 0;
        for (int e = 0; e < TC_CAP; ++e) {
            const float le = R->L[e];
            if (upper ? (le <= bound) : (le >= bound)) {
                R->id[m] = R->id[e];
                R->L[m] = le;
                ++m;
            }
        }
        n = m;
        if (n == TC_CAP) { n = -1; return; }
    }
    R->id[n] = id;
    R->L[n] = L;
    ++n;
}

template <int K, int PARTS, int FMT>
__global__ void __launch_bounds__(tc_threads(PARTS), 1) tc_scan_kernel(const TcScanParams P) {
    constexpr int ST = tc_stages(K, FMT);                // the ring's stages at this K
    static_assert(ST >= 2, "the data-tile ring needs two stages");
    constexpr int EPI_WARPS = 4 * PARTS;
    constexpr int TILE_BYTES = tc_tile_bytes(K, FMT), STAGE_BYTES = tc_stage_bytes(K, FMT);
    constexpr int A_BYTES = tc_a_bytes(K, FMT);
    constexpr int ROW_BYTES = K * tc_esz(FMT);
    constexpr int KS = ROW_BYTES / 32;                  // MMAs per pass (32 bytes of K each)
    constexpr int A_PIECE = TC_M * ROW_BYTES, B_PIECE = TC_N * ROW_BYTES;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;                               // A_hi, A_lo
    unsigned char* sB = smem + A_BYTES;                     // ST tiles
    __shared__ __align__(8) uint64_t a_full, a_empty, b_full[ST], b_empty[ST], acc_full[2], acc_empty[2];
    __shared__ uint32_t tmem_base;

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t T = P.ntiles;
    // Persistent CTAs (one per SM, a cooperative launch): round r of CTA c scans query tile
    // c + r * grid against every data tile (with a grid of one CTA per query tile, each CTA
    // runs one round).  Sweep direction: even rounds (query tiles qt with qt / SMs even)
    // read the data tiles in increasing order, odd rounds in decreasing order, so a round
    // starts on the tiles the last one read most recently (still in L2).  With P.lag > 0 the producers of
    // a round keep within lag chunks of one another (tc_throttle), so the round's CTAs read
    // each data tile from L2 at about the same time and DRAM sees the tile set about once
    // per round.  Tile order does not change the results: the candidate chunks are collected
    // in any order and the rescreen takes the exact extremum with the lowest index.
    const int grid = (int)gridDim.x, nqt = (int)P.nqt;   // nq < 2^31: fewer than 2^24 query tiles

    if (threadIdx.x == 0) {
        mbar_init(&a_full, 1);
        mbar_init(&a_empty, 1);
        for (int s = 0; s < ST; ++s) {
            mbar_init(&b_full[s], 1);
            mbar_init(&b_empty[s], 1 + EPI_WARPS);         // MMA commit + epilogue warps
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], EPI_WARPS);
        }
        fence_mbar_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tb = tmem_base;

    if (warp == 0) {
        // ------------------------------------------------ producer
        if (lane == 0) {
            uint32_t g = 0;                                // data tiles issued by this CTA (< 2^31)
            uint32_t na = 0;                               // query tiles issued
            bool ok = true, throttle = true;
            for (int qt = (int)blockIdx.x, r = 0; ok && qt < nqt; qt += grid, ++r) {
                if (r > 0 && !mbar_wait_bounded(&a_empty, (uint32_t)((r - 1) & 1), P.err)) {
                    ok = false;
                    break;
                }
                mbar_expect_tx(&a_full, A_BYTES);
                bulk_g2s(sA, P.atiles + qt * (int64_t)A_BYTES, A_BYTES, &a_full);
                ++na;
                const bool rev = ((qt / P.wave) & 1) != 0;
                const int members = nqt - r * grid < grid ? nqt - r * grid : grid;
                int* row = P.arrive + (int64_t)r * P.nch;
                for (int64_t t = 0; t < T; ++t, ++g) {
                    if (P.lag > 0 && t % P.ctiles == 0) {
                        // every CTA counts itself in, also after it has stopped waiting
                        const int c = (int)(t / P.ctiles);
                        atomicAdd(row + c, 1);
                        if (throttle && c >= P.lag) throttle = tc_throttle(row + c - P.lag, members);
                    }
                    const int s = (int)(g % ST);
                    if (g >= (uint32_t)ST && !mbar_wait_bounded(&b_empty[s], (g / ST - 1) & 1u, P.err)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&b_full[s], TILE_BYTES);
                    const int64_t tt = rev ? T - 1 - t : t;
                    bulk_g2s(sB + (size_t)s * STAGE_BYTES, P.btiles + tt * (int64_t)TILE_BYTES, TILE_BYTES, &b_full[s]);
                }
            }
            // wait (bounded) for the copies still in flight before leaving
            const uint32_t first = g > (uint32_t)ST ? g - ST : 0u;
            for (uint32_t u = first; u < g; ++u)
                mbar_wait_bounded(&b_full[u % ST], (u / ST) & 1u, ok ? P.err : nullptr);
            if (na > 0) mbar_wait_bounded(&a_full, (na - 1) & 1u, nullptr);
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            // D = FP32 (bits 4-5); A and B formats (bits 7-9, 10-12): TF32 = 2 in kind::tf32,
            // F16 = 0 and BF16 = 1 in kind::f16; K-major A and B; N / 8 and M / 16
            const uint32_t fmt = FMT == TC_BF16 ? 1u : (FMT == TC_FP16 ? 0u : 2u);
            const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                                   ((uint32_t)(TC_M >> 4) << 24);
            const uint32_t a0 = smem_u32(sA);
            uint32_t g = 0;
            bool ok = true;
            for (int qt = (int)blockIdx.x, r = 0; ok && qt < nqt; qt += grid, ++r) {
                if (!mbar_wait_bounded(&a_full, (uint32_t)(r & 1), P.err)) break;
                for (int64_t t = 0; t < T; ++t, ++g) {
                    const int s = (int)(g % ST), b = (int)(g & 1);
                    if (!mbar_wait_bounded(&b_full[s], (g / ST) & 1u, P.err) ||
                        (g >= 2 && !mbar_wait_bounded(&acc_empty[b], (g / 2 - 1) & 1u, P.err))) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t b0 = smem_u32(sB + (size_t)s * STAGE_BYTES);
                    const uint32_t d = tb + (uint32_t)b * TC_N;
                    // piece pairs: TF32 and FP16 hi.hi, hi.lo, lo.hi; BF16 hh, hm, mh, hl, lh, mm
                    constexpr int NPASS = tc_npass(FMT);
                    constexpr int PA[6] = {0, 0, 1, 0, 2, 1}, PB[6] = {0, 1, 0, 2, 0, 1};
#pragma unroll
                    for (int ps = 0; ps < NPASS; ++ps) {
                        const uint32_t ap = a0 + PA[ps] * A_PIECE, bp = b0 + PB[ps] * B_PIECE;
#pragma unroll
                        for (int ks = 0; ks < KS; ++ks)
                            tc_mma<FMT>(d, tc_desc(ap + ks * 256, ROW_BYTES), tc_desc(bp + ks * 256, ROW_BYTES), idesc,
                                       (ps > 0 || ks > 0) ? 1u : 0u);
                    }
                    // the norm block: |x^|^2 (+ |q^|^2 but for FP16) in one more MMA of 32 bytes of K
                    tc_mma<FMT>(d, tc_desc(a0 + tc_pieces(FMT) * A_PIECE, TC_NORM_ROW),
                               tc_desc(b0 + tc_pieces(FMT) * B_PIECE, TC_NORM_ROW),
                               idesc, 1u);
                    tc_commit(&b_empty[s]);
                    tc_commit(&acc_full[b]);
                }
                if (ok) tc_commit(&a_empty);               // the query tile is no longer read
            }
            // the last MMAs must finish before TMEM is released
            if (g > 0) mbar_wait_bounded(&acc_full[(g - 1) & 1], ((g - 1) / 2) & 1u, nullptr);
        }
    } else {
        // ------------------------------------------------ epilogue (warps 2 .. 2 + EPI_WARPS)
        const int quarter = warp % 4, part = (warp - 2) / 4;
        const float INF = __int_as_float(0x7f800000);
        const int T32 = (int)T;                            // N < 2^31, so T < 2^23
        uint32_t g = 0;                                    // data tiles consumed by this CTA
        bool ok = true;
#pragma unroll 1
        for (int qt = (int)blockIdx.x, r = 0; ok && qt < nqt; qt += grid, ++r) {
        const bool rev = ((qt / P.wave) & 1) != 0;
        const int64_t qi = (int64_t)qt * TC_M + quarter * 32 + lane;
        const bool valid = qi < P.nq;
        const float4 qc = valid ? P.qc[qi] : make_float4(1.f, 1.f, 0.f, 1.f);
        // a zero bound (M = 0) must not turn eps * rsqrt(0) into NaN
        const float eps = fmaxf(qc.x, 1e-30f), epsv = qc.y;
        // FP16: s~ = |q^|^2 + 2^-2k (product); a query outside the f16 range (w < 0) keeps
        // overflowed lists, so it goes through the fallback
        const float nq2 = qc.z, usc = fabsf(qc.w);
        const bool act = valid && qc.w > 0.f;
        // the H_up list of this query and column slice; the H_lo list follows TC_MAX_PARTS later
        TcRec* Ru = P.rec + (valid ? ((qi * 2 + 0) * TC_MAX_PARTS + part) : 0);
        float U = INF, Bl = -INF;
        int nu = act ? 0 : -1, nl = nu;
        for (int t = 0; t < T32; ++t, ++g) {
            const int s = (int)(g % ST), b = (int)(g & 1);
            // the accumulator, then the tile's y values and chunk bounds written by the bulk copy
            if (!mbar_wait_bounded(&acc_full[b], (g / 2) & 1u, P.err) ||
                !mbar_wait_bounded(&b_full[s], (g / ST) & 1u, P.err)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const float* ys = reinterpret_cast<const float*>(sB + (size_t)s * STAGE_BYTES + tc_pieces(FMT) * B_PIECE +
                                                             TC_N * TC_NORM_ROW);
            const float2* cbs = reinterpret_cast<const float2*>(ys + TC_N);
            // two 32-column chunks per TMEM wait: both loads are in flight together
#pragma unroll 1
            for (int j = 0; j < TC_N / 32 / PARTS; j += 2) {
                const int col0 = part * (TC_N / PARTS) + j * 32;
                float sv[2][32];
                tmem_ld32x2(tb + ((uint32_t)(quarter * 32) << 16) + (uint32_t)b * TC_N + col0, sv);
                if (j + 2 >= TC_N / 32 / PARTS) {
                    // the warp's last columns of this accumulator are in registers: hand the
                    // buffer back to the MMA warp now, before any square-root work
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&acc_empty[b]);
                }
                // both chunks' smallest s~ and bounds tests first (independent chains), then
                // the square roots only where some query of the warp may find an extremum
                float csm[2];
                bool take[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float cs[4];
#pragma unroll
                    for (int a = 0; a < 4; ++a) cs[a] = INF;
#pragma unroll
                    for (int e = 0; e < 32; e += 4)
                        cs[(e / 4) % 4] = min3f(min3f(cs[(e / 4) % 4], sv[h][e], sv[h][e + 1]), sv[h][e + 2], sv[h][e + 3]);
                    csm[h] = min2f(min3f(cs[0], cs[1], cs[2]), cs[3]);
                    if (FMT == TC_FP16) csm[h] = fmaf(csm[h], usc, nq2);   // monotone: the min s~
                }
                // Every pair of the chunk has s >= S0 = max(min s~ - eps, 0), so its upper value
                // is >= y_min + sqrt(S0) and its lower value <= y_max - sqrt(S0).  The chunk
                // can hold an extremum (or a tie) only if sqrt(S0) <= G = max(U - y_min,
                // y_max - Bl), that is G >= 0 and S0 <= G^2.  In FP32: S0 is taken low by
                // (1 - 2^-23) (one rounding in the subtraction), G^2 high by (1 + 2^-21) (the
                // roundings of the two differences and of the two products), so no chunk that
                // passes the exact test is skipped.  A chunk without data has NaN bounds and
                // fails G >= 0.
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float2 cb = cbs[col0 / 32 + h];
                    const float s0 = fmaxf(csm[h] - eps, 0.f) * (1.f - 0x1p-23f);
                    const float G = fmaxf(U - cb.x, cb.y - Bl);
                    take[h] = __any_sync(0xffffffffu, act && G >= 0.f && s0 <= (G * G) * (1.f + 0x1p-21f));
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (!take[h]) continue;
                    const int col = col0 + h * 32;
                    const int chunk = (int)((rev ? T32 - 1 - t : t) * TC_CHUNKS + col / 32);
                    // four interleaved partial extrema per chunk keep the dependent chains short
                    float cu[4], cl[4];
#pragma unroll
                    for (int a = 0; a < 4; ++a) { cu[a] = INF; cl[a] = -INF; }
#pragma unroll
                    for (int e = 0; e < 32; e += 4) {
                        const int a = (e / 4) % 4;
                        const float4 y4 = *reinterpret_cast<const float4*>(ys + col + e);
                        float2 s0 = make_float2(sv[h][e], sv[h][e + 1]), s1 = make_float2(sv[h][e + 2], sv[h][e + 3]);
                        if (FMT == TC_FP16) {
                            // (scalar FMAs: this path is rare, and two more float2 constants
                            // would not fit the epilogue's registers)
                            s0 = make_float2(fmaf(s0.x, usc, nq2), fmaf(s0.y, usc, nq2));
                            s1 = make_float2(fmaf(s1.x, usc, nq2), fmaf(s1.y, usc, nq2));
                        }
                        const float2 r0 = make_float2(sqrt_approx(fabsf(s0.x)), sqrt_approx(fabsf(s0.y)));
                        const float2 r1 = make_float2(sqrt_approx(fabsf(s1.x)), sqrt_approx(fabsf(s1.y)));
                        const float2 y0 = make_float2(y4.x, y4.y), y1 = make_float2(y4.z, y4.w);
                        const float2 u0 = add2(y0, r0), u1 = add2(y1, r1), l0 = sub2(y0, r0), l1 = sub2(y1, r1);
                        cu[a] = min3f(min3f(cu[a], u0.x, u0.y), u1.x, u1.y);
                        cl[a] = max3f(max3f(cl[a], l0.x, l0.y), l1.x, l1.y);
                    }
                    const float cum = min2f(min3f(cu[0], cu[1], cu[2]), cu[3]);
                    const float clm = max2f(max3f(cl[0], cl[1], cl[2]), cl[3]);
                    if (act) {
                        const float dlt = 1.001f * eps * rsqrt_approx(fmaxf(csm[h], eps)) + epsv;
                        U = fminf(U, cum + dlt);
                        if (cum - dlt <= U) tc_append(Ru, nu, chunk, cum - dlt, U, true);
                        Bl = fmaxf(Bl, clm - dlt);
                        if (clm + dlt >= Bl) tc_append(Ru + TC_MAX_PARTS, nl, chunk, clm + dlt, Bl, false);
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&b_empty[s]);     // the stage's y values are no longer read
        }
        if (valid) {
            Ru->U = U;
            Ru->n = ok ? nu : -1;
            Ru[TC_MAX_PARTS].U = Bl;
            Ru[TC_MAX_PARTS].n = ok ? nl : -1;
        }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tb));
    }
}

// --------------------------------------------------------------- exact rescreen

struct TcRescreenParams {
    int parts;              // candidate lists per (query, bound) that the scan filled
    const float* Q;
    const int* qperm;       // [nq] query position -> query index
    const int* dperm;       // [N] data position -> data index
    const float* Xs;        // [N][d] data rows in position order
    const float* ys;        // [N]
    int64_t nq;
    int d;
    double M;
    double w[D_MAX];
    float sc[D_MAX];        // (float)(M w_j), rounded once on the host (the FP32 filter)
    bool unit_w;            // every w_j == 1: the FP64 distance skips the exact product by 1
    const float* X0;
    const float* y0;
    int64_t N;
    const TcRec* rec;
    float *g, *lo, *hi;
    int32_t *idx_up, *idx_lo;
    int* fb_count;          // queries sent to the fallback (device-side count)
    int* fb_list;
    unsigned* fb_ext;       // [nq][4] the fallback's accumulators, initialised when a query is listed
    unsigned long long* fb_best;    // [nq][2]
    int* fb_idx;            // [nq][2]
};

__device__ __forceinline__ double tc_dist64(const TcRescreenParams& P, const float* q, const float* x) {
    double acc = 0.0;
    if (P.unit_w) {
        for (int i = 0; i < P.d; ++i) {
            const double t = (double)q[i] - (double)x[i];
            acc += t * t;
        }
    } else {
        for (int i = 0; i < P.d; ++i) {
            const double t = ((double)q[i] - (double)x[i]) * P.w[i];
            acc += t * t;
        }
    }
    return sqrt(acc);
}

// (value, index) order of a bound: smaller value first for H_up (side 0), larger for
// H_lo (side 1), then the lower index.
__device__ __forceinline__ bool tc_better(int side, double v, int k, double bv, int bk) {
    if (k < 0) return false;
    if (bk < 0) return true;
    if (v != bv) return side == 0 ? v < bv : v > bv;
    return k < bk;
}

// One warp per query, eight queries per block.  For each bound, every surviving candidate
// chunk is evaluated by the 32 lanes (one point each, coalesced rows) in FP32.  FP32 error
// of y +- M |diag(w)(q - x)|_2 with correctly rounded sqrt: at most
// err = (d + 10) 2^-24 (r + |y|).  A point p can be the FP64 extremum (or tie with it) only
// if v32(p) is within err(p) + err(e) of v32(e) for the best point e seen so far, so the
// warp keeps the running FP32 extremum and the largest error seen, and lists for FP64 only
// the points within twice that error of it.  The lists of the block's eight queries (both
// bounds) are then evaluated in FP64 as one dense batch, one point per thread: the FP64
// pipe (narrow on this part) runs about one full warp per block instead of one per query.
constexpr int TC_RS_THREADS = 256;
constexpr int TC_RS_WARPS = TC_RS_THREADS / 32;
constexpr int TC_RS_CAND = 64;             // per-warp list of points for FP64 evaluation
__global__ void __launch_bounds__(TC_RS_THREADS) tc_rescreen_kernel(const TcRescreenParams P) {
    __shared__ int cbuf[TC_RS_WARPS][TC_RS_CAND];      // data position; ~position for H_lo
    __shared__ double cval[TC_RS_WARPS][TC_RS_CAND];   // their FP64 values
    __shared__ int ccount[TC_RS_WARPS], coff[TC_RS_WARPS + 1];
    __shared__ long long cq[TC_RS_WARPS];              // the warp's query index
    const int wq = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t pos = (int64_t)blockIdx.x * TC_RS_WARPS + wq;   // query position
    int* const mybuf = cbuf[wq];
    // every warp reaches the block barriers below, so no warp returns early
    bool active = pos < P.nq;
    int64_t qi = 0;
    bool finite = false;
    const TcRec* R = P.rec;
    if (active) {
        qi = P.qperm[pos];
        const float* q = P.Q + qi * P.d;
        finite = true;
        for (int i = 0; i < P.d; ++i) finite = finite && isfinite(q[i]);
        R = P.rec + pos * 2 * TC_MAX_PARTS;
        bool over = false;
        for (int b = 0; b < 2; ++b)
            for (int h = 0; h < P.parts; ++h) over = over || R[b * TC_MAX_PARTS + h].n < 0;
        if (finite && over) {
            if (lane == 0) {
                const int slot = atomicAdd(P.fb_count, 1);
                P.fb_list[slot] = (int)qi;
                P.fb_ext[4 * slot + 0] = P.fb_ext[4 * slot + 2] = 0xffffffffu;   // min keys: none yet
                P.fb_ext[4 * slot + 1] = P.fb_ext[4 * slot + 3] = 0u;            // max errors: 0
                P.fb_best[2 * slot] = P.fb_best[2 * slot + 1] = ~0ull;
                P.fb_idx[2 * slot] = P.fb_idx[2 * slot + 1] = 0x7fffffff;
            }
            active = false;
        }
    }
    const float* q = P.Q + qi * P.d;
    double bv[2] = {0.0, 0.0};
    int bk[2] = {-1, -1};
    int nc = 0;                                            // warp-uniform list length
    // a full list is evaluated by the warp itself, one point per lane (rare)
    auto flush = [&]() {
        __syncwarp();
        for (int c = lane; c < nc; c += 32) {
            const int e = mybuf[c];
            const int side = e < 0 ? 1 : 0;
            const int64_t k = e < 0 ? ~e : e;
            const double dist = P.M * tc_dist64(P, q, P.Xs + k * P.d);
            const double v = side == 0 ? (double)P.ys[k] + dist : (double)P.ys[k] - dist;
            const int ko = P.dperm[k];
            if (tc_better(side, v, ko, bv[side], bk[side])) { bv[side] = v; bk[side] = ko; }
        }
        __syncwarp();
        nc = 0;
    };
    if (active && finite) {
        float qs[D_MAX], sc[D_MAX];
#pragma unroll
        for (int i = 0; i < D_MAX; ++i) {
            qs[i] = i < P.d ? q[i] : 0.f;
            sc[i] = i < P.d ? P.sc[i] : 0.f;
        }
        const float erel = (float)(P.d + 10) * 5.9604645e-8f;   // (d + 10) 2^-24
        for (int b = 0; b < 2; ++b) {
            float bound = R[b * TC_MAX_PARTS].U;
            for (int h = 1; h < P.parts; ++h)
                bound = b == 0 ? fminf(bound, R[b * TC_MAX_PARTS + h].U) : fmaxf(bound, R[b * TC_MAX_PARTS + h].U);
            // running FP32 extremum of the bound and the largest error seen (warp-uniform)
            float ext = b == 0 ? __int_as_float(0x7f800000) : -__int_as_float(0x7f800000), emax = 0.f;
            for (int h = 0; h < P.parts; ++h) {
                const TcRec& r = R[b * TC_MAX_PARTS + h];
                for (int e = 0; e < r.n; ++e) {
                    if (b == 0 ? !(r.L[e] <= bound) : !(r.L[e] >= bound)) continue;   // warp-uniform
                    const int64_t k = (int64_t)r.id[e] * 32 + lane;      // data position
                    const bool in = k < P.N;
                    float v32 = b == 0 ? __int_as_float(0x7f800000) : -__int_as_float(0x7f800000), err = 0.f;
                    if (in) {
                        const float* x = P.Xs + k * P.d;
                        float acc = 0.f;
                        for (int i = 0; i < P.d; ++i) {
                            const float t = (qs[i] - x[i]) * sc[i];
                            acc = fmaf(t, t, acc);
                        }
                        const float rr = sqrtf(acc), yy = P.ys[k];
                        v32 = b == 0 ? yy + rr : yy - rr;
                        err = erel * (rr + fabsf(yy));
                    }
                    float cext = v32, cerr = err;
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) {
                        const float o = __shfl_xor_sync(0xffffffffu, cext, off);
                        cext = b == 0 ? fminf(cext, o) : fmaxf(cext, o);
                        cerr = fmaxf(cerr, __shfl_xor_sync(0xffffffffu, cerr, off));
                    }
                    ext = b == 0 ? fminf(ext, cext) : fmaxf(ext, cext);
                    emax = fmaxf(emax, cerr);
                    const bool cand = in && (b == 0 ? v32 <= ext + 2.f * emax : v32 >= ext - 2.f * emax);
                    const unsigned m = __ballot_sync(0xffffffffu, cand);
                    const int n = __popc(m);
                    if (nc + n > TC_RS_CAND) flush();
                    if (cand) mybuf[nc + __popc(m & ((1u << lane) - 1u))] = b == 0 ? (int)k : ~(int)k;
                    nc += n;
                }
            }
        }
    }
    if (lane == 0) {
        ccount[wq] = (active && finite) ? nc : 0;
        cq[wq] = (long long)qi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        coff[0] = 0;
        for (int w = 0; w < TC_RS_WARPS; ++w) coff[w + 1] = coff[w] + ccount[w];
    }
    __syncthreads();
    // the block's listed points, densely, one per thread
    for (int t = threadIdx.x; t < coff[TC_RS_WARPS]; t += TC_RS_THREADS) {
        int w = 0;
        while (coff[w + 1] <= t) ++w;
        const int c = t - coff[w];
        const int e = cbuf[w][c];
        const int64_t k = e < 0 ? ~e : e;
        const double dist = P.M * tc_dist64(P, P.Q + (int64_t)cq[w] * P.d, P.Xs + k * P.d);
        cval[w][c] = e < 0 ? (double)P.ys[k] - dist : (double)P.ys[k] + dist;
    }
    __syncthreads();
    if (!active) return;
    if (finite) {
        for (int c = lane; c < ccount[wq]; c += 32) {
            const int e = mybuf[c];
            const int side = e < 0 ? 1 : 0;
            const int ko = P.dperm[e < 0 ? ~e : e];
            if (tc_better(side, cval[wq][c], ko, bv[side], bk[side])) { bv[side] = cval[wq][c]; bk[side] = ko; }
        }
#pragma unroll
        for (int b = 0; b < 2; ++b) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, bv[b], off);
                const int ok = __shfl_xor_sync(0xffffffffu, bk[b], off);
                if (tc_better(b, ov, ok, bv[b], bk[b])) { bv[b] = ov; bk[b] = ok; }
            }
        }
    }
    if (lane != 0) return;
    double hi = bv[0], lo = bv[1];
    int iu = bk[0], il = bk[1];
    if (!finite || iu < 0 || il < 0) {
        hi = lo = __longlong_as_double(0x7ff8000000000000ll);
        iu = il = -1;
    }
    if (P.g) P.g[qi] = (float)(0.5 * (hi + lo));
    if (P.lo) P.lo[qi] = (float)lo;
    if (P.hi) P.hi[qi] = (float)hi;
    if (P.idx_up) P.idx_up[qi] = iu;
    if (P.idx_lo) P.idx_lo[qi] = il;
}

// --------------------------------------------------------------- device-side fallback
// Queries whose candidate lists overflowed (or, in the fp16 form, lie outside the fp16
// range) are listed by the rescreen in fb_list / fb_count and settled here without the
// host: the grid has a fixed shape and reads the count on the device, so lip_eval on a
// tensor-core handle never waits for the GPU and can be captured in a CUDA graph.  Three
// passes over all N points, each bound handled as a minimum (H_lo as the minimum of
// M |q - x| - y, which negates exactly):
//   pass 0: the FP32 minimum v32 of each bound and the largest FP32 error bound
//           err(p) = (d + 10) 2^-24 (r + |y|) (the rescreen's bound), by atomic min / max
//           of order-preserving keys, so the result does not depend on the order;
//   pass 1: every point with v32 <= min + 2 max err is evaluated in FP64 (the exact
//           minimiser p* and its ties pass: v32(p*) <= v64(p*) + err <= v64(e) + err <=
//           v32(e) + 2 err for the FP32 minimiser e); atomic min of the FP64 value's key;
//   pass 2: the lowest data index whose FP64 value equals that minimum.
// A work item is a group of TC_FB_QG listed queries and a chunk of TC_FB_CHUNK points, so
// a chunk is read once per group.  The results are the exact FP64 envelopes, rounded once,
// like the rescreen's.
constexpr int TC_FB_THREADS = 256, TC_FB_QG = 4, TC_FB_CHUNK = 2048;

struct TcFallbackParams {
    const float* Q;
    int d;
    const float* X0;        // [N][d] the data in index order
    const float* y0;
    int64_t N;
    double M;
    double w[D_MAX];
    float sc[D_MAX];        // (float)(M w_j), as in the rescreen
    bool unit_w;
    const int* fb_count;
    const int* fb_list;
    unsigned* ext;                  // [slot][4]: f2ord(min up), max err up, f2ord(min -lo), max err lo
    unsigned long long* best;       // [slot][2]: d2ord of the FP64 minima
    int* idx;                       // [slot][2]
    float *g, *lo, *hi;
    int32_t *idx_up, *idx_lo;
};

__device__ __forceinline__ unsigned long long d2ord(double v) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double ord2d(unsigned long long k) {
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}
__device__ __forceinline__ float ord2f(unsigned k) {
    return __uint_as_float((k >> 31) ? (k & 0x7fffffffu) : ~k);
}

template <int PASS>
__global__ void __launch_bounds__(TC_FB_THREADS) tc_fallback_kernel(const TcFallbackParams P) {
    __shared__ float qs[TC_FB_QG][D_MAX];
    __shared__ float scs[D_MAX];
    __shared__ double thr[TC_FB_QG][2];
    __shared__ unsigned long long bv[TC_FB_QG][2];
    const int cnt = *P.fb_count;
    const int d = P.d;
    const int64_t nchunks = (P.N + TC_FB_CHUNK - 1) / TC_FB_CHUNK, ngroups = (cnt + TC_FB_QG - 1) / TC_FB_QG;
    const float erel = (float)(d + 10) * 5.9604645e-8f;   // (d + 10) 2^-24
    const int lane = threadIdx.x % 32;
    if (threadIdx.x < D_MAX) scs[threadIdx.x] = P.sc[threadIdx.x];
    for (int64_t it = blockIdx.x; it < ngroups * nchunks; it += gridDim.x) {
        const int s0 = (int)(it / nchunks) * TC_FB_QG;          // first slot of the group
        const int64_t k0 = (it % nchunks) * TC_FB_CHUNK;
        const int ng = min(TC_FB_QG, cnt - s0);
        __syncthreads();                                        // the previous item is done with qs
        for (int t = threadIdx.x; t < TC_FB_QG * D_MAX; t += TC_FB_THREADS) {
            const int gq = t / D_MAX, i = t % D_MAX;
            qs[gq][i] = gq < ng && i < d ? P.Q[(int64_t)P.fb_list[s0 + gq] * d + i] : 0.f;
        }
        if (PASS > 0 && threadIdx.x < 2 * TC_FB_QG) {
            const int gq = threadIdx.x / 2, b = threadIdx.x % 2;
            if (gq < ng) {
                const unsigned* e = P.ext + 4 * (int64_t)(s0 + gq) + 2 * b;
                thr[gq][b] = (double)ord2f(e[0]) + 2.0 * (double)__uint_as_float(e[1]);
                if (PASS == 2) bv[gq][b] = P.best[2 * (int64_t)(s0 + gq) + b];
            }
        }
        __syncthreads();
        float mn[TC_FB_QG][2], em[TC_FB_QG][2];
#pragma unroll
        for (int gq = 0; gq < TC_FB_QG; ++gq)
            mn[gq][0] = mn[gq][1] = __int_as_float(0x7f800000), em[gq][0] = em[gq][1] = 0.f;
        for (int j = threadIdx.x; j < TC_FB_CHUNK; j += TC_FB_THREADS) {
            const int64_t k = k0 + j;
            if (k >= P.N) break;
            const float* x = P.X0 + k * d;
            const float yy = P.y0[k];
#pragma unroll
            for (int gq = 0; gq < TC_FB_QG; ++gq) {
                if (gq >= ng) break;
                float acc = 0.f;
                for (int i = 0; i < d; ++i) {
                    const float t = (qs[gq][i] - x[i]) * scs[i];
                    acc = fmaf(t, t, acc);
                }
                const float rr = sqrtf(acc);
                const float v[2] = {yy + rr, rr - yy};
                if (PASS == 0) {
                    const float err = erel * (rr + fabsf(yy));
                    mn[gq][0] = fminf(mn[gq][0], v[0]);
                    mn[gq][1] = fminf(mn[gq][1], v[1]);
                    em[gq][0] = em[gq][1] = fmaxf(em[gq][0], err);
                } else {
#pragma unroll
                    for (int b = 0; b < 2; ++b) {
                        if (!((double)v[b] <= thr[gq][b])) continue;
                        double acc64 = 0.0;
                        for (int i = 0; i < d; ++i) {
                            const double t = (double)qs[gq][i] - (double)x[i];
                            const double u = P.unit_w ? t : t * P.w[i];
                            acc64 += u * u;
                        }
                        const double dist = P.M * sqrt(acc64);
                        const double v64 = b == 0 ? (double)yy + dist : dist - (double)yy;
                        const int64_t slot = s0 + gq;
                        if (PASS == 1) atomicMin(P.best + 2 * slot + b, d2ord(v64));
                        else if (d2ord(v64) == bv[gq][b]) atomicMin(P.idx + 2 * slot + b, (int)k);
                    }
                }
            }
        }
        if (PASS == 0) {
#pragma unroll
            for (int gq = 0; gq < TC_FB_QG; ++gq) {
#pragma unroll
                for (int b = 0; b < 2; ++b) {
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) {
                        mn[gq][b] = fminf(mn[gq][b], __shfl_xor_sync(0xffffffffu, mn[gq][b], off));
                        em[gq][b] = fmaxf(em[gq][b], __shfl_xor_sync(0xffffffffu, em[gq][b], off));
                    }
                    if (lane == 0 && gq < ng) {
                        unsigned* e = P.ext + 4 * (int64_t)(s0 + gq) + 2 * b;
                        atomicMin(e, f2ord(mn[gq][b]));
                        atomicMax(e + 1, __float_as_uint(em[gq][b]));
                    }
                }
            }
        }
    }
}

__global__ void tc_fallback_finish_kernel(const TcFallbackParams P) {
    const int cnt = *P.fb_count;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < cnt; s += gridDim.x * blockDim.x) {
        const int64_t qi = P.fb_list[s];
        int iu = P.idx[2 * s], il = P.idx[2 * s + 1];
        double hi = ord2d(P.best[2 * s]), lo = -ord2d(P.best[2 * s + 1]);
        if (iu == 0x7fffffff || il == 0x7fffffff) {             // no data
            hi = lo = __longlong_as_double(0x7ff8000000000000ll);
            iu = il = -1;
        }
        if (P.g) P.g[qi] = (float)(0.5 * (hi + lo));
        if (P.lo) P.lo[qi] = (float)lo;
        if (P.hi) P.hi[qi] = (float)hi;
        if (P.idx_up) P.idx_up[qi] = iu;
        if (P.idx_lo) P.idx_lo[qi] = il;
    }
}

// --------------------------------------------------------------- launchers

size_t tc_tile_bytes_for(int d, int fmt) { return (size_t)tc_tile_bytes(tc_k_for_dim(d, fmt), fmt); }
size_t tc_a_bytes_for(int d, int fmt) { return (size_t)tc_a_bytes(tc_k_for_dim(d, fmt), fmt); }
size_t tc_rec_bytes() { return sizeof(TcRec) * 2 * TC_MAX_PARTS; }   // candidate lists per query


// The data's spatial order, then the tiles in that order, the position-ordered copies and
// the chunk bounds.
cudaError_t tc_prepare_data(const float* X0, const float* y0, int64_t N, int d, const double* scale,
                            unsigned* maxbits, char* tiles, int64_t ntiles, int fmt, const TcDataOrder& O,
                            cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(O.bounds, 0, D_MAX * sizeof(float2), st);   // an empty set centres at 0
    if (e == cudaSuccess) e = spatial_order(X0, N, d, O.dperm, O.bounds, O.scratch, st);
    if (e != cudaSuccess) return e;
    TcPrepParams P{};
    P.X0 = X0;
    P.y0 = y0;
    P.N = N;
    P.d = d;
    P.K = tc_k_for_dim(d, fmt);
    for (int j = 0; j < D_MAX; ++j) P.scale[j] = scale[j];
    P.bounds = O.bounds;
    P.maxbits = maxbits;
    P.tiles = tiles;
    P.ntiles = ntiles;
    P.perm = O.dperm;
    P.Xs = O.Xs;
    P.ys = O.ys;
    e = cudaMemsetAsync(maxbits, 0, 2 * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    const int64_t rows = ntiles * TC_N;
    if (rows > 0) {
        const unsigned blocks = (unsigned)((rows + 255) / 256);
        if (fmt == TC_BF16) tc_build_b_kernel<TC_BF16><<<blocks, 256, 0, st>>>(P);
        else if (fmt == TC_FP16) tc_build_b_kernel<TC_FP16><<<blocks, 256, 0, st>>>(P);
        else tc_build_b_kernel<TC_TF32><<<blocks, 256, 0, st>>>(P);
        const int64_t nchunks = ntiles * TC_CHUNKS;
        tc_chunk_bounds_kernel<<<(unsigned)((nchunks + 255) / 256), 256, 0, st>>>(O.ys, N, nchunks, tiles,
                                                                                 tc_tile_bytes(P.K, fmt));
    }
    return cudaGetLastError();
}

// SMs of the current device (148 if the query fails): the scan's persistent grid.
static int tc_sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        sms = 148;
    cudaGetLastError();
    return sms;
}

constexpr int TC_CTILES = 16;                          // data tiles per lockstep chunk
constexpr int64_t TC_WINDOW_DEFAULT = 32ll << 20;      // data bytes a round's sweeps may spread over

static int64_t tc_grid(int64_t nqt) {
    const int64_t sms = tc_sm_count();
    return nqt < sms ? nqt : sms;
}

size_t tc_arrive_bytes(int64_t nq, int64_t ntiles) {
    const int64_t nqt = (nq + TC_M - 1) / TC_M, grid = tc_grid(nqt);
    if (grid < 1) return 0;
    return (size_t)((nqt + grid - 1) / grid) * (size_t)((ntiles + TC_CTILES - 1) / TC_CTILES) * sizeof(int);
}

// One CTA per SM (all of TMEM each, one CTA fits), launched cooperatively so that the
// CTAs of a round are resident together while the soft lockstep waits for one another.
template <int K, int PARTS, int FMT>
static cudaError_t launch_tc_scan_k(const TcScanParams& P, int64_t nqt, bool persistent, cudaStream_t st) {
    const size_t smem = (size_t)tc_a_bytes(K, FMT) + (size_t)tc_stages(K, FMT) * tc_stage_bytes(K, FMT);
    static cudaError_t attr =
        cudaFuncSetAttribute(tc_scan_kernel<K, PARTS, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (attr != cudaSuccess) return attr;
    if (!persistent) {
        tc_scan_kernel<K, PARTS, FMT><<<(unsigned)nqt, tc_threads(PARTS), smem, st>>>(P);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)tc_grid(nqt));
    cfg.blockDim = dim3(tc_threads(PARTS));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, tc_scan_kernel<K, PARTS, FMT>, P);
}

template <int PARTS>
static cudaError_t launch_tc_scan_parts(int K, int fmt, const TcScanParams& P, int64_t nqt, bool pers,
                                         cudaStream_t st) {
    if (fmt == TC_BF16) return K <= 16 ? launch_tc_scan_k<16, PARTS, TC_BF16>(P, nqt, pers, st)
                                       : launch_tc_scan_k<32, PARTS, TC_BF16>(P, nqt, pers, st);
    if (fmt == TC_FP16) return K <= 16 ? launch_tc_scan_k<16, PARTS, TC_FP16>(P, nqt, pers, st)
                                       : launch_tc_scan_k<32, PARTS, TC_FP16>(P, nqt, pers, st);
    if (K == 8) return launch_tc_scan_k<8, PARTS, TC_TF32>(P, nqt, pers, st);
    if (K == 16) return launch_tc_scan_k<16, PARTS, TC_TF32>(P, nqt, pers, st);
    if (K == 24) return launch_tc_scan_k<24, PARTS, TC_TF32>(P, nqt, pers, st);
    return launch_tc_scan_k<32, PARTS, TC_TF32>(P, nqt, pers, st);
}

// Queries: build A, scan, rescreen.  Returns the fallback count through fb (device).
cudaError_t tc_eval_launch(const float* Q, int64_t nq, int d, const double* scale, int64_t N,
                           const unsigned* maxbits, const char* btiles, int64_t ntiles, char* atiles, float4* qc,
                           void* rec, const double* w, double M, const float* X0, const float* y0, float* g, float* lo,
                           float* hi, int32_t* iu, int32_t* il, int* fb_count, int* fb_list, void* fb_state,
                           int* arrive, int64_t window, unsigned* err, int variant, int fmt,
                           const TcDataOrder& O, const TcQueryOrder& QO, cudaEvent_t ev0, cudaEvent_t ev1,
                           cudaStream_t st) {
    const int K = tc_k_for_dim(d, fmt);
    // the queries' spatial order: a tile of 128 positions holds nearby queries
    cudaError_t e = spatial_order(Q, nq, d, QO.qperm, nullptr, QO.scratch, st);
    if (e != cudaSuccess) return e;
    const int parts = (variant & 1) ? 2 : 4;   // variant bit 0: 8 epilogue warps instead of 16
    const int64_t nqt = (nq + TC_M - 1) / TC_M;
    TcQueryParams A{};
    A.Q = Q;
    A.qperm = QO.qperm;
    A.nq = nq;
    A.d = d;
    A.K = K;
    for (int j = 0; j < D_MAX; ++j) A.scale[j] = scale[j];
    A.bounds = O.bounds;
    A.N = N;
    A.maxbits = maxbits;
    A.atiles = atiles;
    A.qc = qc;
    const unsigned ablocks = (unsigned)((nqt * TC_M + 255) / 256);
    if (fmt == TC_BF16) tc_build_a_kernel<TC_BF16><<<ablocks, 256, 0, st>>>(A);
    else if (fmt == TC_FP16) tc_build_a_kernel<TC_FP16><<<ablocks, 256, 0, st>>>(A);
    else tc_build_a_kernel<TC_TF32><<<ablocks, 256, 0, st>>>(A);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    TcScanParams S{};
    S.atiles = atiles;
    S.btiles = btiles;
    S.qc = qc;
    S.nq = nq;
    S.ntiles = ntiles;
    S.rec = static_cast<TcRec*>(rec);
    S.err = err;
    S.nqt = nqt;
    const int sms = tc_sm_count();
    S.wave = sms;
    // variant bit 2: one CTA per query tile instead of persistent CTAs (no lockstep then);
    // bit 1 turns the soft lockstep of the persistent CTAs' data sweep off
    const int64_t rounds = nqt > 0 ? (nqt + (nqt < sms ? nqt : sms) - 1) / (nqt < sms ? nqt : sms) : 0;
    const bool persistent = (variant & 4) == 0 && rounds * ntiles < ((int64_t)1 << 31);   // 32-bit ring counters
    if (persistent && (variant & 2) == 0 && nqt > 0) {
        S.arrive = arrive;
        S.ctiles = TC_CTILES;
        S.nch = (int)((ntiles + TC_CTILES - 1) / TC_CTILES);
        // a producer may run ahead of its round's slowest by about `window` bytes of tiles
        const int64_t win = window > 0 ? window : TC_WINDOW_DEFAULT;
        const int64_t lag = win / ((int64_t)tc_tile_bytes(K, fmt) * TC_CTILES);
        S.lag = (int)(lag < 1 ? 1 : (lag > S.nch ? S.nch : lag));
        if ((e = cudaMemsetAsync(arrive, 0, tc_arrive_bytes(nq, ntiles), st)) != cudaSuccess) return e;
    }
    if (ev0 && (e = cudaEventRecord(ev0, st)) != cudaSuccess) return e;     // the scan kernel alone
    e = parts == 2 ? launch_tc_scan_parts<2>(K, fmt, S, nqt, persistent, st)
                   : launch_tc_scan_parts<4>(K, fmt, S, nqt, persistent, st);
    if (e != cudaSuccess) return e;
    if (ev1 && (e = cudaEventRecord(ev1, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(fb_count, 0, sizeof(int), st)) != cudaSuccess) return e;
    TcRescreenParams R{};
    R.parts = parts;
    R.Q = Q;
    R.qperm = QO.qperm;
    R.dperm = O.dperm;
    R.Xs = O.Xs;
    R.ys = O.ys;
    R.nq = nq;
    R.d = d;
    R.M = M;
    R.unit_w = true;
    for (int j = 0; j < D_MAX; ++j) {
        R.w[j] = w[j];
        R.sc[j] = j < d ? (float)(M * w[j]) : 0.f;
        if (j < d && w[j] != 1.0) R.unit_w = false;
    }
    R.X0 = X0;
    R.y0 = y0;
    R.N = N;
    R.rec = static_cast<const TcRec*>(rec);
    R.g = g;
    R.lo = lo;
    R.hi = hi;
    R.idx_up = iu;
    R.idx_lo = il;
    R.fb_count = fb_count;
    R.fb_list = fb_list;
    unsigned* fb_ext = static_cast<unsigned*>(fb_state);
    unsigned long long* fb_best = reinterpret_cast<unsigned long long*>(fb_ext + 4 * nq);
    int* fb_idx = reinterpret_cast<int*>(fb_best + 2 * nq);
    R.fb_ext = fb_ext;
    R.fb_best = fb_best;
    R.fb_idx = fb_idx;
    tc_rescreen_kernel<<<(unsigned)((nq + TC_RS_WARPS - 1) / TC_RS_WARPS), TC_RS_THREADS, 0, st>>>(R);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the listed queries, without reading their count back
    TcFallbackParams F{};
    F.Q = Q;
    F.d = d;
    F.X0 = X0;
    F.y0 = y0;
    F.N = N;
    F.M = M;
    for (int j = 0; j < D_MAX; ++j) {
        F.w[j] = w[j];
        F.sc[j] = R.sc[j];
    }
    F.unit_w = R.unit_w;
    F.fb_count = fb_count;
    F.fb_list = fb_list;
    F.ext = fb_ext;
    F.best = fb_best;
    F.idx = fb_idx;
    F.g = g;
    F.lo = lo;
    F.hi = hi;
    F.idx_up = iu;
    F.idx_lo = il;
    const unsigned fgrid = (unsigned)sms * 4;
    tc_fallback_kernel<0><<<fgrid, TC_FB_THREADS, 0, st>>>(F);
    tc_fallback_kernel<1><<<fgrid, TC_FB_THREADS, 0, st>>>(F);
    tc_fallback_kernel<2><<<fgrid, TC_FB_THREADS, 0, st>>>(F);
    tc_fallback_finish_kernel<<<(unsigned)sms, 256, 0, st>>>(F);
    return cudaGetLastError();
}

size_t tc_fallback_state_bytes(int64_t nq) { return (size_t)nq * (4 * sizeof(unsigned) + 2 * 8 + 2 * sizeof(int)); }

}  // namespace lip
