// Lipschitz constant of the data (Sec. 5): M_est = max_{i<j} |y^i - y^j| / dist(x^i, x^j)
// with the symmetric weighted norm, N^2/2 pair work and no pair matrix in memory.
//
// Layout: the same 4-point AoSoA groups as the envelope scan, but unscaled (w * sign
// only) and without the aux channel.  Pair (i, j) is compared through the squared ratio
// (y_i - y_j)^2 * rcp(dist^2): one reciprocal per pair, no square root, no divide.
// dist = 0 gives rcp = +Inf, so equal y (0 * Inf = NaN) drops out of the NaN-ignoring
// max and different y gives +Inf, as the definition asks; padding points (y = NaN) and
// the i = j pairs of diagonal tiles drop out the same way.
//
// Grid: (I-tile, J-tile) pairs with J >= I (of one block-cyclic part of them when the
// pairs are shared out over GPUs); each CTA keeps EST_R I-points per thread in
// registers and streams the J-tile from shared memory.  The winning J-chunk of each
// thread row is rescanned to recover the exact j, CTAs write one candidate each, and a
// single-CTA pass picks the maximum (lowest (i, j) on ties) and recomputes it in FP64.
#include "launch.h"

namespace lip {

constexpr int EST_THREADS = 128;
constexpr int EST_R = 4;
constexpr int EST_TILE = EST_THREADS * EST_R;        // points per I-tile and per J-tile
constexpr int EST_TILE_GROUPS = EST_TILE / GROUP;
constexpr int EST_NARROW_MAX = 16;                   // d above this takes estimate_wide_kernel

template <int NORM, int D>
__device__ __forceinline__ void est_group(const float2 (&xi)[D], float2 yi, const float4 (&x)[D + 1], float (&r2)[4]) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float2 t[D];
#pragma unroll
        for (int j = 0; j < D; ++j) t[j] = sub2(xi[j], half_of(x[j], h));
        float2 den;
        if constexpr (NORM == LIP_L2) {
            den = mul2(t[0], t[0]);
#pragma unroll
            for (int j = 1; j < D; ++j) den = fma2(t[j], t[j], den);
        } else if constexpr (NORM == LIP_L1) {
            float2 acc = make_float2(fabsf(t[0].x), fabsf(t[0].y));
#pragma unroll
            for (int j = 1; j < D; ++j) acc = make_float2(acc.x + fabsf(t[j].x), acc.y + fabsf(t[j].y));
            den = mul2(acc, acc);
        } else {
            float a[D], b[D];
#pragma unroll
            for (int j = 0; j < D; ++j) { a[j] = fabsf(t[j].x); b[j] = fabsf(t[j].y); }
            const float2 acc = make_float2(max_reduce<D>(a), max_reduce<D>(b));
            den = mul2(acc, acc);
        }
        const float2 dy = sub2(yi, half_of(x[D], h));
        const float2 num = mul2(dy, dy);
        const float2 q = mul2(num, make_float2(rcp_approx(den.x), rcp_approx(den.y)));
        r2[2 * h] = q.x;
        r2[2 * h + 1] = q.y;
    }
}

// (ratio, i, j) ordering: larger ratio first, then lower i, then lower j.
__device__ __forceinline__ bool est_better(float r, int i, int j, float rb, int ib, int jb) {
    if (ib < 0) return i >= 0;
    if (i < 0) return false;
    if (r != rb) return r > rb;
    if (i != ib) return i < ib;
    return j < jb;
}

// Block reduction of the threads' best pairs (fixed shape, so the result does not depend
// on timing) and the block's candidate record.
__device__ __forceinline__ void est_block_write(const EstParams& P, int bi, int bj, float tb, int ti, int tj) {
    const int tid = threadIdx.x;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, tb, off);
        const int oi = __shfl_xor_sync(0xffffffffu, ti, off);
        const int oj = __shfl_xor_sync(0xffffffffu, tj, off);
        if (est_better(ob, oi, oj, tb, ti, tj)) { tb = ob; ti = oi; tj = oj; }
    }
    __shared__ float sb[EST_THREADS / 32];
    __shared__ int si[EST_THREADS / 32], sj[EST_THREADS / 32];
    if ((tid & 31) == 0) { sb[tid >> 5] = tb; si[tid >> 5] = ti; sj[tid >> 5] = tj; }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < EST_THREADS / 32; ++w)
            if (est_better(sb[w], si[w], sj[w], tb, ti, tj)) { tb = sb[w]; ti = si[w]; tj = sj[w]; }
        P.cand[(size_t)bi * P.nb + bj] = make_float4(tb, __int_as_float(ti), __int_as_float(tj), ti >= 0 ? 1.f : 0.f);
    }
}

template <int NORM, int D>
__global__ void __launch_bounds__(EST_THREADS)
estimate_kernel(const EstParams P) {
    constexpr int NCH = D + 1;
    const int bi = blockIdx.x, bj = blockIdx.y;
    if (bj < bi) return;
    if (((int64_t)bi * P.nb + bj) % P.nparts != P.part) return;
    __shared__ __align__(16) float4 tile[EST_TILE_GROUPS * NCH];
    const int tid = threadIdx.x;

    // J-tile to shared memory (contiguous groups of the layout).
    const float4* src = P.lay + (size_t)bj * EST_TILE_GROUPS * NCH;
    for (int k = tid; k < EST_TILE_GROUPS * NCH; k += EST_THREADS) tile[k] = __ldg(src + k);

    // I-points to registers (duplicated for the packed pair arithmetic).
    float2 xi[EST_R][D];
    float2 yi[EST_R];
    int ii[EST_R];
#pragma unroll
    for (int r = 0; r < EST_R; ++r) {
        const int64_t i = (int64_t)bi * EST_TILE + r * EST_THREADS + tid;
        ii[r] = (int)i;
        const float* g = reinterpret_cast<const float*>(P.lay + (size_t)(i / GROUP) * NCH);
        const int lane = (int)(i % GROUP);
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const float v = __ldg(g + j * GROUP + lane);
            xi[r][j] = make_float2(v, v);
        }
        const float v = __ldg(g + D * GROUP + lane);
        yi[r] = make_float2(v, v);
    }
    __syncthreads();

    float best[EST_R], prev[EST_R];
    int bc[EST_R];
#pragma unroll
    for (int r = 0; r < EST_R; ++r) { best[r] = -1.f; prev[r] = -1.f; bc[r] = -1; }

    for (int c = 0; c < EST_TILE_GROUPS; c += CHUNK_GROUPS) {
#pragma unroll 2
        for (int gi = 0; gi < CHUNK_GROUPS; ++gi) {
            float4 x[NCH];
#pragma unroll
            for (int ch = 0; ch < NCH; ++ch) x[ch] = tile[(c + gi) * NCH + ch];
#pragma unroll
            for (int r = 0; r < EST_R; ++r) {
                float q[4];
                est_group<NORM, D>(xi[r], yi[r], x, q);
                best[r] = max3f(max3f(best[r], q[0], q[1]), q[2], q[3]);
            }
        }
#pragma unroll
        for (int r = 0; r < EST_R; ++r) {
            bc[r] = best[r] > prev[r] ? c / CHUNK_GROUPS : bc[r];
            prev[r] = best[r];
        }
    }

    // Exact j of each row's maximum (lowest j on ties), then the thread's best row.
    float tb = -1.f;
    int ti = -1, tj = -1;
#pragma unroll
    for (int r = 0; r < EST_R; ++r) {
        if (bc[r] < 0) continue;
        int jbest = -1;
#pragma unroll 1
        for (int gi = 0; gi < CHUNK_GROUPS; ++gi) {
            const int g = bc[r] * CHUNK_GROUPS + gi;
            float4 x[NCH];
#pragma unroll
            for (int ch = 0; ch < NCH; ++ch) x[ch] = tile[g * NCH + ch];
            float q[4];
            est_group<NORM, D>(xi[r], yi[r], x, q);
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (jbest < 0 && q[e] == best[r]) jbest = bj * EST_TILE + g * GROUP + e;
        }
        if (jbest < 0) continue;
        const int a = min(ii[r], jbest), b = max(ii[r], jbest);
        if (est_better(best[r], a, b, tb, ti, tj)) { tb = best[r]; ti = a; tj = b; }
    }

    est_block_write(P, bi, bj, tb, ti, tj);
}

// d > 16: the same tiles, grid and candidate records.  Each thread keeps its EST_R
// I-points as plain floats and reads a J-group's coordinates from shared memory one
// channel at a time (the packed form's duplicated registers do not fit at these widths);
// the squared ratio is formed in the same order of operations as est_group, and the row
// maximum is tracked per pair (strict >, so the lowest j on ties; NaN never wins).
template <int NORM>
__global__ void __launch_bounds__(EST_THREADS)
estimate_wide_kernel(const EstParams P, int d) {
    const int nch = d + 1;
    const int bi = blockIdx.x, bj = blockIdx.y;
    if (bj < bi) return;
    if (((int64_t)bi * P.nb + bj) % P.nparts != P.part) return;
    extern __shared__ __align__(16) float4 wtile[];     // EST_TILE_GROUPS * nch
    const int tid = threadIdx.x;
    const float4* src = P.lay + (size_t)bj * EST_TILE_GROUPS * nch;
    for (int k = tid; k < EST_TILE_GROUPS * nch; k += EST_THREADS) wtile[k] = __ldg(src + k);
    float xi[EST_R][D_MAX];
    float yi[EST_R];
    int ii[EST_R];
#pragma unroll
    for (int r = 0; r < EST_R; ++r) {
        const int64_t i = (int64_t)bi * EST_TILE + r * EST_THREADS + tid;
        ii[r] = (int)i;
        const float* g = reinterpret_cast<const float*>(P.lay + (size_t)(i / GROUP) * nch);
        const int lane = (int)(i % GROUP);
#pragma unroll
        for (int j = 0; j < D_MAX; ++j) xi[r][j] = j < d ? __ldg(g + j * GROUP + lane) : 0.f;
        yi[r] = __ldg(g + d * GROUP + lane);
    }
    __syncthreads();
    float best[EST_R];
    int bjr[EST_R];
#pragma unroll
    for (int r = 0; r < EST_R; ++r) { best[r] = -1.f; bjr[r] = -1; }
    for (int gi = 0; gi < EST_TILE_GROUPS; ++gi) {
        const float4* grp = wtile + gi * nch;
        float acc[EST_R][4];
#pragma unroll
        for (int j = 0; j < D_MAX; ++j) {
            if (j >= d) break;
            const float4 xv = grp[j];
            const float xe[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
            for (int r = 0; r < EST_R; ++r)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float t = xi[r][j] - xe[e];
                    if (NORM == LIP_L2) acc[r][e] = j == 0 ? t * t : fmaf(t, t, acc[r][e]);
                    else if (NORM == LIP_L1) acc[r][e] = j == 0 ? fabsf(t) : acc[r][e] + fabsf(t);
                    else acc[r][e] = j == 0 ? fabsf(t) : fmaxf(acc[r][e], fabsf(t));
                }
        }
        const float4 yv = grp[d];
        const float ye[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
        for (int r = 0; r < EST_R; ++r)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float den = NORM == LIP_L2 ? acc[r][e] : acc[r][e] * acc[r][e];
                const float dy = yi[r] - ye[e];
                const float q = (dy * dy) * rcp_approx(den);
                if (q > best[r]) { best[r] = q; bjr[r] = bj * EST_TILE + gi * GROUP + e; }
            }
    }
    float tb = -1.f;
    int ti = -1, tj = -1;
#pragma unroll
    for (int r = 0; r < EST_R; ++r) {
        if (bjr[r] < 0) continue;
        const int a = min(ii[r], bjr[r]), b = max(ii[r], bjr[r]);
        if (est_better(best[r], a, b, tb, ti, tj)) { tb = best[r]; ti = a; tj = b; }
    }
    est_block_write(P, bi, bj, tb, ti, tj);
}

template <typename T>
__device__ double est_ratio_fp64(const EstFinalParams& P, int i, int j) {
    const T* X = static_cast<const T*>(P.X0);
    const T* y = static_cast<const T*>(P.y0);
    double acc = 0.0;
    for (int c = 0; c < P.d; ++c) {
        const double v = fabs((double)X[(int64_t)i * P.d + c] - (double)X[(int64_t)j * P.d + c]) * P.w[c];
        if (P.norm == LIP_L1) acc += v;
        else if (P.norm == LIP_L2) acc += v * v;
        else acc = v > acc ? v : acc;
    }
    const double dist = P.norm == LIP_L2 ? sqrt(acc) : acc;
    const double dy = fabs((double)y[i] - (double)y[j]);
    if (dist == 0.0) return dy == 0.0 ? 0.0 : (double)INFINITY;
    return dy / dist;
}

__global__ void estimate_final_kernel(const EstFinalParams P) {
    const int tid = threadIdx.x;
    float tb = -1.f;
    int ti = -1, tj = -1;
    for (int64_t k = tid; k < (int64_t)P.nb * P.nb; k += blockDim.x) {
        const int bi = (int)(k / P.nb), bj = (int)(k % P.nb);
        if (bj < bi || k % P.nparts != P.part) continue;
        const float4 c = P.cand[k];
        if (c.w == 0.f) continue;
        const int i = __float_as_int(c.y), j = __float_as_int(c.z);
        if (est_better(c.x, i, j, tb, ti, tj)) { tb = c.x; ti = i; tj = j; }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, tb, off);
        const int oi = __shfl_xor_sync(0xffffffffu, ti, off);
        const int oj = __shfl_xor_sync(0xffffffffu, tj, off);
        if (est_better(ob, oi, oj, tb, ti, tj)) { tb = ob; ti = oi; tj = oj; }
    }
    __shared__ float sb[32];
    __shared__ int si[32], sj[32];
    if ((tid & 31) == 0) { sb[tid >> 5] = tb; si[tid >> 5] = ti; sj[tid >> 5] = tj; }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < (int)(blockDim.x / 32); ++w)
            if (est_better(sb[w], si[w], sj[w], tb, ti, tj)) { tb = sb[w]; ti = si[w]; tj = sj[w]; }
        double M = 0.0;
        if (ti >= 0) M = P.elem_bytes == 8 ? est_ratio_fp64<double>(P, ti, tj) : est_ratio_fp64<float>(P, ti, tj);
        P.out[0] = M;
        P.out[1] = (double)ti;
        P.out[2] = (double)tj;
        if (P.write_key) P.out[3] = ti >= 0 ? (double)tb : -1.0;
    }
}

template <int NORM, int D>
static cudaError_t launch_est(const EstParams& P, cudaStream_t st) {
    estimate_kernel<NORM, D><<<dim3(P.nb, P.nb), EST_THREADS, 0, st>>>(P);
    return cudaGetLastError();
}

template <int NORM, int... Ds>
static cudaError_t est_dispatch_d(int d, const EstParams& P, cudaStream_t st, std::integer_sequence<int, Ds...>) {
    cudaError_t e = cudaErrorInvalidValue;
    ((d == Ds + 1 ? (e = launch_est<NORM, Ds + 1>(P, st), 0) : 0), ...);
    return e;
}

int estimate_tile_points() { return EST_TILE; }

// FP32 layout for the estimate: coordinate j scaled by P.scale[j] (the norm weight), y.
template <typename T>
__global__ void est_layout_kernel(const HotParams P) {
    const int64_t k = P.k0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P.k1) return;
    const T* x = static_cast<const T*>(P.X0) + k * P.d;
    float* lay = static_cast<float*>(P.hot);
    const int64_t base = (k / GROUP) * (int64_t)P.nch * GROUP + (k % GROUP);
    for (int j = 0; j < P.d; ++j) lay[base + (int64_t)j * GROUP] = (float)(P.scale[j] * (double)x[j]);
    lay[base + (int64_t)P.d * GROUP] = (float)static_cast<const T*>(P.y0)[k];
}

cudaError_t launch_estimate_layout(int elem_bytes, const HotParams& P, cudaStream_t st) {
    const int64_t n = P.k1 - P.k0;
    if (n <= 0) return cudaSuccess;
    const unsigned g = (unsigned)((n + 255) / 256);
    if (elem_bytes == 8) est_layout_kernel<double><<<g, 256, 0, st>>>(P);
    else est_layout_kernel<float><<<g, 256, 0, st>>>(P);
    return cudaGetLastError();
}

template <int NORM>
static cudaError_t launch_est_wide(int d, const EstParams& P, cudaStream_t st) {
    const int smem = EST_TILE_GROUPS * (D_MAX + 1) * (int)sizeof(float4);
    static cudaError_t attr = cudaFuncSetAttribute(estimate_wide_kernel<NORM>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (attr != cudaSuccess) return attr;
    estimate_wide_kernel<NORM><<<dim3(P.nb, P.nb), EST_THREADS, EST_TILE_GROUPS * (d + 1) * sizeof(float4), st>>>(P, d);
    return cudaGetLastError();
}

cudaError_t launch_estimate(int norm, int d, const EstParams& P, cudaStream_t st) {
    if (d > EST_NARROW_MAX) {
        switch (norm) {
            case LIP_L1: return launch_est_wide<LIP_L1>(d, P, st);
            case LIP_L2: return launch_est_wide<LIP_L2>(d, P, st);
            case LIP_LINF: return launch_est_wide<LIP_LINF>(d, P, st);
            default: return cudaErrorInvalidValue;
        }
    }
    auto seq = std::make_integer_sequence<int, EST_NARROW_MAX>{};
    switch (norm) {
        case LIP_L1: return est_dispatch_d<LIP_L1>(d, P, st, seq);
        case LIP_L2: return est_dispatch_d<LIP_L2>(d, P, st, seq);
        case LIP_LINF: return est_dispatch_d<LIP_LINF>(d, P, st, seq);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_estimate_final(const EstFinalParams& P, cudaStream_t st) {
    estimate_final_kernel<<<1, 1024, 0, st>>>(P);
    return cudaGetLastError();
}

}  // namespace lip
