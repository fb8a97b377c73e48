// Lipschitz constant of the data (Sec. 5): M_est = max_{i<j} |y^i - y^j| / dist(x^i, x^j)
// with the symmetric weighted norm, N^2/2 pair work and no pair matrix in memory.
//
// Layout: the same 4-point AoSoA groups as the envelope scan, without M, signs or the
// aux channel; power-of-two norm weights scale it exactly, other weights multiply the
// coordinate differences in the kernel (WT).  Pair (i, j) is compared through the squared ratio
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
#include "estimate.cuh"

namespace lip {

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

template <int NORM, int D, bool WT>
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
    float2 wt[D];
#pragma unroll
    for (int j = 0; j < D; ++j) wt[j] = WT ? make_float2(P.w[j], P.w[j]) : make_float2(1.f, 1.f);
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
                est_group<NORM, D, WT>(xi[r], yi[r], x, wt, q);
                best[r] = max3f(best[r], max3f(q[0], q[1], q[2]), q[3]);   // one link of the chain per group
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
            est_group<NORM, D, WT>(xi[r], yi[r], x, wt, q);
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
template <int NORM, bool WT>
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
                    const float t = WT ? __fmul_rn(__fsub_rn(xi[r][j], xe[e]), P.w[j]) : xi[r][j] - xe[e];
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

// The ratio of data points i and j in FP64, in the definition's order of operations with
// no contraction (the value of a plain IEEE double evaluation of Sec. 5's formula); -1 for
// a pair at distance 0 with equal values, which the definition leaves out.
template <typename T>
__device__ double est_ratio_fp64(const EstFinalParams& P, int64_t i, int64_t j) {
    const T* X = static_cast<const T*>(P.X0);
    const T* y = static_cast<const T*>(P.y0);
    double acc = 0.0;
    for (int c = 0; c < P.d; ++c) {
        const double v = __dmul_rn(fabs(__dsub_rn((double)X[i * P.d + c], (double)X[j * P.d + c])), P.w[c]);
        if (P.norm == LIP_L1) acc = __dadd_rn(acc, v);
        else if (P.norm == LIP_L2) acc = __dadd_rn(acc, __dmul_rn(v, v));
        else acc = v > acc ? v : acc;
    }
    const double dist = P.norm == LIP_L2 ? __dsqrt_rn(acc) : acc;
    const double dy = fabs(__dsub_rn((double)y[i], (double)y[j]));
    if (dist == 0.0) return dy == 0.0 ? -1.0 : (double)INFINITY;
    return __ddiv_rn(dy, dist);
}

// T = q* (1 - 2^-16), the exact selection's threshold (rounded down).
__device__ __forceinline__ float est_threshold(float qs) { return __fmul_rd(qs, 0.9999847412109375f); }

// q*: the largest FP32 squared ratio over the part's candidates; then the list of the
// part's tile pairs whose candidate reaches T, for the exact selection.
__global__ void estimate_final_kernel(const EstFinalParams P) {
    const int tid = threadIdx.x;
    float tb = -1.f;
    int ti = -1, tj = -1;
    const int64_t n = (int64_t)P.nb * P.nb;
    for (int64_t k = tid; k < n; k += blockDim.x) {
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
    __shared__ float s_q;
    __shared__ int s_count;
    if ((tid & 31) == 0) { sb[tid >> 5] = tb; si[tid >> 5] = ti; sj[tid >> 5] = tj; }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < (int)(blockDim.x / 32); ++w)
            if (est_better(sb[w], si[w], sj[w], tb, ti, tj)) { tb = sb[w]; ti = si[w]; tj = sj[w]; }
        s_q = ti >= 0 ? tb : -1.f;
        s_count = 0;
    }
    __syncthreads();
    const float qs = s_q;
    if (qs >= 0.f) {
        const float T = est_threshold(qs);
        for (int64_t k = tid; k < n; k += blockDim.x) {
            const int bi = (int)(k / P.nb), bj = (int)(k % P.nb);
            if (bj < bi || k % P.nparts != P.part) continue;
            const float4 c = P.cand[k];
            if (c.w != 0.f && c.x >= T) P.list[atomicAdd(&s_count, 1)] = ((unsigned)bi << 16) | (unsigned)bj;
        }
    }
    __syncthreads();
    if (tid == 0) {
        P.state->q = qs >= 0.f ? __float_as_int(qs) : -1;
        P.state->count = s_count;
        P.state->ratio = 0ull;
        P.state->key = ~0ull;
    }
}

// Exact selection (Sec. 5's maximum and the lowest (i, j) on ties, in FP64).  The screen's
// FP32 squared ratio q of a pair is within a relative (2d + 16) 2^-24 of the exact one for
// FP32 data (each weighted difference rounded at most three times, at most d + 2 roundings
// in the sums and squares, a reciprocal of at most 2 ulps and the product), so the pair
// with the largest FP64 ratio has q >= T = q* (1 - 2^-16) for every d <= 32, and its tile
// pair's screen maximum reaches T.  The listed tile pairs are cut into items of
// EXACT_ROWS row positions against the 512 column positions; a block stages an item's
// rows and columns from the layout in shared memory, forms each pair's q again with a
// scalar form of the same arithmetic (the same bound holds), and re-evaluates the pairs
// with q >= T in FP64 (est_ratio_fp64, on data indices through P.perm).  PASS 1 keeps the
// largest ratio R* (atomicMax of its bits: non-negative doubles order as integers), PASS
// 2 the smallest key among the pairs whose ratio is R*.  Data whose weighted coordinate
// differences fall into FP32's subnormal range, or whose ratios overflow FP32, are
// outside the bound.
constexpr int EXACT_ROWS = 16;      // 32 items a tile pair, so a few listed pairs spread over many blocks
constexpr int EXACT_THREADS = 256;

template <typename T, int PASS>
__global__ void __launch_bounds__(EXACT_THREADS) estimate_exact_kernel(const EstFinalParams P) {
    const int qb = *reinterpret_cast<const volatile int*>(&P.state->q);
    if (qb < 0) return;
    const int64_t items = (int64_t)*reinterpret_cast<const volatile int*>(&P.state->count) * (EST_TILE / EXACT_ROWS);
    const float Tq = est_threshold(__int_as_float(qb));
    const double Rs =
        PASS == 2 ? __longlong_as_double(*reinterpret_cast<const volatile long long*>(&P.state->ratio)) : 0.0;
    const int nch = P.d + 1;
    extern __shared__ __align__(16) float4 xs[];          // the item's rows, then the column tile
    float* fi = reinterpret_cast<float*>(xs);
    float* fj = reinterpret_cast<float*>(xs + (EXACT_ROWS / GROUP) * nch);
    double rbest = -1.0;
    unsigned long long kbest = ~0ull;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const unsigned tp = P.list[it / (EST_TILE / EXACT_ROWS)];
        const int bi = (int)(tp >> 16), bj = (int)(tp & 0xffffu);
        const int r0 = (int)(it % (EST_TILE / EXACT_ROWS)) * EXACT_ROWS;      // first row within tile bi
        __syncthreads();                                   // the previous item's reads are done
        const float4* rs = P.lay + ((size_t)bi * EST_TILE + r0) / GROUP * nch;
        for (int k = threadIdx.x; k < (EXACT_ROWS / GROUP) * nch; k += blockDim.x) xs[k] = rs[k];
        const float4* cs = P.lay + (size_t)bj * EST_TILE_GROUPS * nch;
        for (int k = threadIdx.x; k < EST_TILE_GROUPS * nch; k += blockDim.x)
            xs[(EXACT_ROWS / GROUP) * nch + k] = cs[k];
        __syncthreads();
        for (int p = threadIdx.x; p < EXACT_ROWS * EST_TILE; p += blockDim.x) {
            const int a = p / EST_TILE, b = p % EST_TILE;
            const int64_t pa = (int64_t)bi * EST_TILE + r0 + a, pb = (int64_t)bj * EST_TILE + b;
            if (pa >= pb || pb >= P.N) continue;           // each unordered pair once, no padding
            const float* xa = fi + (a / GROUP) * nch * GROUP + a % GROUP;
            const float* xb = fj + (b / GROUP) * nch * GROUP + b % GROUP;
            float acc = 0.f;
            for (int k = 0; k < P.d; ++k) {
                float t = __fsub_rn(xa[k * GROUP], xb[k * GROUP]);
                if (P.weighted) t = __fmul_rn(t, (float)P.w[k]);
                if (P.norm == LIP_L2) acc = __fmaf_rn(t, t, acc);
                else if (P.norm == LIP_L1) acc = __fadd_rn(acc, fabsf(t));
                else acc = fmaxf(acc, fabsf(t));
            }
            const float den = P.norm == LIP_L2 ? acc : __fmul_rn(acc, acc);
            const float dy = __fsub_rn(xa[P.d * GROUP], xb[P.d * GROUP]);
            const float q = __fmul_rn(__fmul_rn(dy, dy), rcp_approx(den));
            if (!(q >= Tq)) continue;
            const int64_t da = P.perm ? P.perm[pa] : pa, db = P.perm ? P.perm[pb] : pb;
            const int64_t i = da < db ? da : db, j = da < db ? db : da;
            const double r = est_ratio_fp64<T>(P, i, j);
            if (PASS == 1) {
                rbest = r > rbest ? r : rbest;
            } else if (r == Rs) {
                const unsigned long long key = ((unsigned long long)i << 32) | (unsigned long long)j;
                kbest = key < kbest ? key : kbest;
            }
        }
    }
    unsigned long long v = PASS == 1 ? (rbest >= 0.0 ? (unsigned long long)__double_as_longlong(rbest) : 0ull) : kbest;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
        v = PASS == 1 ? (u > v ? u : v) : (u < v ? u : v);
    }
    __shared__ unsigned long long red[EXACT_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < EXACT_THREADS / 32; ++w)
            v = PASS == 1 ? (red[w] > v ? red[w] : v) : (red[w] < v ? red[w] : v);
        if (PASS == 1 && v != 0ull) atomicMax(&P.state->ratio, v);
        if (PASS == 2 && v != ~0ull) atomicMin(&P.state->key, v);
    }
}

// {R*, i, j} (and R* again as the key that orders parts), or {0, -1, -1} without a pair.
__global__ void estimate_exact_finish_kernel(const EstFinalParams P) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const EstExactState S = *P.state;
    const bool ok = S.q >= 0 && S.key != ~0ull;
    const double M = ok ? __longlong_as_double((long long)S.ratio) : 0.0;
    P.out[0] = M;
    P.out[1] = ok ? (double)(S.key >> 32) : -1.0;
    P.out[2] = ok ? (double)(S.key & 0xffffffffull) : -1.0;
    if (P.write_key) P.out[3] = ok ? M : -1.0;
}

template <int NORM, int D>
static cudaError_t launch_est(const EstParams& P, cudaStream_t st) {
    if (P.weighted) estimate_kernel<NORM, D, true><<<dim3(P.nb, P.nb), EST_THREADS, 0, st>>>(P);
    else estimate_kernel<NORM, D, false><<<dim3(P.nb, P.nb), EST_THREADS, 0, st>>>(P);
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
    const int64_t src = P.gather ? (int64_t)P.gather[k] : k;     // position k holds point src
    const T* x = static_cast<const T*>(P.X0) + src * P.d;
    float* lay = static_cast<float*>(P.hot);
    const int64_t base = (k / GROUP) * (int64_t)P.nch * GROUP + (k % GROUP);
    for (int j = 0; j < P.d; ++j) lay[base + (int64_t)j * GROUP] = (float)(P.scale[j] * (double)x[j]);
    lay[base + (int64_t)P.d * GROUP] = (float)static_cast<const T*>(P.y0)[src];
}

cudaError_t launch_estimate_layout(int elem_bytes, const HotParams& P, cudaStream_t st) {
    const int64_t n = P.k1 - P.k0;
    if (n <= 0) return cudaSuccess;
    const unsigned g = (unsigned)((n + 255) / 256);
    if (elem_bytes == 8) est_layout_kernel<double><<<g, 256, 0, st>>>(P);
    else est_layout_kernel<float><<<g, 256, 0, st>>>(P);
    return cudaGetLastError();
}

template <int NORM, bool WT>
static cudaError_t launch_est_wide(int d, const EstParams& P, cudaStream_t st) {
    const int smem = EST_TILE_GROUPS * (D_MAX + 1) * (int)sizeof(float4);
    static cudaError_t attr = cudaFuncSetAttribute(estimate_wide_kernel<NORM, WT>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (attr != cudaSuccess) return attr;
    estimate_wide_kernel<NORM, WT><<<dim3(P.nb, P.nb), EST_THREADS, EST_TILE_GROUPS * (d + 1) * sizeof(float4), st>>>(P, d);
    return cudaGetLastError();
}

cudaError_t launch_estimate(int norm, int d, const EstParams& P, cudaStream_t st) {
    if (d > EST_NARROW_MAX) {
        switch (norm) {
            case LIP_L1: return P.weighted ? launch_est_wide<LIP_L1, true>(d, P, st) : launch_est_wide<LIP_L1, false>(d, P, st);
            case LIP_L2: return P.weighted ? launch_est_wide<LIP_L2, true>(d, P, st) : launch_est_wide<LIP_L2, false>(d, P, st);
            case LIP_LINF:
                return P.weighted ? launch_est_wide<LIP_LINF, true>(d, P, st) : launch_est_wide<LIP_LINF, false>(d, P, st);
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

// The exact passes run on a fixed grid of two blocks per SM (the listed items are few
// except for degenerate data such as constant y).
cudaError_t launch_estimate_exact(const EstFinalParams& P, cudaStream_t st) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int smem = (EXACT_ROWS / GROUP + EST_TILE_GROUPS) * (P.d + 1) * (int)sizeof(float4);
    if (smem > 48 * 1024) {          // per device, so set on every call that needs it
        cudaError_t e = P.elem_bytes == 8
            ? cudaFuncSetAttribute(estimate_exact_kernel<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)
            : cudaFuncSetAttribute(estimate_exact_kernel<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = P.elem_bytes == 8
                ? cudaFuncSetAttribute(estimate_exact_kernel<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)
                : cudaFuncSetAttribute(estimate_exact_kernel<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    const int grid = 2 * sms;
    if (P.elem_bytes == 8) {
        estimate_exact_kernel<double, 1><<<grid, EXACT_THREADS, smem, st>>>(P);
        estimate_exact_kernel<double, 2><<<grid, EXACT_THREADS, smem, st>>>(P);
    } else {
        estimate_exact_kernel<float, 1><<<grid, EXACT_THREADS, smem, st>>>(P);
        estimate_exact_kernel<float, 2><<<grid, EXACT_THREADS, smem, st>>>(P);
    }
    estimate_exact_finish_kernel<<<1, 32, 0, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_estimate_final(const EstFinalParams& P, cudaStream_t st) {
    estimate_final_kernel<<<1, 1024, 0, st>>>(P);
    return launch_estimate_exact(P, st);
}

}  // namespace lip
