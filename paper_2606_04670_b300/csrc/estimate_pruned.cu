// Pruned Lipschitz-constant estimate (Sec. 5: M_est = max_{i<j} |y^i - y^j| / dist): the
// FP32 screen of the full estimate with most of the N^2/2 pairs ruled out by bounds,
// followed by the same exact FP64 selection (estimate.cu), so the result is the FP64
// definition's exactly (the value, then the lowest i, then the lowest j).
//
// The estimate layout is built in the spatial order of the points, with a record (box of
// the points in layout coordinates, smallest and largest y) per 16-point chunk and per
// 512-point tile.  For two records A and B, every pair (i in A, j in B) has
//   |y_i - y_j| <= max(yhi_A - ylo_B, yhi_B - ylo_A)           (IEEE rounding is monotone)
//   FP32 dist^2 >= the same FP32 operations on the gaps between the boxes
//                  (max(lo_B - hi_A, lo_A - hi_B, 0) per coordinate),
// so its FP32 squared ratio q = (y_i - y_j)^2 rcp(dist^2) is at most
//   UB = num_ub rcp(den_lb) (1 + 2^-18)
// (rcp.approx's relative error and the final product's rounding are far below the
// margin).  The screen runs the tile pairs diagonal band first (neighbouring tiles in the
// spatial order hold the close pairs, whose ratios are the large ones) and keeps the
// largest q found so far in one device word (atomicMax of its bits): a block skips a tile
// pair whose UB is below (1 - 2^-16) times it, and a warp skips a chunk for each of its
// four rows of 32 points whose UB against the chunk is below (1 - 2^-16) times that word
// (all (row, chunk) pairs of the tile pair tested at once, one chunk per lane).
// Every pair with q >= q* (1 - 2^-16) -- the exact selection's threshold -- is therefore
// evaluated, and each tile pair's largest evaluated q is recorded; the select kernel lists
// the tile pairs whose record reaches the threshold.
#include "estimate.cuh"

namespace lip {

namespace {

constexpr int EP_CG = 4;                                   // groups per chunk: 16-point chunks
constexpr int EP_CHUNKS = EST_TILE_GROUPS / EP_CG;         // 32 chunks per tile

// Record layout: lo[D], hi[D], ylo, yhi (the same as the pruned scan's, aux-free).  With
// WT the gaps are multiplied by the weights as the pair arithmetic multiplies the
// differences (rounding of a product by w >= 0 is monotone too).
template <int NORM, int D, bool WT>
__device__ __forceinline__ float pair_ub(const float* A, const float* B, const float (&w)[D]) {
    float g[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        g[j] = fmaxf(fmaxf(__fsub_rn(B[j], A[D + j]), __fsub_rn(A[j], B[D + j])), 0.f);
        if constexpr (WT) g[j] = __fmul_rn(g[j], w[j]);
    }
    float den;
    if constexpr (NORM == LIP_L2) {
        den = __fmul_rn(g[0], g[0]);
#pragma unroll
        for (int j = 1; j < D; ++j) den = __fmaf_rn(g[j], g[j], den);
    } else if constexpr (NORM == LIP_L1) {
        float acc = g[0];
#pragma unroll
        for (int j = 1; j < D; ++j) acc = __fadd_rn(acc, g[j]);
        den = __fmul_rn(acc, acc);
    } else {
        float acc = g[0];
#pragma unroll
        for (int j = 1; j < D; ++j) acc = fmaxf(acc, g[j]);
        den = __fmul_rn(acc, acc);
    }
    const float nub = fmaxf(__fsub_rn(A[2 * D + 1], B[2 * D]), __fsub_rn(B[2 * D + 1], A[2 * D]));
    const float num = __fmul_rn(nub, nub);
    return __fmul_rn(__fmul_rn(num, rcp_approx(den)), 1.000003814697265625f);   // 1 + 2^-18
}

template <int D>
__device__ __forceinline__ void load_record(const float4* rec, float (&b)[pruned_box_f4(D) * 4]) {
#pragma unroll
    for (int k = 0; k < pruned_box_f4(D); ++k) {
        const float4 v = rec[k];
        b[4 * k] = v.x;
        b[4 * k + 1] = v.y;
        b[4 * k + 2] = v.z;
        b[4 * k + 3] = v.w;
    }
}

// Block k -> tile pair (I, J >= I), diagonal band b = J - I first: band b starts at
// b nb - b (b - 1) / 2.
__device__ __forceinline__ void band_pair(int64_t k, int nb, int& I, int& J) {
    double disc = (2.0 * nb + 1.0) * (2.0 * nb + 1.0) - 8.0 * (double)k;
    int b = (int)(((2.0 * nb + 1.0) - sqrt(disc > 0.0 ? disc : 0.0)) * 0.5);
    if (b < 0) b = 0;
    auto start = [&](int64_t bb) { return bb * nb - bb * (bb - 1) / 2; };
    while (b > 0 && start(b) > k) --b;
    while (b + 1 < nb && start(b + 1) <= k) ++b;
    I = (int)(k - start(b));
    J = I + b;
}

// (1 - 2^-16) x, rounded down: what a bound must reach for its pairs to stay candidates.
__device__ __forceinline__ float ep_margin(float x) { return __fmul_rd(x, 0.9999847412109375f); }

template <int NORM, int D, bool WT>
__global__ void __launch_bounds__(EST_THREADS) estimate_pruned_kernel(const EstPrunedParams P) {
    constexpr int NCH = D + 1;
    constexpr int NB4 = pruned_box_f4(D);
    __shared__ __align__(16) float4 tile[EST_TILE_GROUPS * NCH];
    __shared__ __align__(16) float4 crec[EP_CHUNKS * NB4];
    __shared__ float red[EST_THREADS / 32];
    __shared__ int wcnt[EST_THREADS / 32];
    int I, J;
    band_pair(blockIdx.x, P.nb, I, J);
    const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
    const int gb = *reinterpret_cast<const volatile int*>(P.gbest);
    // the largest squared ratio found so far
    const float L = gb >= 0 ? __int_as_float(gb) : -1.f;
    float w1[D];
    float2 wt[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        w1[j] = WT ? P.w[j] : 1.f;
        wt[j] = make_float2(w1[j], w1[j]);
    }
    {
        float A[NB4 * 4], B[NB4 * 4];
        load_record<D>(P.tbox + (int64_t)I * NB4, A);
        load_record<D>(P.tbox + (int64_t)J * NB4, B);
        // a tile without data has NaN bounds; a tile pair below the margin of L holds no candidate
        if (!(A[2 * D] == A[2 * D]) || !(B[2 * D] == B[2 * D]) || pair_ub<NORM, D, WT>(A, B, w1) < ep_margin(L)) {
            if (tid == 0) P.bq[blockIdx.x] = -1.f;
            return;
        }
    }
    const float4* src = P.lay + (size_t)J * EST_TILE_GROUPS * NCH;
    for (int k = tid; k < EST_TILE_GROUPS * NCH; k += EST_THREADS) tile[k] = __ldg(src + k);
    for (int k = tid; k < EP_CHUNKS * NB4; k += EST_THREADS) crec[k] = __ldg(P.cbox + (int64_t)J * EP_CHUNKS * NB4 + k);
    // row points: row r of the warp is the 32 consecutive positions warp * 128 + 32 r + lane
    // of tile I (one per lane), so that a row's points are neighbours in space
    float2 xi[EST_R][D];
    float2 yi[EST_R];
    {
        const float* layf = reinterpret_cast<const float*>(P.lay);
#pragma unroll
        for (int r = 0; r < EST_R; ++r) {
            const int64_t p = (int64_t)I * EST_TILE + warp * 128 + 32 * r + lane;
            const float* gp = layf + (p / GROUP) * NCH * GROUP + p % GROUP;
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const float v = __ldg(gp + j * GROUP);
                xi[r][j] = make_float2(v, v);
            }
            const float v = __ldg(gp + D * GROUP);
            yi[r] = make_float2(v, v);
        }
    }
    // each row's record (padding, y = NaN, drops out), in shared memory for the tests
    __shared__ __align__(16) float rrec[EST_THREADS / 32][EST_R][NB4 * 4];
    unsigned rlive = 0u;                  // rows holding data
#pragma unroll
    for (int r = 0; r < EST_R; ++r) {
        const bool live = yi[r].x == yi[r].x;
        if (__any_sync(0xffffffffu, live)) rlive |= 1u << r;
#pragma unroll
        for (int j = 0; j <= D; ++j) {
            const float v = j < D ? xi[r][j].x : yi[r].x;
            float lo = live ? v : __int_as_float(0x7f800000), hi = live ? v : -__int_as_float(0x7f800000);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
                hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
            }
            if (lane == 0) {
                rrec[warp][r][j < D ? j : 2 * D] = lo;
                rrec[warp][r][j < D ? D + j : 2 * D + 1] = hi;
            }
        }
        if (lane == 0)
            for (int k = 2 * D + 2; k < NB4 * 4; ++k) rrec[warp][r][k] = 0.f;
    }
    if (P.work && tid == 0) atomicAdd(P.work, 1ull);     // tile pairs entered
    __syncthreads();

    float best = -1.f;                    // this thread's largest squared ratio
    int nev = 0;                          // (row, chunk) pairs this warp evaluated
    // Every (row, chunk) pair of the tile pair is tested at once, against the margin of the
    // latest global maximum: lane c takes chunk c, one round per row (bit c of cm[r]).
    static_assert(EP_CHUNKS == 32, "one chunk per lane");
    unsigned cm[EST_R];
    {
        const int gn = *reinterpret_cast<const volatile int*>(P.gbest);
        const float lim = ep_margin(fmaxf(L, gn >= 0 ? __int_as_float(gn) : -1.f));
        float B[NB4 * 4];
        load_record<D>(crec + lane * NB4, B);
        const bool cvalid = B[2 * D] == B[2 * D];
#pragma unroll
        for (int r = 0; r < EST_R; ++r) {
            bool need = false;
            if (cvalid && ((rlive >> r) & 1u)) {
                float A[NB4 * 4];
#pragma unroll
                for (int k = 0; k < NB4 * 4; ++k) A[k] = rrec[warp][r][k];
                need = !(pair_ub<NORM, D, WT>(A, B, w1) < lim);
            }
            cm[r] = __ballot_sync(0xffffffffu, need);
        }
    }
    unsigned any = 0u;
#pragma unroll
    for (int r = 0; r < EST_R; ++r) any |= cm[r];
    for (unsigned left = any; left; left &= left - 1) {
        const int c = __ffs(left) - 1;
        unsigned rows = 0u;
#pragma unroll
        for (int r = 0; r < EST_R; ++r) rows |= ((cm[r] >> c) & 1u) << r;
        nev += __popc(rows);
#pragma unroll 2
        for (int gi = 0; gi < EP_CG; ++gi) {
            const int g = c * EP_CG + gi;
            float4 x[NCH];
#pragma unroll
            for (int ch = 0; ch < NCH; ++ch) x[ch] = tile[g * NCH + ch];
#pragma unroll
            for (int r = 0; r < EST_R; ++r) {
                if (!((rows >> r) & 1u)) continue;         // warp-uniform
                float q[4];
                est_group<NORM, D, WT>(xi[r], yi[r], x, wt, q);
                best = max3f(best, max3f(q[0], q[1], q[2]), q[3]);   // one link of the chain per group
            }
        }
    }
    if (lane == 0) wcnt[warp] = nev;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (lane == 0) red[warp] = best;
    __syncthreads();
    if (tid == 0) {
        float b = red[0];
        int n = wcnt[0];
        for (int w = 1; w < EST_THREADS / 32; ++w) {
            b = fmaxf(b, red[w]);
            n += wcnt[w];
        }
        P.bq[blockIdx.x] = b >= 0.f ? b : -1.f;
        if (b >= 0.f && b > L) atomicMax(P.gbest, __float_as_int(b));   // non-negative floats order as ints
        if (P.work && n) atomicAdd(P.work + 1, (unsigned long long)n);
    }
}

// q* and the list of tile pairs whose largest value reaches q* (1 - 2^-16), for the exact
// selection; one block.
__global__ void estimate_pruned_select_kernel(const EstPrunedParams P, const EstFinalParams F) {
    __shared__ int s_count;
    const int gb = *P.gbest;
    const float qs = gb >= 0 ? __int_as_float(gb) : -1.f;
    if (threadIdx.x == 0) s_count = 0;
    __syncthreads();
    if (qs >= 0.f) {
        const float T = ep_margin(qs);
        const int64_t npairs = (int64_t)P.nb * (P.nb + 1) / 2;
        for (int64_t k = threadIdx.x; k < npairs; k += blockDim.x) {
            if (!(P.bq[k] >= T)) continue;
            int I, J;
            band_pair(k, P.nb, I, J);
            F.list[atomicAdd(&s_count, 1)] = ((unsigned)I << 16) | (unsigned)J;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        F.state->q = qs >= 0.f ? gb : -1;
        F.state->count = s_count;
        F.state->ratio = 0ull;
        F.state->key = ~0ull;
    }
}

template <int NORM, int D>
cudaError_t launch_ep(const EstPrunedParams& P, cudaStream_t st) {
    const int64_t npairs = (int64_t)P.nb * (P.nb + 1) / 2;
    if (P.weighted) estimate_pruned_kernel<NORM, D, true><<<(unsigned)npairs, EST_THREADS, 0, st>>>(P);
    else estimate_pruned_kernel<NORM, D, false><<<(unsigned)npairs, EST_THREADS, 0, st>>>(P);
    return cudaGetLastError();
}

template <int NORM, int... Ds>
cudaError_t ep_dispatch(int d, const EstPrunedParams& P, cudaStream_t st, std::integer_sequence<int, Ds...>) {
    cudaError_t e = cudaErrorInvalidValue;
    ((d == Ds + 1 ? (e = launch_ep<NORM, Ds + 1>(P, st), 0) : 0), ...);
    return e;
}

}  // namespace

constexpr int EP_DMAX = 8;

bool estimate_pruned_available(int d) { return d >= 1 && d <= EP_DMAX; }

cudaError_t launch_estimate_pruned_select(const EstPrunedParams& P, const EstFinalParams& F, cudaStream_t st) {
    estimate_pruned_select_kernel<<<1, 1024, 0, st>>>(P, F);
    return cudaGetLastError();
}

cudaError_t launch_estimate_pruned(int norm, int d, const EstPrunedParams& P, cudaStream_t st) {
    if (!estimate_pruned_available(d)) return cudaErrorInvalidValue;
    const auto seq = std::make_integer_sequence<int, EP_DMAX>{};
    if (norm == LIP_L1) return ep_dispatch<LIP_L1>(d, P, st, seq);
    if (norm == LIP_L2) return ep_dispatch<LIP_L2>(d, P, st, seq);
    return ep_dispatch<LIP_LINF>(d, P, st, seq);
}

}  // namespace lip
