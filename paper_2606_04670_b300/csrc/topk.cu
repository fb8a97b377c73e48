// k > 1 neighbours (Sec. 5, extra features): H_up^k = sum_j wk_j v_(j) over the k smallest
// upper bounds y^i + M dist_up(q, x^i), H_lo^k over the k largest lower bounds, g their
// midpoint.  The scan keeps, per query and per data split, sorted lists of the K best
// values (K = k rounded up to 2, 4 or 8; the extra weights are zero) with strict
// comparisons, so equal values stay in data-index order; the merge picks the k best over
// the splits by (value, index), re-evaluates them in FP64 from the caller's data, and
// forms the weighted sums.  It reads the same scan layout as lip_eval (coordinates
// scaled by M w and mirrored, y after them).
#include "launch.h"

namespace lip {

constexpr int TOPK_THREADS = 128;

// DM: register arrays for a layout of up to DM coordinates (16, or 32 for the widest handles)
template <typename T, int NORM, int K, int DM>
__global__ void __launch_bounds__(TOPK_THREADS) topk_scan_kernel(const TopkParams P) {
    using V4 = typename Vec4<T>::type;
    const int64_t qi = (int64_t)blockIdx.x * TOPK_THREADS + threadIdx.x;
    const int split = blockIdx.y;
    const T inf = (T)INFINITY;
    T q[DM];
    const T* Qp = static_cast<const T*>(P.Q);
#pragma unroll
    for (int j = 0; j < DM; ++j)
        q[j] = (qi < P.nq && j < P.d) ? (T)(P.scale[j] * (double)Qp[qi * P.d + P.perm[j]]) : (T)0;
    T bu[K], bl[K];
    int ku[K], kl[K];
#pragma unroll
    for (int e = 0; e < K; ++e) { bu[e] = inf; bl[e] = -inf; ku[e] = -1; kl[e] = -1; }
    const V4* hot = static_cast<const V4*>(P.hot);
    const int64_t g0 = (int64_t)split * P.groups_per_split;
    const int64_t g1 = g0 + P.groups_per_split < P.ngroups ? g0 + P.groups_per_split : P.ngroups;
    for (int64_t g = g0; g < g1 && qi < P.nq; ++g) {
        T x[DM + 1][4];
#pragma unroll
        for (int ch = 0; ch <= DM; ++ch) {
            if (ch < P.dl || ch == P.dl) {
                const V4 v = hot[g * P.nch + (ch < P.dl ? ch : P.dl)];
                const int c = ch < P.dl ? ch : DM;
                x[c][0] = v.x; x[c][1] = v.y; x[c][2] = v.z; x[c][3] = v.w;
            }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            T au = 0, al = 0;
#pragma unroll
            for (int j = 0; j < DM; ++j) {
                if (j >= P.dl) break;
                const T t = q[j] - x[j][e];
                T u, l;
                if (j < P.C) { u = t > 0 ? t : (T)0; l = t < 0 ? -t : (T)0; }
                else { u = t < 0 ? -t : t; l = u; }
                if (NORM == LIP_L1) { au += u; al += l; }
                else if (NORM == LIP_L2) { au += u * u; al += l * l; }
                else { au = u > au ? u : au; al = l > al ? l : al; }
            }
            if (NORM == LIP_L2) { au = sqrt(au); al = sqrt(al); }
            const int k = (int)(g * 4 + e);
            T vu = x[DM][e] + au, vl = x[DM][e] - al;
            if (vu < bu[K - 1]) {           // bubble the new value into the ascending list
                int kk = k;
#pragma unroll
                for (int p = 0; p < K; ++p)
                    if (vu < bu[p]) {
                        const T tv = bu[p]; bu[p] = vu; vu = tv;
                        const int tk = ku[p]; ku[p] = kk; kk = tk;
                    }
            }
            if (vl > bl[K - 1]) {           // and into the descending list
                int kk = k;
#pragma unroll
                for (int p = 0; p < K; ++p)
                    if (vl > bl[p]) {
                        const T tv = bl[p]; bl[p] = vl; vl = tv;
                        const int tk = kl[p]; kl[p] = kk; kk = tk;
                    }
            }
        }
    }
    if (qi >= P.nq) return;
    T* pv = static_cast<T*>(P.partial);
    const int64_t base = ((int64_t)split * P.nq + qi) * 2 * K;
    int* pk = reinterpret_cast<int*>(pv + (int64_t)gridDim.y * P.nq * 2 * K);
#pragma unroll
    for (int e = 0; e < K; ++e) {
        pv[base + e] = bu[e];
        pk[base + e] = ku[e];
        pv[base + K + e] = bl[e];
        pk[base + K + e] = kl[e];
    }
}

template <typename T>
__global__ void topk_merge_kernel(const TopkMergeParams P) {
    const int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= P.nq) return;
    const T* pv = static_cast<const T*>(P.partial);
    const int* pk = reinterpret_cast<const int*>(pv + (int64_t)P.nsplit * P.nq * 2 * P.K);
    const T* q = static_cast<const T*>(P.Q) + qi * P.d;
    bool finite = true;
    for (int i = 0; i < P.d; ++i) finite = finite && isfinite((double)q[i]);
    MergeParams mp{};
    mp.d = P.d;
    mp.norm = P.norm;
    for (int i = 0; i < D_MAX; ++i) { mp.mon[i] = P.mon[i]; mp.w[i] = P.w[i]; }
    double res[2];
    for (int side = 0; side < 2; ++side) {
        // k best over the splits by (approximate value, index)
        T sv[8];
        int sk[8];
        for (int e = 0; e < P.k; ++e) { sv[e] = side == 0 ? (T)INFINITY : -(T)INFINITY; sk[e] = -1; }
        for (int s = 0; s < P.nsplit; ++s) {
            const int64_t base = ((int64_t)s * P.nq + qi) * 2 * P.K + side * P.K;
            for (int e = 0; e < P.K; ++e) {
                T v = pv[base + e];
                int kk = pk[base + e];
                if (kk < 0) break;
                for (int p = 0; p < P.k; ++p) {
                    const bool better = sk[p] < 0 || (side == 0 ? v < sv[p] : v > sv[p]) || (v == sv[p] && kk < sk[p]);
                    if (better) {
                        const T tv = sv[p]; sv[p] = v; v = tv;
                        const int tk = sk[p]; sk[p] = kk; kk = tk;
                        if (kk < 0) break;
                    }
                }
            }
        }
        // exact values in FP64, ordered again by (value, index) before weighting
        double ev[8];
        int ek[8];
        bool all = finite;
        for (int e = 0; e < P.k; ++e) {
            ek[e] = sk[e];
            if (sk[e] < 0) { all = false; ev[e] = 0.0; continue; }
            const T* x = static_cast<const T*>(P.X0) + (int64_t)sk[e] * P.d;
            const double dist = dist_fp64<T>(mp, q, x, side == 0 ? +1 : -1);
            const double yy = (double)static_cast<const T*>(P.y0)[sk[e]];
            ev[e] = side == 0 ? yy + P.M * dist : yy - P.M * dist;
        }
        for (int a = 1; a < P.k; ++a)
            for (int b = a; b > 0; --b) {
                const bool sw = side == 0 ? (ev[b] < ev[b - 1] || (ev[b] == ev[b - 1] && ek[b] < ek[b - 1]))
                                          : (ev[b] > ev[b - 1] || (ev[b] == ev[b - 1] && ek[b] < ek[b - 1]));
                if (!sw) break;
                const double tv = ev[b]; ev[b] = ev[b - 1]; ev[b - 1] = tv;
                const int tk = ek[b]; ek[b] = ek[b - 1]; ek[b - 1] = tk;
            }
        double sum = 0.0;
        for (int e = 0; e < P.k; ++e) sum += P.wk[e] * ev[e];
        res[side] = all ? sum : __longlong_as_double(0x7ff8000000000000ll);
        int32_t* out = side == 0 ? P.idx_up : P.idx_lo;
        if (out)
            for (int e = 0; e < P.k; ++e) out[qi * P.k + e] = all ? ek[e] : -1;
    }
    if (P.g) static_cast<T*>(P.g)[qi] = (T)(0.5 * (res[0] + res[1]));
    if (P.hi) static_cast<T*>(P.hi)[qi] = (T)res[0];
    if (P.lo) static_cast<T*>(P.lo)[qi] = (T)res[1];
}

template <typename T, int NORM, int DM>
static cudaError_t topk_by_k(int K, const TopkParams& P, int gx, int gy, cudaStream_t st) {
    if (K == 2) topk_scan_kernel<T, NORM, 2, DM><<<dim3(gx, gy), TOPK_THREADS, 0, st>>>(P);
    else if (K == 4) topk_scan_kernel<T, NORM, 4, DM><<<dim3(gx, gy), TOPK_THREADS, 0, st>>>(P);
    else topk_scan_kernel<T, NORM, 8, DM><<<dim3(gx, gy), TOPK_THREADS, 0, st>>>(P);
    return cudaGetLastError();
}

template <typename T, int DM>
static cudaError_t topk_by_norm_w(int norm, int K, const TopkParams& P, int gx, int gy, cudaStream_t st) {
    if (norm == LIP_L1) return topk_by_k<T, LIP_L1, DM>(K, P, gx, gy, st);
    if (norm == LIP_L2) return topk_by_k<T, LIP_L2, DM>(K, P, gx, gy, st);
    return topk_by_k<T, LIP_LINF, DM>(K, P, gx, gy, st);
}

template <typename T>
static cudaError_t topk_by_norm(int norm, int K, const TopkParams& P, int gx, int gy, cudaStream_t st) {
    return P.dl > 16 ? topk_by_norm_w<T, 32>(norm, K, P, gx, gy, st) : topk_by_norm_w<T, 16>(norm, K, P, gx, gy, st);
}

int topk_threads() { return TOPK_THREADS; }

cudaError_t launch_topk(int elem_bytes, int norm, int K, const TopkParams& P, int gx, int gy, const TopkMergeParams& M,
                        cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (gy > 0) {
        e = elem_bytes == 8 ? topk_by_norm<double>(norm, K, P, gx, gy, st) : topk_by_norm<float>(norm, K, P, gx, gy, st);
        if (e != cudaSuccess) return e;
    }
    const unsigned gm = (unsigned)((M.nq + 127) / 128);
    if (elem_bytes == 8) topk_merge_kernel<double><<<gm, 128, 0, st>>>(M);
    else topk_merge_kernel<float><<<gm, 128, 0, st>>>(M);
    return cudaGetLastError();
}

}  // namespace lip
