// Multi-GPU evaluation by data shards (one process per GPU): each rank holds a slice of
// the data and scans it; the ranks' partial extrema are merged by one all-reduce MIN on
// packed 64-bit keys, the owner of each winning datum re-evaluates it in FP64, and a
// second all-reduce (MIN of the upper values, MAX of the lower ones) gives every rank the
// exact bounds.  The kernels here are the per-rank steps around those two collectives.
//
// Key of a bound (the order of the single-GPU merge): the FP32 scan value made orderable
// as an unsigned 32-bit integer (smaller value first for the upper bound, larger first for
// the lower bound through -v), shifted left by 31, with the global data index (< 2^31) in
// the low 31 bits.  The MIN over ranks is then the smallest value with the lowest index
// on ties, which is what lip_eval's split merge takes on one GPU, so a data-sharded
// evaluation returns lip_eval's results bit for bit.  INT64_MAX means "no candidate"
// (no data in the shard, or a non-finite query).
#include "launch.h"

namespace lip {

constexpr int64_t SHARD_NONE = 0x7fffffffffffffffll;
constexpr int64_t SHARD_IDX_MASK = 0x7fffffffll;

__device__ __forceinline__ int64_t shard_key(float v, int64_t idx) {
    return ((int64_t)f2ord(v) << 31) | (idx & SHARD_IDX_MASK);
}

// Per query: the best of the splits (lowest split, hence lowest index, on exact ties) as
// packed keys with the global index index_base + local index.
template <typename T>
__global__ void shard_keys_kernel(const PartialRec<float>* part, int nsplit, int64_t nq, const T* Q, int d,
                                  int64_t index_base, int64_t* key_up, int64_t* key_lo) {
    const int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= nq) return;
    float bu = 0.f, bl = 0.f;
    int iu = -1, il = -1;
    for (int s = 0; s < nsplit; ++s) {
        const PartialRec<float> r = part[(int64_t)s * nq + qi];
        if (r.iu >= 0 && (iu < 0 || r.vu < bu)) { bu = r.vu; iu = r.iu; }
        if (r.il >= 0 && (il < 0 || r.vl > bl)) { bl = r.vl; il = r.il; }
    }
    bool finite = true;
    for (int i = 0; i < d; ++i) finite = finite && isfinite((double)Q[qi * d + i]);
    key_up[qi] = (finite && iu >= 0) ? shard_key(bu, index_base + iu) : SHARD_NONE;
    key_lo[qi] = (finite && il >= 0) ? shard_key(-bl, index_base + il) : SHARD_NONE;
}

// Owner's FP64 re-evaluation: for each query whose winning global index falls in this
// rank's range [index_base, index_base + N), the exact bound of that datum (as the split
// merge computes it); +Inf / -Inf elsewhere, the neutral values of the MIN / MAX that
// follows.
template <typename T>
__global__ void shard_reeval_kernel(const MergeParams P, int64_t index_base, int64_t N, const int64_t* key_up,
                                    const int64_t* key_lo, double* hi64, double* lo64) {
    const int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= P.nq) return;
    const T* q = static_cast<const T*>(P.Q) + qi * P.d;
    const T* X0 = static_cast<const T*>(P.X0);
    const T* y0 = static_cast<const T*>(P.y0);
    double hi = INFINITY, lo = -INFINITY;
    const int64_t ku = key_up[qi], kl = key_lo[qi];
    if (ku != SHARD_NONE) {
        const int64_t k = (ku & SHARD_IDX_MASK) - index_base;
        if (k >= 0 && k < N) hi = (double)y0[k] + P.M * dist_fp64<T>(P, q, X0 + k * P.d, +1);
    }
    if (kl != SHARD_NONE) {
        const int64_t k = (kl & SHARD_IDX_MASK) - index_base;
        if (k >= 0 && k < N) lo = (double)y0[k] - P.M * dist_fp64<T>(P, q, X0 + k * P.d, -1);
    }
    hi64[qi] = hi;
    lo64[qi] = lo;
}

// The outputs from the merged keys and the merged exact bounds, as the split merge writes
// them: g = (hi + lo) / 2 in FP64, rounded once; NaN and -1 without a candidate.
template <typename T>
__global__ void shard_finish_kernel(int64_t nq, const int64_t* key_up, const int64_t* key_lo, const double* hi64,
                                    const double* lo64, T* g, T* lo, T* hi, int32_t* idx_up, int32_t* idx_lo) {
    const int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= nq) return;
    const int64_t ku = key_up[qi], kl = key_lo[qi];
    double h = hi64[qi], l = lo64[qi];
    int iu = -1, il = -1;
    if (ku == SHARD_NONE || kl == SHARD_NONE) {
        h = l = __longlong_as_double(0x7ff8000000000000ll);
    } else {
        iu = (int)(ku & SHARD_IDX_MASK);
        il = (int)(kl & SHARD_IDX_MASK);
    }
    if (g) g[qi] = (T)(0.5 * (h + l));
    if (lo) lo[qi] = (T)l;
    if (hi) hi[qi] = (T)h;
    if (idx_up) idx_up[qi] = iu;
    if (idx_lo) idx_lo[qi] = il;
}

static unsigned blocks_for(int64_t n) { return (unsigned)((n + 255) / 256); }

cudaError_t launch_shard_keys(int elem_bytes, const void* partial, int nsplit, int64_t nq, const void* Q, int d,
                              int64_t index_base, int64_t* key_up, int64_t* key_lo, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    const PartialRec<float>* p = static_cast<const PartialRec<float>*>(partial);
    if (elem_bytes == 8)
        shard_keys_kernel<double><<<blocks_for(nq), 256, 0, st>>>(p, nsplit, nq, static_cast<const double*>(Q), d,
                                                                  index_base, key_up, key_lo);
    else
        shard_keys_kernel<float><<<blocks_for(nq), 256, 0, st>>>(p, nsplit, nq, static_cast<const float*>(Q), d,
                                                                 index_base, key_up, key_lo);
    return cudaGetLastError();
}

cudaError_t launch_shard_reeval(int elem_bytes, const MergeParams& P, int64_t index_base, int64_t N,
                                const int64_t* key_up, const int64_t* key_lo, double* hi64, double* lo64,
                                cudaStream_t st) {
    if (P.nq <= 0) return cudaSuccess;
    if (elem_bytes == 8)
        shard_reeval_kernel<double><<<blocks_for(P.nq), 256, 0, st>>>(P, index_base, N, key_up, key_lo, hi64, lo64);
    else
        shard_reeval_kernel<float><<<blocks_for(P.nq), 256, 0, st>>>(P, index_base, N, key_up, key_lo, hi64, lo64);
    return cudaGetLastError();
}

cudaError_t launch_shard_finish(int elem_bytes, int64_t nq, const int64_t* key_up, const int64_t* key_lo,
                                const double* hi64, const double* lo64, void* g, void* lo, void* hi, int32_t* idx_up,
                                int32_t* idx_lo, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    if (elem_bytes == 8)
        shard_finish_kernel<double><<<blocks_for(nq), 256, 0, st>>>(nq, key_up, key_lo, hi64, lo64,
                                                                    static_cast<double*>(g), static_cast<double*>(lo),
                                                                    static_cast<double*>(hi), idx_up, idx_lo);
    else
        shard_finish_kernel<float><<<blocks_for(nq), 256, 0, st>>>(nq, key_up, key_lo, hi64, lo64,
                                                                   static_cast<float*>(g), static_cast<float*>(lo),
                                                                   static_cast<float*>(hi), idx_up, idx_lo);
    return cudaGetLastError();
}

}  // namespace lip
