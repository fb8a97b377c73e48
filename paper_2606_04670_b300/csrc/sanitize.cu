// Deferred finiteness check of appended data (lip_add_async, lip_add_host_async).
//
// lip_add checks that new points are finite by reading a flag back, which waits for the
// GPU.  The deferred form never waits: the check runs on the device, records
// ERRBIT_NONFINITE in the handle's status word (reported by lip_check), and replaces
// every new point that holds a NaN or Inf by a copy of a finite point (the handle's first
// point if it already held data, else the first finite new point, else x = 0, y = 0), so
// no later kernel ever reads a non-finite datum.  Two passes over the n new rows:
//   pass 0: per row, finite or not; the lowest finite new row (atomic min on the
//           unsigned row index, the slot preset to 0xffffffff by a memset);
//   pass 1: each non-finite row is overwritten by the source row.
#include "launch.h"

namespace lip {

namespace {

template <typename T>
__device__ __forceinline__ bool row_finite(const T* X, const T* y, int64_t i, int d) {
    bool ok = isfinite((double)y[i]);
    for (int j = 0; j < d; ++j) ok = ok && isfinite((double)X[i * d + j]);
    return ok;
}

template <typename T>
__global__ void sanitize_scan_kernel(const T* X, const T* y, int64_t n0, int64_t n, int d, unsigned* err,
                                     unsigned* first_ok) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t i = n0 + k;
    if (row_finite(X, y, i, d)) atomicMin(first_ok, (unsigned)i);
    else atomicOr(err, ERRBIT_NONFINITE);
}

template <typename T>
__global__ void sanitize_fix_kernel(T* X, T* y, int64_t n0, int64_t n, int d, const unsigned* first_ok) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t i = n0 + k;
    if (row_finite(X, y, i, d)) return;
    // a finite source row (never one of the rows this kernel writes), or none
    const unsigned f = *first_ok;
    const bool has = n0 > 0 || f != 0xffffffffu;
    const int64_t src = n0 > 0 ? 0 : (int64_t)f;
    for (int j = 0; j < d; ++j) X[i * d + j] = has ? X[src * d + j] : T(0);
    y[i] = has ? y[src] : T(0);
}

}  // namespace

cudaError_t launch_sanitize(int es, void* X0, void* y0, int64_t n0, int64_t n, int d, unsigned* err,
                            unsigned* first_ok, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(first_ok, 0xff, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (es == 8) {
        sanitize_scan_kernel<double><<<blocks, 256, 0, st>>>(static_cast<const double*>(X0),
                                                             static_cast<const double*>(y0), n0, n, d, err, first_ok);
        sanitize_fix_kernel<double><<<blocks, 256, 0, st>>>(static_cast<double*>(X0), static_cast<double*>(y0), n0, n,
                                                            d, first_ok);
    } else {
        sanitize_scan_kernel<float><<<blocks, 256, 0, st>>>(static_cast<const float*>(X0),
                                                            static_cast<const float*>(y0), n0, n, d, err, first_ok);
        sanitize_fix_kernel<float><<<blocks, 256, 0, st>>>(static_cast<float*>(X0), static_cast<float*>(y0), n0, n, d,
                                                           first_ok);
    }
    return cudaGetLastError();
}

}  // namespace lip
