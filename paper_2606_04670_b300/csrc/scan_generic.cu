// Generic scan kernels (any shape up to D_MAX, FP32 or FP64), split merge, layout builder.
#include "launch.h"

namespace lip {

template <typename T, int NORM, int DP>
cudaError_t launch_scan_generic(const ScanParams& P, int gx, int gy, cudaStream_t st) {
    constexpr int R = generic_rows(DP);
    scan_generic_kernel<T, NORM, DP, R><<<dim3(gx, gy), SCAN_THREADS, 0, st>>>(P);
    return cudaGetLastError();
}

template <typename T, int NORM, int DP>
static ScanKernelInfo gen_info() {
    ScanKernelInfo e;
    e.launch = &launch_scan_generic<T, NORM, DP>;
    e.kernel = reinterpret_cast<const void*>(&scan_generic_kernel<T, NORM, DP, generic_rows(DP)>);
    e.rows = generic_rows(DP);
    e.nch = DP + 1;
    return e;
}

template <typename T, int NORM>
static ScanKernelInfo gen_by_dim(int dl) {
    switch (dl) {
        case 2: return gen_info<T, NORM, 2>();
        case 4: return gen_info<T, NORM, 4>();
        case 8: return gen_info<T, NORM, 8>();
        case 12: return gen_info<T, NORM, 12>();
        case 16: return gen_info<T, NORM, 16>();
        case 24: return gen_info<T, NORM, 24>();
        case 32: return gen_info<T, NORM, 32>();
        default: return {};
    }
}

template <typename T>
static ScanKernelInfo gen_by_norm(int norm, int dl) {
    switch (norm) {
        case LIP_L1: return gen_by_dim<T, LIP_L1>(dl);
        case LIP_L2: return gen_by_dim<T, LIP_L2>(dl);
        case LIP_LINF: return gen_by_dim<T, LIP_LINF>(dl);
        default: return {};
    }
}

ScanKernelInfo scan_generic_info(int elem_bytes, int norm, int dl) {
    return elem_bytes == 8 ? gen_by_norm<double>(norm, dl) : gen_by_norm<float>(norm, dl);
}

ScanKernelInfo scan_exact_info_l1(int C, int U, int v);
ScanKernelInfo scan_exact_info_l2(int C, int U, int v);
ScanKernelInfo scan_exact_info_linf(int C, int U, int v);

ScanKernelInfo scan_exact_info(int norm, int C, int U, int variant) {
    switch (norm) {
        case LIP_L1: return scan_exact_info_l1(C, U, variant);
        case LIP_L2: return scan_exact_info_l2(C, U, variant);
        case LIP_LINF: return scan_exact_info_linf(C, U, variant);
        default: return {};
    }
}

static unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

cudaError_t launch_merge(int elem_bytes, const MergeParams& P, cudaStream_t st) {
    if (P.nq <= 0) return cudaSuccess;
    if (elem_bytes == 8) merge_kernel<double><<<blocks_for(P.nq, 256), 256, 0, st>>>(P);
    else merge_kernel<float><<<blocks_for(P.nq, 256), 256, 0, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_build_hot(int elem_bytes, const HotParams& P, cudaStream_t st) {
    const int64_t n = P.k1 - P.k0;
    if (n <= 0) return cudaSuccess;
    if (elem_bytes == 8) build_hot_kernel<double><<<blocks_for(n, 256), 256, 0, st>>>(P);
    else build_hot_kernel<float><<<blocks_for(n, 256), 256, 0, st>>>(P);
    return cudaGetLastError();
}

// The FMA-pipe square root of the exact kernels' variants 2-5, element by element (tests).
__global__ void sqrt_fma_kernel(const float* s, float* out, int64_t n) {
    const int64_t i = 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (i >= n) return;
    const float2 r = sqrt_fma2(make_float2(s[i], i + 1 < n ? s[i + 1] : 0.f));
    out[i] = r.x;
    if (i + 1 < n) out[i + 1] = r.y;
}

cudaError_t launch_sqrt_fma(const float* s, float* out, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    sqrt_fma_kernel<<<blocks_for((n + 1) / 2, 256), 256, 0, st>>>(s, out, n);
    return cudaGetLastError();
}

cudaError_t launch_pad_hot(int elem_bytes, void* hot, int64_t k0, int64_t k1, int nch, int dl, cudaStream_t st) {
    const int64_t n = k1 - k0;
    if (n <= 0) return cudaSuccess;
    if (elem_bytes == 8) pad_hot_kernel<double><<<blocks_for(n, 256), 256, 0, st>>>(hot, k0, k1, nch, dl);
    else pad_hot_kernel<float><<<blocks_for(n, 256), 256, 0, st>>>(hot, k0, k1, nch, dl);
    return cudaGetLastError();
}

}  // namespace lip
