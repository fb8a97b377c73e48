// Host-side pieces of the pruned scan (scan_pruned.cuh): the chunk records of the
// position-ordered layout and the kernel tables of the three norms.
#include "launch.h"
#include "scan_pruned_inst.cuh"

namespace lip {

PrunedKernelInfo scan_pruned_info_l1(int C, int U, int v);
PrunedKernelInfo scan_pruned_info_l2(int C, int U, int v);
PrunedKernelInfo scan_pruned_info_linf(int C, int U, int v);

namespace {

// One thread per `cpts`-point chunk of the layout `hot` (groups of 4 points, nch float4
// channels: coordinates 0..D-1, y, then aux when `aux`): the box of its real points
// (positions < N) in layout coordinates, the smallest y and the largest value of the
// lower bound's channel (aux when present, else y).  A chunk without real points gets NaN.
__global__ void pruned_box_kernel(const float* hot, int64_t N, int64_t nchunks, int D, int nch, int aux, int nb4,
                                  int cpts, float4* box) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nchunks) return;
    float lo[D_MAX], hi[D_MAX];
    for (int j = 0; j < D; ++j) {
        lo[j] = __int_as_float(0x7f800000);
        hi[j] = -__int_as_float(0x7f800000);
    }
    float ylo = __int_as_float(0x7f800000), yhv = -__int_as_float(0x7f800000);
    bool any = false;
    for (int p = 0; p < cpts; ++p) {
        const int64_t pos = c * cpts + p;
        if (pos >= N) break;
        const int64_t g = pos / GROUP, e = pos % GROUP;
        const float* base = hot + (g * nch) * GROUP + e;
        for (int j = 0; j < D; ++j) {
            const float v = base[j * GROUP];
            lo[j] = fminf(lo[j], v);
            hi[j] = fmaxf(hi[j], v);
        }
        const float y = base[D * GROUP];
        ylo = fminf(ylo, y);
        yhv = fmaxf(yhv, aux ? base[(D + 1) * GROUP] : y);
        any = true;
    }
    float* out = reinterpret_cast<float*>(box + c * nb4);
    const float nan = __int_as_float(0x7fc00000);
    for (int j = 0; j < D; ++j) {
        out[j] = any ? lo[j] : nan;
        out[D + j] = any ? hi[j] : nan;
    }
    out[2 * D] = any ? ylo : nan;
    out[2 * D + 1] = any ? yhv : nan;
    for (int k = 2 * D + 2; k < nb4 * 4; ++k) out[k] = 0.f;
}

// One thread per `per` consecutive chunks: the union of their records (chunks without
// data, NaN, drop out of the min / max; all empty gives NaN).
__global__ void pruned_super_kernel(const float4* box, int64_t nsuper, int per, int D, int nb4, float4* sbox) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsuper) return;
    float* out = reinterpret_cast<float*>(sbox + s * nb4);
    const float inf = __int_as_float(0x7f800000), nan = __int_as_float(0x7fc00000);
    for (int j = 0; j < D; ++j) {
        out[j] = inf;
        out[D + j] = -inf;
    }
    out[2 * D] = inf;
    out[2 * D + 1] = -inf;
    bool any = false;
    for (int c = 0; c < per; ++c) {
        const float* b = reinterpret_cast<const float*>(box + (s * per + c) * nb4);
        if (!(b[2 * D] == b[2 * D])) continue;
        any = true;
        for (int j = 0; j < D; ++j) {
            out[j] = fminf(out[j], b[j]);
            out[D + j] = fmaxf(out[D + j], b[D + j]);
        }
        out[2 * D] = fminf(out[2 * D], b[2 * D]);
        out[2 * D + 1] = fmaxf(out[2 * D + 1], b[2 * D + 1]);
    }
    if (!any)
        for (int k = 0; k < 2 * D + 2; ++k) out[k] = nan;
    for (int k = 2 * D + 2; k < nb4 * 4; ++k) out[k] = 0.f;
}

}  // namespace

PrunedKernelInfo scan_pruned_info(int norm, int C, int U, int variant) {
    switch (norm) {
        case LIP_L1: return scan_pruned_info_l1(C, U, variant);
        case LIP_L2: return scan_pruned_info_l2(C, U, variant);
        case LIP_LINF: return scan_pruned_info_linf(C, U, variant);
        default: return {};
    }
}

int pruned_box_floats(int D) { return pruned_box_f4(D) * 4; }

cudaError_t launch_chunk_records(const void* hot, int64_t N, int64_t nchunks, int D, int nch, bool aux, void* box,
                                 cudaStream_t st, int cpts) {
    if (nchunks <= 0) return cudaSuccess;
    pruned_box_kernel<<<(unsigned)((nchunks + 127) / 128), 128, 0, st>>>(
        static_cast<const float*>(hot), N, nchunks, D, nch, aux ? 1 : 0, pruned_box_f4(D), cpts,
        static_cast<float4*>(box));
    return cudaGetLastError();
}

cudaError_t launch_pruned_boxes(const void* hot, int64_t N, int64_t nchunks, int D, int nch, bool aux, void* box,
                                void* sbox, cudaStream_t st) {
    cudaError_t e = launch_chunk_records(hot, N, nchunks, D, nch, aux, box, st, PRUNED_CG * GROUP);
    if (e != cudaSuccess) return e;
    return launch_record_union(box, nchunks / PRUNED_CPS, PRUNED_CPS, D, sbox, st);
}

cudaError_t launch_record_union(const void* box, int64_t nsuper, int per, int D, void* sbox, cudaStream_t st) {
    if (nsuper <= 0) return cudaSuccess;
    pruned_super_kernel<<<(unsigned)((nsuper + 127) / 128), 128, 0, st>>>(static_cast<const float4*>(box), nsuper, per,
                                                                          D, pruned_box_f4(D),
                                                                          static_cast<float4*>(sbox));
    return cudaGetLastError();
}

}  // namespace lip
