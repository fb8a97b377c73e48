// Host-side pieces of the pruned scan (scan_pruned.cuh): the chunk records of the
// position-ordered layout and the kernel tables of the three norms.
#include "launch.h"
#include "scan_pruned_inst.cuh"

namespace lip {

PrunedKernelInfo scan_pruned_info_l1(int C, int U, int v);
PrunedKernelInfo scan_pruned_info_l2(int C, int U, int v);
PrunedKernelInfo scan_pruned_info_linf(int C, int U, int v);

namespace {

// One warp per `cpts`-point chunk (cpts <= 32) of the layout `hot` (groups of 4 points,
// nch float4 channels: coordinates 0..D-1, y, then aux when `aux`), lane p reading point
// p: the box of its real points (positions < N) in layout coordinates, the smallest y and
// the largest value of the lower bound's channel (aux when present, else y).  A chunk
// without real points gets NaN.
__global__ void pruned_box_kernel(const float* hot, int64_t N, int64_t nchunks, int D, int nch, int aux, int nb4,
                                  int cpts, float4* box) {
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    if (c >= nchunks) return;                      // whole warps leave together
    const int64_t pos = c * cpts + lane;
    const bool real = lane < cpts && pos < N;
    const float* base = hot + ((pos / GROUP) * nch) * GROUP + pos % GROUP;
    const float inf = __int_as_float(0x7f800000), nan = __int_as_float(0x7fc00000);
    const bool any = __any_sync(0xffffffffu, real);
    float* out = reinterpret_cast<float*>(box + c * nb4);
    for (int k = 0; k < 2 * D + 2; ++k) {
        // lo (k < D) and ylo (k = 2D) fold by min from the coordinate / y channel, hi and
        // the value maximum by max from the coordinate / lower-bound channel
        const bool is_min = k < D || k == 2 * D;
        const int ch = k < D ? k : (k < 2 * D ? k - D : (k == 2 * D ? D : (aux ? D + 1 : D)));
        float v = real ? base[ch * GROUP] : (is_min ? inf : -inf);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float w = __shfl_xor_sync(0xffffffffu, v, o);
            v = is_min ? fminf(v, w) : fmaxf(v, w);
        }
        if (lane == 0) out[k] = any ? v : nan;
    }
    if (lane == 0)
        for (int k = 2 * D + 2; k < nb4 * 4; ++k) out[k] = 0.f;
}

// One warp per `per` consecutive chunks (per <= 32): lane c reads chunk c's record and
// the lanes fold the union (chunks without data, NaN, drop out of the min / max; all
// empty gives NaN).
__global__ void pruned_super_kernel(const float4* box, int64_t nsuper, int per, int D, int nb4, float4* sbox) {
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    if (s >= nsuper) return;                       // whole warps leave together
    const float inf = __int_as_float(0x7f800000), nan = __int_as_float(0x7fc00000);
    const float* b = reinterpret_cast<const float*>(box + (s * per + lane) * nb4);
    const bool has = lane < per && b[2 * D] == b[2 * D];
    const bool any = __any_sync(0xffffffffu, has);
    float* out = reinterpret_cast<float*>(sbox + s * nb4);
    for (int k = 0; k < 2 * D + 2; ++k) {
        // lo (k < D) and ylo (k = 2D) fold by min, hi and the value maximum by max
        const bool is_min = k < D || k == 2 * D;
        float v = has ? b[k] : (is_min ? inf : -inf);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float w = __shfl_xor_sync(0xffffffffu, v, o);
            v = is_min ? fminf(v, w) : fmaxf(v, w);
        }
        if (lane == 0) out[k] = any ? v : nan;
    }
    if (lane == 0)
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
    if (cpts < 1 || cpts > 32) return cudaErrorInvalidValue;
    pruned_box_kernel<<<(unsigned)((nchunks * 32 + 127) / 128), 128, 0, st>>>(
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
    if (per < 1 || per > 32) return cudaErrorInvalidValue;
    pruned_super_kernel<<<(unsigned)((nsuper * 32 + 127) / 128), 128, 0, st>>>(static_cast<const float4*>(box), nsuper,
                                                                               per, D, pruned_box_f4(D),
                                                                               static_cast<float4*>(sbox));
    return cudaGetLastError();
}

}  // namespace lip
