// Spatial order of a point set: a 16-bit Morton key per point (the first min(d, 16)
// coordinates, each cut into 2^(16 / D) cells of its bounding box and interleaved), then a
// stable LSD radix sort of the keys in two 8-bit passes, giving the permutation
// position -> index.  Points close in space get close positions, so consecutive runs of
// points are spatially coherent.  Every step is deterministic: counts are atomics on
// integers, the scan has a fixed shape, and within a block the scatter ranks equal digits
// by warp, then lane, which is index order.
#include "launch.h"

namespace lip {

namespace {

constexpr int ORD_THREADS = 256;     // elements per block in the radix passes
constexpr int ORD_WARPS = ORD_THREADS / 32;
constexpr int ORD_BINS = 256;

__device__ __forceinline__ unsigned ord_key_bits(float f) {
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord_key_float(unsigned o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// Per-coordinate bounding box of the finite coordinates (order-preserving bits).
__global__ void ord_bbox_kernel(const float* X, int64_t n, int d, unsigned* box) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int j = 0; j < d && j < 16; ++j) {
        const float v = X[i * d + j];
        if (!isfinite(v)) continue;
        atomicMin(&box[j], ord_key_bits(v));
        atomicMax(&box[16 + j], ord_key_bits(v));
    }
}

__global__ void ord_key_kernel(const float* X, int64_t n, int d, const unsigned* box, unsigned* keys, int* idx) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int D = d < 16 ? d : 16;
    const int b = 16 / D;                          // bits per coordinate
    const int cells = 1 << b;
    int cell[16];
    for (int j = 0; j < D; ++j) {
        const float lo = ord_key_float(box[j]), hi = ord_key_float(box[16 + j]);
        const float v = X[i * d + j];
        int c = 0;
        if (isfinite(v) && hi > lo) {
            const float u = (v - lo) / (hi - lo) * (float)cells;
            c = u >= (float)(cells - 1) ? cells - 1 : (u > 0.f ? (int)u : 0);
        }
        cell[j] = c;
    }
    unsigned key = 0u;
    for (int l = b - 1; l >= 0; --l)
        for (int j = 0; j < D; ++j) key = (key << 1) | (unsigned)((cell[j] >> l) & 1);
    keys[i] = key;
    idx[i] = (int)i;
}

// Digit counts per block, stored digit-major: table[digit * nblocks + block].
__global__ void __launch_bounds__(ORD_THREADS) ord_hist_kernel(const unsigned* keys, int64_t n, int shift,
                                                              int* table, int nblocks) {
    __shared__ int cnt[ORD_BINS];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * ORD_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 0xffu], 1);
    __syncthreads();
    table[(int64_t)threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// Exclusive prefix sums of the table in place (one block; each thread takes a contiguous
// run, then the runs' totals are scanned).
__global__ void __launch_bounds__(1024) ord_scan_kernel(int* table, int64_t total) {
    __shared__ int part[1024];
    const int t = threadIdx.x;
    const int64_t per = (total + 1023) / 1024;
    const int64_t a = (int64_t)t * per, b = a + per < total ? a + per : total;
    int s = 0;
    for (int64_t i = a; i < b; ++i) s += table[i];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = t > 0 ? part[t - 1] : 0;
    for (int64_t i = a; i < b; ++i) {
        const int v = table[i];
        table[i] = run;
        run += v;
    }
}

// Stable scatter: position = start of the digit in this block (from the scanned table) +
// count of the digit in earlier warps of the block + count among earlier lanes.
__global__ void __launch_bounds__(ORD_THREADS) ord_scatter_kernel(const unsigned* keys, const int* idx, int64_t n,
                                                                 int shift, const int* table, int nblocks,
                                                                 unsigned* keys_out, int* idx_out) {
    __shared__ int wc[ORD_WARPS][ORD_BINS + 1];
    for (int i = threadIdx.x; i < ORD_WARPS * (ORD_BINS + 1); i += ORD_THREADS) (&wc[0][0])[i] = 0;
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * ORD_THREADS + threadIdx.x;
    const bool valid = i < n;
    const unsigned key = valid ? keys[i] : 0u;
    const int digit = valid ? (int)((key >> shift) & 0xffu) : ORD_BINS;     // ORD_BINS: no element
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const unsigned peers = __match_any_sync(0xffffffffu, digit);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (rank == 0) wc[warp][digit] = __popc(peers);
    __syncthreads();
    {
        // exclusive prefix over the warps, one digit per thread
        const int dgt = threadIdx.x;
        int run = 0;
        for (int w = 0; w < ORD_WARPS; ++w) {
            const int v = wc[w][dgt];
            wc[w][dgt] = run;
            run += v;
        }
    }
    __syncthreads();
    if (!valid) return;
    const int64_t pos = (int64_t)table[(int64_t)digit * nblocks + blockIdx.x] + wc[warp][digit] + rank;
    keys_out[pos] = key;
    idx_out[pos] = idx[i];
}

}  // namespace

size_t spatial_order_scratch(int64_t n) {
    const int64_t nb = (n + ORD_THREADS - 1) / ORD_THREADS;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    return al(32 * sizeof(unsigned)) + 2 * al((size_t)n * sizeof(unsigned)) + al((size_t)n * sizeof(int)) +
           al((size_t)nb * ORD_BINS * sizeof(int));
}

cudaError_t spatial_order(const float* X, int64_t n, int d, int* perm, void* scratch, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const int nb = (int)((n + ORD_THREADS - 1) / ORD_THREADS);
    char* s = static_cast<char*>(scratch);
    unsigned* box = reinterpret_cast<unsigned*>(s);
    unsigned* ka = reinterpret_cast<unsigned*>(s + al(32 * sizeof(unsigned)));
    unsigned* kb = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(ka) + al((size_t)n * sizeof(unsigned)));
    int* ia = reinterpret_cast<int*>(reinterpret_cast<char*>(kb) + al((size_t)n * sizeof(unsigned)));
    int* table = reinterpret_cast<int*>(reinterpret_cast<char*>(ia) + al((size_t)n * sizeof(int)));
    cudaError_t e = cudaMemsetAsync(box, 0xff, 16 * sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(box + 16, 0, 16 * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)nb;
    ord_bbox_kernel<<<blocks, ORD_THREADS, 0, st>>>(X, n, d, box);
    ord_key_kernel<<<blocks, ORD_THREADS, 0, st>>>(X, n, d, box, ka, perm);
    // pass 1: low byte (ka, perm) -> (kb, ia); pass 2: high byte (kb, ia) -> (ka, perm)
    ord_hist_kernel<<<blocks, ORD_THREADS, 0, st>>>(ka, n, 0, table, nb);
    ord_scan_kernel<<<1, 1024, 0, st>>>(table, (int64_t)nb * ORD_BINS);
    ord_scatter_kernel<<<blocks, ORD_THREADS, 0, st>>>(ka, perm, n, 0, table, nb, kb, ia);
    ord_hist_kernel<<<blocks, ORD_THREADS, 0, st>>>(kb, n, 8, table, nb);
    ord_scan_kernel<<<1, 1024, 0, st>>>(table, (int64_t)nb * ORD_BINS);
    ord_scatter_kernel<<<blocks, ORD_THREADS, 0, st>>>(kb, ia, n, 8, table, nb, ka, perm);
    return cudaGetLastError();
}

int spatial_order_launches() { return 8; }

}  // namespace lip
