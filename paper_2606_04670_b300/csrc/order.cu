// Spatial order of a point set: a 16-bit Hilbert key per point (the first min(d, 16)
// coordinates, each cut into 2^(16 / D) cells of its bounding box), then a
// stable LSD radix sort of the keys in two 8-bit passes, giving the permutation
// position -> index.  Points close in space get close positions, so consecutive runs of
// points are spatially coherent.  Every step is deterministic: counts are atomics on
// integers, the scan has a fixed shape, and within a block the scatter ranks equal digits
// by sub-tile, then warp, then lane, which is index order.
#include "launch.h"

namespace lip {

namespace {

constexpr int ORD_THREADS = 256;                    // threads per block in the radix passes
constexpr int ORD_WARPS = ORD_THREADS / 32;
constexpr int ORD_SUB = 16;                         // most 256-key sub-tiles per block, in index order
constexpr int ORD_TILE = ORD_THREADS * ORD_SUB;     // most keys per block
constexpr int ORD_NB_TARGET = 64;                   // blocks wanted before sub-tiles grow past 1
constexpr int ORD_BINS = 256;
constexpr int ORD_BOX_BLOCKS = 296;                 // grid of the bounding-box pass (2 per SM)
constexpr int ORD_SCAN_THREADS = 1024;              // the one-block scan, 4 entries per thread

__device__ __forceinline__ unsigned ord_key_bits(float f) {
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord_key_float(unsigned o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// Per-coordinate bounding box of the finite coordinates (order-preserving bits):
// box[j] = min, box[D_MAX + j] = max.  The grid strides over the row-major array with
// `per` = d * floor(256 / d) threads a block, so thread t always sees coordinate t % d and
// the loads are coalesced; a block folds its threads' extrema per coordinate, then one
// atomic per coordinate and block.
__global__ void __launch_bounds__(ORD_THREADS) ord_bbox_kernel(const float* X, int64_t n, int d, unsigned* box) {
    __shared__ unsigned slo[ORD_THREADS], shi[ORD_THREADS];
    const int per = ORD_THREADS / d * d;
    const int t = threadIdx.x;
    unsigned lo = 0xffffffffu, hi = 0u;
    if (t < per) {
        const int64_t total = n * d, stride = (int64_t)gridDim.x * per;
#pragma unroll 4
        for (int64_t e = (int64_t)blockIdx.x * per + t; e < total; e += stride) {
            const float v = X[e];
            if (isfinite(v)) {
                const unsigned k = ord_key_bits(v);
                lo = min(lo, k);
                hi = max(hi, k);
            }
        }
    }
    slo[t] = lo;
    shi[t] = hi;
    __syncthreads();
    if (t < d) {
        for (int s = t + d; s < per; s += d) {
            lo = min(lo, slo[s]);
            hi = max(hi, shi[s]);
        }
        atomicMin(&box[t], lo);
        atomicMax(&box[D_MAX + t], hi);
    }
}

// The Hilbert key of each point: the cell coordinates are turned into the "transposed"
// Hilbert index by J. Skilling's method (Programming the Hilbert curve, AIP Conf. Proc.
// 707, 2004: from the top bit down, each coordinate either inverts the low bits of the
// first or exchanges its low bits with it; then a Gray code across the coordinates), and
// the transposed bits are interleaved as a Morton key would be.  Consecutive cells of the
// Hilbert curve are always neighbours, so runs of the order have smaller boxes than
// Morton runs, which jump at every level boundary.  Block 0 also writes the box as
// floats, (0, 0) for a coordinate with no finite value.
__global__ void ord_key_kernel(const float* X, int64_t n, int d, const unsigned* box, unsigned* keys, int* idx,
                               float2* bounds) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (bounds && blockIdx.x == 0 && threadIdx.x < d) {
        const unsigned a = box[threadIdx.x], b = box[D_MAX + threadIdx.x];
        bounds[threadIdx.x] = a <= b ? make_float2(ord_key_float(a), ord_key_float(b)) : make_float2(0.f, 0.f);
    }
    if (i >= n) return;
    const int D = d < 16 ? d : 16;
    const int b = 16 / D;                          // bits per coordinate
    const int cells = 1 << b;
    // the loops over the coordinates are unrolled to 16 with a guard, so that cell[] stays
    // in registers (its indices are compile-time constants)
    int cell[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        int c = 0;
        if (j < D) {
            const float lo = ord_key_float(box[j]), hi = ord_key_float(box[D_MAX + j]);
            const float v = X[i * d + j];
            if (isfinite(v) && hi > lo) {
                const float u = (v - lo) / (hi - lo) * (float)cells;
                c = u >= (float)(cells - 1) ? cells - 1 : (u > 0.f ? (int)u : 0);
            }
        }
        cell[j] = c;
    }
    if (D > 1) {
        const int top = 1 << (b - 1);
        for (int q = top; q > 1; q >>= 1) {
            const int p = q - 1;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                if (j >= D) break;
                if (cell[j] & q) {
                    cell[0] ^= p;                               // invert the low bits
                } else {
                    const int t = (cell[0] ^ cell[j]) & p;      // exchange the low bits
                    cell[0] ^= t;
                    cell[j] ^= t;
                }
            }
        }
#pragma unroll
        for (int j = 1; j < 16; ++j)
            if (j < D) cell[j] ^= cell[j - 1];                 // Gray code
        int last = 0;
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (j == D - 1) last = cell[j];
        int t = 0;
        for (int q = top; q > 1; q >>= 1)
            if (last & q) t ^= q - 1;
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (j < D) cell[j] ^= t;
    }
    unsigned key = 0u;
    for (int l = b - 1; l >= 0; --l)
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (j < D) key = (key << 1) | (unsigned)((cell[j] >> l) & 1);
    keys[i] = key;
    idx[i] = (int)i;
}

// Digit counts per block of sub x 256 keys, stored digit-major: table[digit * nblocks +
// block].  Lanes with equal digits add once per warp (their leader adds the group's size).
__global__ void __launch_bounds__(ORD_THREADS) ord_hist_kernel(const unsigned* keys, int64_t n, int shift,
                                                              int* table, int nblocks, int sub) {
    __shared__ int cnt[ORD_BINS + 1];
    cnt[threadIdx.x] = 0;
    if (threadIdx.x == 0) cnt[ORD_BINS] = 0;
    __syncthreads();
    const int lane = threadIdx.x % 32;
    const int64_t base = (int64_t)blockIdx.x * sub * ORD_THREADS;
    for (int s = 0; s < sub; ++s) {
        const int64_t i = base + (int64_t)s * ORD_THREADS + threadIdx.x;
        const int digit = i < n ? (int)((keys[i] >> shift) & 0xffu) : ORD_BINS;
        const unsigned peers = __match_any_sync(0xffffffffu, digit);
        if (lane == __ffs(peers) - 1) atomicAdd(&cnt[digit], __popc(peers));
    }
    __syncthreads();
    table[(int64_t)threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// Exclusive prefix sums of the table in place (one block; total is a multiple of 4).  The
// block walks the table in chunks of 16384 entries: each thread loads 16 consecutive
// entries as four int4, the threads' sums are scanned by warp shuffles and then across the
// warps, and a running carry links the chunks.
constexpr int ORD_SCAN_PER = 16;                    // entries a thread takes per chunk
__global__ void __launch_bounds__(ORD_SCAN_THREADS) ord_scan_kernel(int* table, int64_t total) {
    __shared__ int wsum[ORD_SCAN_THREADS / 32];
    const int t = threadIdx.x, lane = t % 32, warp = t / 32;
    int carry = 0;
    for (int64_t c = 0; c < total; c += ORD_SCAN_PER * ORD_SCAN_THREADS) {
        const int64_t i = c + ORD_SCAN_PER * (int64_t)t;
        int4 v[ORD_SCAN_PER / 4];
        int own = 0;
#pragma unroll
        for (int k = 0; k < ORD_SCAN_PER / 4; ++k) {
            v[k] = make_int4(0, 0, 0, 0);
            if (i + 4 * k < total) v[k] = *reinterpret_cast<const int4*>(table + i + 4 * k);
            own += v[k].x + v[k].y + v[k].z + v[k].w;
        }
        int x = own;                               // inclusive scan over the warp
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int s = wsum[lane];                    // inclusive scan over the warps' totals
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            wsum[lane] = s;
        }
        __syncthreads();
        int run = carry + (warp > 0 ? wsum[warp - 1] : 0) + x - own;
#pragma unroll
        for (int k = 0; k < ORD_SCAN_PER / 4; ++k) {
            if (i + 4 * k < total) {
                int4 o;
                o.x = run;
                run += v[k].x;
                o.y = run;
                run += v[k].y;
                o.z = run;
                run += v[k].z;
                o.w = run;
                run += v[k].w;
                *reinterpret_cast<int4*>(table + i + 4 * k) = o;
            }
        }
        carry += wsum[ORD_SCAN_THREADS / 32 - 1];
        __syncthreads();                           // wsum is rewritten by the next chunk
    }
}

// Stable scatter, one sub-tile of 256 keys at a time in index order: position = running
// start of the digit in this block (from the scanned table, advanced by each sub-tile's
// counts) + count of the digit in earlier warps of the sub-tile + count among earlier lanes.
__global__ void __launch_bounds__(ORD_THREADS) ord_scatter_kernel(const unsigned* keys, const int* idx, int64_t n,
                                                                 int shift, const int* table, int nblocks, int sub,
                                                                 unsigned* keys_out, int* idx_out) {
    __shared__ int wc[ORD_WARPS][ORD_BINS + 1];    // column ORD_BINS: lanes past the end
    __shared__ int run[ORD_BINS];
    const int t = threadIdx.x, warp = t / 32, lane = t % 32;
    for (int k = t; k < ORD_WARPS * (ORD_BINS + 1); k += ORD_THREADS) (&wc[0][0])[k] = 0;
    run[t] = table[(int64_t)t * nblocks + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * sub * ORD_THREADS;
    for (int s = 0; s < sub; ++s) {
        const int64_t first = base + (int64_t)s * ORD_THREADS;
        if (first >= n) break;                     // uniform over the block
        __syncthreads();                           // wc cleared, run advanced
        const int64_t i = first + t;
        const bool valid = i < n;
        const unsigned key = valid ? keys[i] : 0u;
        const int digit = valid ? (int)((key >> shift) & 0xffu) : ORD_BINS;
        const unsigned peers = __match_any_sync(0xffffffffu, digit);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (rank == 0) wc[warp][digit] = __popc(peers);
        __syncthreads();
        int tot = 0;                               // digit t: exclusive prefix over the warps
        for (int w = 0; w < ORD_WARPS; ++w) {
            const int v = wc[w][t];
            wc[w][t] = tot;
            tot += v;
        }
        __syncthreads();
        if (valid) {
            const int64_t pos = (int64_t)run[digit] + wc[warp][digit] + rank;
            keys_out[pos] = key;
            idx_out[pos] = idx[i];
        }
        __syncthreads();                           // every read of run and wc is done
        for (int w = 0; w < ORD_WARPS; ++w) wc[w][t] = 0;
        run[t] += tot;
    }
}

size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

// 256-key sub-tiles per block: as few as keep about ORD_NB_TARGET blocks busy (more
// blocks, shorter serial loops), at most ORD_SUB (a bounded digit table to scan).
int ord_sub(int64_t n) {
    const int64_t s = (n + (int64_t)ORD_NB_TARGET * ORD_THREADS - 1) / ((int64_t)ORD_NB_TARGET * ORD_THREADS);
    return (int)(s < 1 ? 1 : (s > ORD_SUB ? ORD_SUB : s));
}

}  // namespace

size_t spatial_order_scratch(int64_t n) {
    const int64_t tile = (int64_t)ord_sub(n) * ORD_THREADS;
    const int64_t nb = (n + tile - 1) / tile;
    return al256(2 * D_MAX * sizeof(unsigned)) + 2 * al256((size_t)n * sizeof(unsigned)) +
           al256((size_t)n * sizeof(int)) + al256((size_t)nb * ORD_BINS * sizeof(int));
}

cudaError_t spatial_order(const float* X, int64_t n, int d, int* perm, float2* bounds, void* scratch,
                          cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (d < 1 || d > D_MAX) return cudaErrorInvalidValue;
    const int sub = ord_sub(n);
    const int nb = (int)((n + (int64_t)sub * ORD_THREADS - 1) / ((int64_t)sub * ORD_THREADS));
    char* s = static_cast<char*>(scratch);
    unsigned* box = reinterpret_cast<unsigned*>(s);
    unsigned* ka = reinterpret_cast<unsigned*>(s + al256(2 * D_MAX * sizeof(unsigned)));
    unsigned* kb = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(ka) + al256((size_t)n * sizeof(unsigned)));
    int* ia = reinterpret_cast<int*>(reinterpret_cast<char*>(kb) + al256((size_t)n * sizeof(unsigned)));
    int* table = reinterpret_cast<int*>(reinterpret_cast<char*>(ia) + al256((size_t)n * sizeof(int)));
    cudaError_t e = cudaMemsetAsync(box, 0xff, D_MAX * sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(box + D_MAX, 0, D_MAX * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    const int per = ORD_THREADS / d * d;
    const int64_t box_need = (n * d + per - 1) / per;
    const unsigned box_blocks = (unsigned)(box_need < ORD_BOX_BLOCKS ? box_need : ORD_BOX_BLOCKS);
    ord_bbox_kernel<<<box_blocks, ORD_THREADS, 0, st>>>(X, n, d, box);
    ord_key_kernel<<<(unsigned)((n + ORD_THREADS - 1) / ORD_THREADS), ORD_THREADS, 0, st>>>(X, n, d, box, ka, perm,
                                                                                          bounds);
    // pass 1: low byte (ka, perm) -> (kb, ia); pass 2: high byte (kb, ia) -> (ka, perm)
    const unsigned blocks = (unsigned)nb;
    const int64_t entries = (int64_t)nb * ORD_BINS;
    ord_hist_kernel<<<blocks, ORD_THREADS, 0, st>>>(ka, n, 0, table, nb, sub);
    ord_scan_kernel<<<1, ORD_SCAN_THREADS, 0, st>>>(table, entries);
    ord_scatter_kernel<<<blocks, ORD_THREADS, 0, st>>>(ka, perm, n, 0, table, nb, sub, kb, ia);
    ord_hist_kernel<<<blocks, ORD_THREADS, 0, st>>>(kb, n, 8, table, nb, sub);
    ord_scan_kernel<<<1, ORD_SCAN_THREADS, 0, st>>>(table, entries);
    ord_scatter_kernel<<<blocks, ORD_THREADS, 0, st>>>(kb, ia, n, 8, table, nb, sub, ka, perm);
    return cudaGetLastError();
}

int spatial_order_launches() { return 8; }

}  // namespace lip
