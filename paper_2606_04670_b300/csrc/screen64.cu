// Exact FP64 envelopes for FP64 handles (LIP_FP64) at the FP32 rate.
//
// B300 runs FP64 at a small fraction of its FP32 rate, so an FP64 handle does not scan in
// FP64.  It keeps a float copy of its layout (the FP32 handles' layout) and:
//   1. scans it with the FP32 kernels, giving per query an approximate minimum b_up and
//      maximum b_lo;
//   2. scans it again in FP32 and recomputes in FP64, from the caller's data, only the pairs
//      whose FP32 value can still reach the exact extremum: v32 <= b_up + 2 delta (and
//      v32 >= b_lo - 2 delta);
//   3. merges the splits as usual (lowest index on ties) and writes the FP64 values.
// Every FP32 value here is within delta of the FP64 value of the same pair, with
//   delta = 2^-21 (d + 4)^2 (Qm + R) + 2^-20 (d + 2) Y,
// R the largest |M w x_i| of the data, Qm that of the query, Y the largest |y|: each scaled
// coordinate is rounded once or twice to float (2^-24 of its magnitude), the differences,
// the d-term sum or maximum, the square root (sqrt.approx) and the final addition each add
// a few ulps of at most d (Qm + R) or Y, and the L1 kernels' auxiliary channel adds C
// roundings of y - sum x; the factor covers all of them at least twice.  So the exact
// extremum's pair passes the test (its FP32 value is within delta of the exact extremum,
// and b_up is within delta of a value at least as large), and the result is the FP64 one.
#include "launch.h"

namespace lip {

namespace {

constexpr int S64_THREADS = 128;

// The FP32 layout of an FP64 handle (the format of build_hot_kernel<float>), from the
// caller's double data; also the largest |scaled coordinate| and |y| (float bits).
__global__ void build_hot32_kernel(const HotParams P, unsigned* maxbits) {
    const int64_t k = P.k0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P.k1) return;
    const double* x = static_cast<const double*>(P.X0) + k * P.d;
    const double yv = static_cast<const double*>(P.y0)[k];
    float* hot = static_cast<float*>(P.hot);
    const int64_t base = (k / GROUP) * (int64_t)P.nch * GROUP + (k % GROUP);
    float sx = 0.f, amax = 0.f;
    for (int j = 0; j < P.dl; ++j) {
        float v = 0.f;
        if (j < P.d) v = (float)(P.scale[j] * x[P.perm[j]]);
        hot[base + (int64_t)j * GROUP] = v;
        if (j < P.C) sx = sx + v;
        amax = fmaxf(amax, fabsf(v));
    }
    const float y32 = (float)yv;
    hot[base + (int64_t)P.dl * GROUP] = y32;
    if (P.aux) hot[base + (int64_t)(P.dl + 1) * GROUP] = y32 - sx;
    atomicMax(&maxbits[0], __float_as_uint(amax));
    atomicMax(&maxbits[1], __float_as_uint(fabsf(y32)));
}

__global__ void to_float_kernel(const double* a, int64_t n, float* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)a[i];
}

template <int NORM, int DP>
__global__ void __launch_bounds__(S64_THREADS) screen64_kernel(const Screen64Params P) {
    const int64_t qi = (int64_t)blockIdx.x * S64_THREADS + threadIdx.x;
    const int split = blockIdx.y;
    if (qi >= P.nq) return;
    const double* q64 = P.Q + qi * P.M.d;
    float q[DP];
    float qm = 0.f;
#pragma unroll
    for (int j = 0; j < DP; ++j) {
        q[j] = j < P.M.d ? (float)(P.scale[j] * q64[P.perm[j]]) : 0.f;
        qm = fmaxf(qm, fabsf(q[j]));
    }
    // the FP32 pass's extrema over its splits
    float b_up = INFINITY, b_lo = -INFINITY;
    bool any = false;
    for (int s = 0; s < P.nsplit1; ++s) {
        const PartialRec<float> r = P.partial1[(int64_t)s * P.nq + qi];
        if (r.iu >= 0) { b_up = fminf(b_up, r.vu); any = true; }
        if (r.il >= 0) b_lo = fmaxf(b_lo, r.vl);
    }
    const float R = __uint_as_float(P.maxbits[0]), Y = __uint_as_float(P.maxbits[1]);
    const float dd = (float)(P.M.d + 4);
    const float delta = ldexpf(dd * dd * (qm + R), -21) + ldexpf((float)(P.M.d + 2) * Y, -20);
    const float Uu = any ? b_up + 2.f * delta : -INFINITY;   // no candidate without an FP32 result
    const float Ul = any ? b_lo - 2.f * delta : INFINITY;
    double bu = INFINITY, bl = -INFINITY;
    int iu = -1, il = -1;
    const float4* hot = reinterpret_cast<const float4*>(P.hot32);
    const double* X0 = static_cast<const double*>(P.M.X0);
    const double* y0 = static_cast<const double*>(P.M.y0);
    const int64_t g0 = (int64_t)split * P.groups_per_split;
    const int64_t g1 = g0 + P.groups_per_split < P.ngroups ? g0 + P.groups_per_split : P.ngroups;
    for (int64_t g = g0; g < g1; ++g) {
        float x[DP][4];
#pragma unroll
        for (int j = 0; j < DP; ++j) {
            const float4 v = j < P.dl ? hot[g * P.nch + j] : make_float4(0.f, 0.f, 0.f, 0.f);
            x[j][0] = v.x; x[j][1] = v.y; x[j][2] = v.z; x[j][3] = v.w;
        }
        const float4 yv = hot[g * P.nch + P.dl];
        const float yy[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float au = 0.f, al = 0.f;
#pragma unroll
            for (int j = 0; j < DP; ++j) {
                const float t = q[j] - x[j][e];
                float u, l;
                if (j < P.C) { u = fmaxf(t, 0.f); l = fmaxf(-t, 0.f); }
                else { u = fabsf(t); l = u; }
                if (NORM == LIP_L1) { au += u; al += l; }
                else if (NORM == LIP_L2) { au = fmaf(u, u, au); al = fmaf(l, l, al); }
                else { au = fmaxf(au, u); al = fmaxf(al, l); }
            }
            if (NORM == LIP_L2) { au = sqrt_approx(au); al = sqrt_approx(al); }
            const float vu = yy[e] + au, vl = yy[e] - al;      // NaN (padding) fails both tests
            const int k = (int)(g * GROUP + e);
            if (vu <= Uu) {
                const double v = y0[k] + P.M.M * dist_fp64<double>(P.M, q64, X0 + (int64_t)k * P.M.d, +1);
                if (v < bu) { bu = v; iu = k; }
            }
            if (vl >= Ul) {
                const double v = y0[k] - P.M.M * dist_fp64<double>(P.M, q64, X0 + (int64_t)k * P.M.d, -1);
                if (v > bl) { bl = v; il = k; }
            }
        }
    }
    PartialRec<double> r;
    r.vu = bu; r.vl = bl; r.iu = iu; r.il = il; r.pad0 = 0; r.pad1 = 0;
    P.partial2[(int64_t)split * P.nq + qi] = r;
}

template <int NORM>
static void screen_norm(const Screen64Params& P, dim3 grid, cudaStream_t st) {
    if (P.dl <= 4) screen64_kernel<NORM, 4><<<grid, S64_THREADS, 0, st>>>(P);
    else if (P.dl <= 8) screen64_kernel<NORM, 8><<<grid, S64_THREADS, 0, st>>>(P);
    else if (P.dl <= 12) screen64_kernel<NORM, 12><<<grid, S64_THREADS, 0, st>>>(P);
    else if (P.dl <= 16) screen64_kernel<NORM, 16><<<grid, S64_THREADS, 0, st>>>(P);
    else if (P.dl <= 24) screen64_kernel<NORM, 24><<<grid, S64_THREADS, 0, st>>>(P);
    else screen64_kernel<NORM, 32><<<grid, S64_THREADS, 0, st>>>(P);
}

}  // namespace

int screen64_threads() { return S64_THREADS; }

cudaError_t launch_build_hot32(const HotParams& P, unsigned* maxbits, cudaStream_t st) {
    const int64_t n = P.k1 - P.k0;
    if (n <= 0) return cudaSuccess;
    build_hot32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(P, maxbits);
    return cudaGetLastError();
}

cudaError_t launch_to_float(const double* a, int64_t n, float* out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    to_float_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, n, out);
    return cudaGetLastError();
}

cudaError_t launch_screen64(int norm, const Screen64Params& P, int gx, int gy, cudaStream_t st) {
    if (gy <= 0) return cudaSuccess;
    const dim3 grid((unsigned)gx, (unsigned)gy);
    if (norm == LIP_L1) screen_norm<LIP_L1>(P, grid, st);
    else if (norm == LIP_L2) screen_norm<LIP_L2>(P, grid, st);
    else screen_norm<LIP_LINF>(P, grid, st);
    return cudaGetLastError();
}

}  // namespace lip
