// The estimate's pair arithmetic (Sec. 5, M_est), shared by the full all-pairs kernel
// (estimate.cu) and the pruned one (estimate_pruned.cu): tile sizes, the squared ratio of
// a row point against a 4-point group, and the order of candidates.
#pragma once

#include "launch.h"

namespace lip {

constexpr int EST_THREADS = 128;
constexpr int EST_R = 4;
constexpr int EST_TILE = EST_THREADS * EST_R;        // points per I-tile and per J-tile
constexpr int EST_TILE_GROUPS = EST_TILE / GROUP;
constexpr int EST_NARROW_MAX = 16;                   // d above this takes estimate_wide_kernel

// Weights that are not powers of two are applied to the coordinate differences (WT):
// the difference of two nearby FP32 coordinates is exact, while a weight rounded into
// each coordinate beforehand would leave an error as large as the difference itself.
// Power-of-two weights scale the layout exactly and take the WT = false form.
template <int NORM, int D, bool WT>
__device__ __forceinline__ void est_group(const float2 (&xi)[D], float2 yi, const float4 (&x)[D + 1],
                                          const float2 (&wt)[D], float (&r2)[4]) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float2 t[D];
#pragma unroll
        for (int j = 0; j < D; ++j) {
            t[j] = sub2(xi[j], half_of(x[j], h));
            if constexpr (WT) t[j] = mul2(t[j], wt[j]);
        }
        float2 den;
        if constexpr (NORM == LIP_L2) {
            den = mul2(t[0], t[0]);
#pragma unroll
            for (int j = 1; j < D; ++j) den = fma2(t[j], t[j], den);
        } else if constexpr (NORM == LIP_L1) {
            float2 acc = make_float2(fabsf(t[0].x), fabsf(t[0].y));
#pragma unroll
            for (int j = 1; j < D; ++j) acc = make_float2(acc.x + fabsf(t[j].x), acc.y + fabsf(t[j].y));
            den = mul2(acc, acc);
        } else {
            float a[D], b[D];
#pragma unroll
            for (int j = 0; j < D; ++j) { a[j] = fabsf(t[j].x); b[j] = fabsf(t[j].y); }
            const float2 acc = make_float2(max_reduce<D>(a), max_reduce<D>(b));
            den = mul2(acc, acc);
        }
        const float2 dy = sub2(yi, half_of(x[D], h));
        const float2 num = mul2(dy, dy);
        const float2 q = mul2(num, make_float2(rcp_approx(den.x), rcp_approx(den.y)));
        r2[2 * h] = q.x;
        r2[2 * h + 1] = q.y;
    }
}

// (ratio, i, j) ordering: larger ratio first, then lower i, then lower j.
__device__ __forceinline__ bool est_better(float r, int i, int j, float rb, int ib, int jb) {
    if (ib < 0) return i >= 0;
    if (i < 0) return false;
    if (r != rb) return r > rb;
    if (i != ib) return i < ib;
    return j < jb;
}

}  // namespace lip
