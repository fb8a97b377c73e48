// Penalty smoothing (Sec. 4.4, Eq. (optim)): the objective
//
//   Phi(eps) = (1/p) ||eps||^2 + S1 + S2,
//   S1 = sum_{i != k} ((z_i - z_k - M dist_up(x^i, x^k))_+)^2          Eq. (const1)
//   S2 = sum_{i != k} ((z_k - z_i - M dist_lo(x^i, x^k))_+)^2          Eq. (const2)
//
// with z = y + eps, and its gradient, as one fused pass over the pairs (no N x N
// storage), driven by L-BFGS.  dist_lo(x^i, x^k) = dist_up(x^k, x^i), so Eq. (const2)'s
// term of (i, k) is Eq. (const1)'s term of (k, i): S2 = S1 and
//
//   Phi = ||eps||^2 / p + 2 S1,   dPhi/deps_j = 2 eps_j / p + 4 (R_j - C_j),
//   R_j = sum_k (z_j - z_k - M dist_up(x^j, x^k))_+,  C_j = sum_i (z_i - z_j - M dist_up(x^i, x^j))_+.
//
// The pass visits each unordered pair {i, k} once, from row i < k.  It forms v_ik (the
// const1 term) and v_ki (the term with i second), of which at most one is positive, adds
// q = (v_ik)_+ - (v_ki)_+ to R_i - C_i and q^2 to the row's share of S1 without atomics,
// and owes row k the term -q.  That column term is zero unless the pair violates the
// Lipschitz condition; it goes to a signed 64-bit fixed-point accumulator with integer
// atomics.  Integer sums do not depend on the order of the atomics, so results stay
// reproducible; the scale 2^(61 - e) with N (max z - min z) < 2^e keeps every column sum
// below 2^61 in magnitude.  Terms come four data points at a time: one warp vote per group
// decides whether the warp sums the group's column terms (a shuffle tree in a fixed order)
// for lane 0 to add, so the cost stays bounded when many pairs violate (line-search trial
// points).
// Pair terms are FP32 on the scaled layout (coordinates times M w, mirrored where
// decreasing, constrained first); each thread adds them in FP32 within a 128-point tile
// and in FP64 across tiles, and the splits are summed in FP64 in a fixed order.  FP64
// handles take an FP64 layout and FP64 pair terms (smooth_pass64_kernel below).
#include "launch.h"

namespace lip {

namespace {

constexpr int SM_THREADS = 128;
constexpr int SM_TILE = 128;
constexpr int RED_BLOCKS = 256;     // fixed reduction shape: results do not depend on timing

// Order-preserving unsigned bits of a float (larger float, larger bits).
__device__ __forceinline__ unsigned ord_bits(float f) {
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord_float(unsigned o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// Fixed-point scale of the column sums: 2^(61 - e) with N (max z - min z) < 2^e.
__device__ __forceinline__ double col_scale(const SmoothParams& P) {
    const double range = (double)ord_float(P.zbits[0]) + (double)ord_float(P.zbits[1]);
    const double bound = fmax((double)P.N * range, 0x1p-60);       // the scale stays below 2^121
    return ldexp(1.0, 61 - (ilogb(bound) + 1));
}

// The layout of z = y + eps; also zeroes the column sums and records the range of z.
__global__ void smooth_layout_kernel(const SmoothParams P, const double* eps) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P.npad) return;
    float* r = P.rec + k * (P.dp + 4);
    unsigned zmax = 0u, nzmax = 0u;
    if (k < P.N) {
        for (int j = 0; j < P.dp; ++j) {
            const int64_t i = k * P.d + P.perm[j];
            const double x = P.es == 8 ? static_cast<const double*>(P.X0)[i] : (double)static_cast<const float*>(P.X0)[i];
            r[j] = j < P.d ? (float)(P.scale[j] * x) : 0.f;
        }
        const double y = P.es == 8 ? static_cast<const double*>(P.y0)[k] : (double)static_cast<const float*>(P.y0)[k];
        const float z = (float)(y + eps[k]);
        r[P.dp] = z;
        zmax = ord_bits(z);
        nzmax = ord_bits(-z);
        P.colfix[k] = 0ull;
    } else {
        for (int j = 0; j < P.dp; ++j) r[j] = 0.f;
        r[P.dp] = __int_as_float(0x7fc00000);          // padding: NaN terms are never positive
    }
    r[P.dp + 1] = r[P.dp + 2] = r[P.dp + 3] = 0.f;
    const unsigned act = __activemask();
    zmax = __reduce_max_sync(act, zmax);
    nzmax = __reduce_max_sync(act, nzmax);
    if ((int)(threadIdx.x & 31) == __ffs(act) - 1) {
        atomicMax(&P.zbits[0], zmax);
        atomicMax(&P.zbits[1], nzmax);
    }
}

// Distances from the two rows (halves of x2) to data point xk: dist_up(x^i, x^k) in au
// and dist_up(x^k, x^i) in ar (the same for the symmetric distance).
template <int NORM, int DP, bool MONO>
__device__ __forceinline__ void smooth_dists(const float2 (&x2)[DP], const float* xk, int C, float2& au, float2& ar) {
    au = make_float2(0.f, 0.f);
    ar = au;
#pragma unroll
    for (int j = 0; j < DP; ++j) {
        const float2 t = sub2(x2[j], make_float2(xk[j], xk[j]));
        if (MONO && j < C) {
            const float2 u = make_float2(fmaxf(t.x, 0.f), fmaxf(t.y, 0.f));
            const float2 v = make_float2(fmaxf(-t.x, 0.f), fmaxf(-t.y, 0.f));
            if (NORM == LIP_L1) { au = add2(au, u); ar = add2(ar, v); }
            else if (NORM == LIP_L2) { au = fma2(u, u, au); ar = fma2(v, v, ar); }
            else {
                au = make_float2(fmaxf(au.x, u.x), fmaxf(au.y, u.y));
                ar = make_float2(fmaxf(ar.x, v.x), fmaxf(ar.y, v.y));
            }
        } else {
            if (NORM == LIP_L1) au = make_float2(au.x + fabsf(t.x), au.y + fabsf(t.y));
            else if (NORM == LIP_L2) au = fma2(t, t, au);
            else au = make_float2(fmaxf(au.x, fabsf(t.x)), fmaxf(au.y, fabsf(t.y)));
            if (MONO) {
                if (NORM == LIP_L1) ar = make_float2(ar.x + fabsf(t.x), ar.y + fabsf(t.y));
                else if (NORM == LIP_L2) ar = fma2(t, t, ar);
                else ar = make_float2(fmaxf(ar.x, fabsf(t.x)), fmaxf(ar.y, fabsf(t.y)));
            }
        }
    }
    if (NORM == LIP_L2) {
        au = make_float2(sqrt_approx(au.x), sqrt_approx(au.y));
        if (MONO) ar = make_float2(sqrt_approx(ar.x), sqrt_approx(ar.y));
    }
    if (!MONO) ar = au;
}

// The pair (i, k)'s share of the gradient for both rows: q = (v_ik)_+ - (v_ki)_+, with
// v_ik = z_i - z_k - M dist_up(x^i, x^k) (Eq. (const1)) and v_ki = z_k - z_i - M
// dist_up(x^k, x^i).  v_ik + v_ki = -M (dist_up(x^i, x^k) + dist_up(x^k, x^i)) <= 0, so at
// most one is positive: q = max(v_ik, 0) + min(-v_ki, 0), and q^2 is the pair's share of
// S1 (both orders).  Row i gains R_i - C_i += q and row k gains R_k - C_k -= q.  top
// tracks the largest of v_ik and v_ki (a positive one means a column term is owed).
// NaN (padding, absent rows) gives q = 0 and leaves top alone.
template <bool MASK>
__device__ __forceinline__ float2 smooth_q(float2 z2, float zk, float2 au, float2 ar, bool ma, bool mb, float& top) {
    const float2 dz = sub2(z2, make_float2(zk, zk));
    float2 v1 = sub2(dz, au);                     // v_ik
    float2 w2 = add2(dz, ar);                     // -v_ki
    if (MASK && ma) { v1.x = -INFINITY; w2.x = INFINITY; }
    if (MASK && mb) { v1.y = -INFINITY; w2.y = INFINITY; }
    top = max3f(top, max3f(v1.x, v1.y, -w2.x), -w2.y);
    return add2(make_float2(fmaxf(v1.x, 0.f), fmaxf(v1.y, 0.f)), make_float2(fminf(w2.x, 0.f), fminf(w2.y, 0.f)));
}

// Each thread owns two rows (i and i + 128 of its block's 256), packed into the halves of
// float2 registers, so the distance, the pair's share q and the two sums are f32x2
// operations.  A row takes the data k > i of its split; on the two tiles that hold the
// block's own rows the pairs with k <= i are masked.
template <int NORM, int DP, bool MONO>
__global__ void __launch_bounds__(SM_THREADS) smooth_pass_kernel(const SmoothParams P) {
    constexpr int PR = DP + 4;
    __shared__ float4 tile4[SM_TILE * PR / 4];
    const float* tile = reinterpret_cast<const float*>(tile4);
    const int tid = threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.x * SM_THREADS * 2;
    const int64_t ia = i0 + tid, ib = ia + SM_THREADS;
    const int split = blockIdx.y;
    const bool va = ia < P.N, vb = ib < P.N;
    float2 x2[DP];
#pragma unroll
    for (int j = 0; j < DP; ++j)
        x2[j] = make_float2(va ? P.rec[ia * PR + j] : 0.f, vb ? P.rec[ib * PR + j] : 0.f);
    // an absent row's z is NaN: its q is 0
    const float nan = __int_as_float(0x7fc00000);
    const float2 z2 = make_float2(va ? P.rec[ia * PR + DP] : nan, vb ? P.rec[ib * PR + DP] : nan);
    const float fscale = (float)col_scale(P);                        // a power of 2
    double Da = 0.0, Sa = 0.0, Db = 0.0, Sb = 0.0;
    const int64_t split_begin = (int64_t)split * P.points_per_split;
    const int64_t k_begin = split_begin > i0 ? split_begin : i0;     // i0 is a multiple of the tile
    const int64_t k_end = split_begin + P.points_per_split < P.npad ? split_begin + P.points_per_split : P.npad;
    for (int64_t k0 = k_begin; k0 < k_end; k0 += SM_TILE) {
        __syncthreads();
        const float4* src = reinterpret_cast<const float4*>(P.rec + k0 * PR);
        for (int t = tid; t < SM_TILE * PR / 4; t += SM_THREADS) tile4[t] = src[t];
        __syncthreads();
        const bool diag = k0 < i0 + 2 * SM_THREADS;                     // holds some k <= i
        float2 dsum = make_float2(0.f, 0.f), ssum = dsum;
        for (int kg = 0; kg < SM_TILE; kg += 4) {
            float2 q[4];
            float top = -INFINITY;
            if (!diag) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float* xk = tile + (kg + u) * PR;
                    float2 au, ar;
                    smooth_dists<NORM, DP, MONO>(x2, xk, P.C, au, ar);
                    q[u] = smooth_q<false>(z2, xk[DP], au, ar, false, false, top);
                }
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float* xk = tile + (kg + u) * PR;
                    float2 au, ar;
                    smooth_dists<NORM, DP, MONO>(x2, xk, P.C, au, ar);
                    const int64_t kk = k0 + kg + u;
                    q[u] = smooth_q<true>(z2, xk[DP], au, ar, kk <= ia, kk <= ib, top);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                dsum = add2(dsum, q[u]);
                ssum = fma2(q[u], q[u], ssum);
            }
            if (__any_sync(0xffffffffu, top > 0.f)) {
                // row k is owed R_k - C_k -= q: summed over the warp's 64 rows in a fixed
                // shuffle order, then added in signed fixed point by lane 0
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    float cs = q[u].x + q[u].y;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) cs += __shfl_xor_sync(0xffffffffu, cs, o);
                    const int64_t kk = k0 + kg + u;
                    if ((tid & 31) == 0 && kk < P.N && cs != 0.f)
                        atomicAdd(&P.colfix[kk], (unsigned long long)__float2ll_rn(-cs * fscale));
                }
            }
        }
        Da += (double)dsum.x; Sa += (double)ssum.x;
        Db += (double)dsum.y; Sb += (double)ssum.y;
    }
    if (va) {
        double* out = P.partial + ((int64_t)split * P.N + ia) * 2;
        out[0] = Da; out[1] = Sa;
    }
    if (vb) {
        double* out = P.partial + ((int64_t)split * P.N + ib) * 2;
        out[0] = Db; out[1] = Sb;
    }
}

// ------------------------------------------------------------ FP64 handles
// The same objective with every pair term in FP64: the layout holds the scaled
// coordinates and z in double, each thread owns one row, and the row and column sums are
// formed exactly as above (the column terms in the same signed fixed point; its scale
// comes from the range of z rounded outwards to FP32).

__global__ void smooth_layout64_kernel(const SmoothParams P, const double* eps) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P.npad) return;
    double* r = P.rec64 + k * (P.dp + 2);
    unsigned zmax = 0u, nzmax = 0u;
    if (k < P.N) {
        const double* X = static_cast<const double*>(P.X0);
        for (int j = 0; j < P.dp; ++j) r[j] = j < P.d ? P.scale[j] * X[k * P.d + P.perm[j]] : 0.0;
        const double z = static_cast<const double*>(P.y0)[k] + eps[k];
        r[P.dp] = z;
        zmax = ord_bits(__double2float_ru(z));
        nzmax = ord_bits(__double2float_ru(-z));
        P.colfix[k] = 0ull;
    } else {
        for (int j = 0; j < P.dp; ++j) r[j] = 0.0;
        r[P.dp] = __longlong_as_double(0x7ff8000000000000ll);   // padding: NaN terms are never positive
    }
    r[P.dp + 1] = 0.0;
    const unsigned act = __activemask();
    zmax = __reduce_max_sync(act, zmax);
    nzmax = __reduce_max_sync(act, nzmax);
    if ((int)(threadIdx.x & 31) == __ffs(act) - 1) {
        atomicMax(&P.zbits[0], zmax);
        atomicMax(&P.zbits[1], nzmax);
    }
}

// dist_up(x^i, x^k) in au and dist_up(x^k, x^i) in ar, in FP64.
template <int NORM, int DP, bool MONO>
__device__ __forceinline__ void smooth_dists64(const double (&xi)[DP], const double* xk, int C, double& au,
                                               double& ar) {
    au = 0.0;
    ar = 0.0;
#pragma unroll
    for (int j = 0; j < DP; ++j) {
        const double t = xi[j] - xk[j];
        if (MONO && j < C) {
            const double u = fmax(t, 0.0), v = fmax(-t, 0.0);
            if (NORM == LIP_L1) { au += u; ar += v; }
            else if (NORM == LIP_L2) { au = fma(u, u, au); ar = fma(v, v, ar); }
            else { au = fmax(au, u); ar = fmax(ar, v); }
        } else {
            const double a = fabs(t);
            if (NORM == LIP_L1) au += a;
            else if (NORM == LIP_L2) au = fma(t, t, au);
            else au = fmax(au, a);
            if (MONO) {
                if (NORM == LIP_L1) ar += a;
                else if (NORM == LIP_L2) ar = fma(t, t, ar);
                else ar = fmax(ar, a);
            }
        }
    }
    if (NORM == LIP_L2) {
        au = sqrt(au);
        if (MONO) ar = sqrt(ar);
    }
    if (!MONO) ar = au;
}

// One row per thread: q = (v_ik)_+ - (v_ki)_+ for the data k > i of the split, summed into
// R_i - C_i and S1 in FP64; the column terms -q as in smooth_pass_kernel.
template <int NORM, int DP, bool MONO>
__global__ void __launch_bounds__(SM_THREADS) smooth_pass64_kernel(const SmoothParams P) {
    constexpr int PR = DP + 2;
    __shared__ double tile[SM_TILE * PR];
    const int tid = threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.x * SM_THREADS;
    const int64_t ia = i0 + tid;
    const int split = blockIdx.y;
    const bool va = ia < P.N;
    double xi[DP];
#pragma unroll
    for (int j = 0; j < DP; ++j) xi[j] = va ? P.rec64[ia * PR + j] : 0.0;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    const double z = va ? P.rec64[ia * PR + DP] : nan;           // an absent row's q is 0
    const double fscale = col_scale(P);
    double Da = 0.0, Sa = 0.0;
    const int64_t split_begin = (int64_t)split * P.points_per_split;
    const int64_t k_begin = split_begin > i0 ? split_begin : i0;     // i0 is a multiple of the tile
    const int64_t k_end = split_begin + P.points_per_split < P.npad ? split_begin + P.points_per_split : P.npad;
    for (int64_t k0 = k_begin; k0 < k_end; k0 += SM_TILE) {
        __syncthreads();
        for (int t = tid; t < SM_TILE * PR; t += SM_THREADS) tile[t] = P.rec64[k0 * PR + t];
        __syncthreads();
        const bool diag = k0 < i0 + SM_THREADS;                          // holds some k <= i
        for (int kg = 0; kg < SM_TILE; kg += 4) {
            double q[4];
            double top = -INFINITY;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const double* xk = tile + (kg + u) * PR;
                double au, ar;
                smooth_dists64<NORM, DP, MONO>(xi, xk, P.C, au, ar);
                const double dz = z - xk[DP];
                double v1 = dz - au;                  // v_ik
                double w2 = dz + ar;                  // -v_ki
                if (diag && k0 + kg + u <= ia) { v1 = -INFINITY; w2 = INFINITY; }
                top = fmax(top, fmax(v1, -w2));
                q[u] = fmax(v1, 0.0) + fmin(w2, 0.0);
                Da += q[u];
                Sa = fma(q[u], q[u], Sa);
            }
            if (__any_sync(0xffffffffu, top > 0.0)) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    double cs = q[u];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) cs += __shfl_xor_sync(0xffffffffu, cs, o);
                    const int64_t kk = k0 + kg + u;
                    if ((tid & 31) == 0 && kk < P.N && cs != 0.0)
                        atomicAdd(&P.colfix[kk], (unsigned long long)__double2ll_rn(-cs * fscale));
                }
            }
        }
    }
    if (va) {
        double* out = P.partial + ((int64_t)split * P.N + ia) * 2;
        out[0] = Da;
        out[1] = Sa;
    }
}

// grad_i = 2 eps_i / p + 4 (R_i - C_i); per-block sums of S_i and eps_i^2.
__global__ void __launch_bounds__(256) smooth_finish_kernel(const SmoothParams P, const double* eps, double* grad,
                                                            double* block_sums) {
    __shared__ double red[2][256];
    const double cscale = col_scale(P);
    double sS = 0.0, sE = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.N; i += (int64_t)gridDim.x * blockDim.x) {
        double D = 0.0, S = 0.0;                     // D = R_i - C_i
        for (int s = 0; s < P.nsplit; ++s) {
            const double* v = P.partial + ((int64_t)s * P.N + i) * 2;
            D += v[0];
            S += v[1];
        }
        D += (double)(long long)P.colfix[i] / cscale;
        if (grad) grad[i] = 2.0 * eps[i] / P.p + 4.0 * D;
        sS += S;
        sE += eps[i] * eps[i];
    }
    red[0][threadIdx.x] = sS;
    red[1][threadIdx.x] = sE;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            red[0][threadIdx.x] += red[0][threadIdx.x + w];
            red[1][threadIdx.x] += red[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        block_sums[2 * blockIdx.x] = red[0][0];
        block_sums[2 * blockIdx.x + 1] = red[1][0];
    }
}

// Phi = sum eps^2 / p + 2 S1 from the block sums, in a fixed order.
__global__ void smooth_total_kernel(const double* block_sums, int nblocks, double p, double* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double S = 0.0, E = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        S += block_sums[2 * b];
        E += block_sums[2 * b + 1];
    }
    out[0] = E / p + 2.0 * S;
    out[1] = S;
}

// ------------------------------------------------------------ vector kernels (L-BFGS)

// Fixed-shape two-level reductions: per-block sums of a*b (op 0) or maxima of |a| (op 1),
// then one block over the RED_BLOCKS partials.
__global__ void __launch_bounds__(256) vec_reduce_kernel(const double* a, const double* b, int64_t n, int op,
                                                         double* partial) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc = op == 0 ? acc + a[i] * b[i] : fmax(acc, fabs(a[i]));
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = op == 0 ? red[threadIdx.x] + red[threadIdx.x + w]
                                                        : fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(256) vec_reduce_final_kernel(const double* partial, int nb, int op, double* out) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc = op == 0 ? acc + partial[i] : fmax(acc, partial[i]);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = op == 0 ? red[threadIdx.x] + red[threadIdx.x + w]
                                                        : fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// out = a + alpha * b (out may alias a or b)
__global__ void vec_axpy_kernel(double* out, const double* a, double alpha, const double* b, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i] + alpha * b[i];
}

__global__ void vec_scale_kernel(double* out, const double* a, double alpha, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = alpha * a[i];
}

// y0 <- y0 + eps (the smoothed values, in the handle's storage type)
__global__ void apply_eps_kernel(void* y0, int es, const double* eps, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (es == 8) static_cast<double*>(y0)[i] += eps[i];
    else static_cast<float*>(y0)[i] = (float)((double)static_cast<float*>(y0)[i] + eps[i]);
}

template <int NORM, int DP>
void pass_shape(const SmoothParams& P, dim3 grid, cudaStream_t st) {
    if (P.C > 0) smooth_pass_kernel<NORM, DP, true><<<grid, SM_THREADS, 0, st>>>(P);
    else smooth_pass_kernel<NORM, DP, false><<<grid, SM_THREADS, 0, st>>>(P);
}

template <int NORM, int DP>
void pass64_shape(const SmoothParams& P, dim3 grid, cudaStream_t st) {
    if (P.C > 0) smooth_pass64_kernel<NORM, DP, true><<<grid, SM_THREADS, 0, st>>>(P);
    else smooth_pass64_kernel<NORM, DP, false><<<grid, SM_THREADS, 0, st>>>(P);
}

template <int NORM>
void pass64_norm(const SmoothParams& P, dim3 grid, cudaStream_t st) {
    switch (P.dp) {
        case 4: pass64_shape<NORM, 4>(P, grid, st); break;
        case 8: pass64_shape<NORM, 8>(P, grid, st); break;
        case 12: pass64_shape<NORM, 12>(P, grid, st); break;
        case 16: pass64_shape<NORM, 16>(P, grid, st); break;
        default: pass64_shape<NORM, 32>(P, grid, st); break;
    }
}

template <int NORM>
void pass_norm(const SmoothParams& P, dim3 grid, cudaStream_t st) {
    if (P.es == 8) {
        pass64_norm<NORM>(P, grid, st);
        return;
    }
    switch (P.dp) {
        case 4: pass_shape<NORM, 4>(P, grid, st); break;
        case 8: pass_shape<NORM, 8>(P, grid, st); break;
        case 12: pass_shape<NORM, 12>(P, grid, st); break;
        case 16: pass_shape<NORM, 16>(P, grid, st); break;
        default: pass_shape<NORM, 32>(P, grid, st); break;
    }
}

}  // namespace

int smooth_tile() { return SM_TILE; }
int smooth_rows_per_block(int es) { return es == 8 ? SM_THREADS : SM_THREADS * 2; }
int smooth_reduce_blocks() { return RED_BLOCKS; }

// Phi and its gradient at eps: layout, the pair pass, the finishing sums.  out[0] = Phi,
// out[1] = S1 (device); grad may be NULL.  block_sums holds 2 * RED_BLOCKS doubles.
cudaError_t launch_smooth_objective(const SmoothParams& P, const double* eps, double* grad, double* block_sums,
                                    double* out, int gx, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(P.zbits, 0, 2 * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    if (P.es == 8) smooth_layout64_kernel<<<(unsigned)((P.npad + 255) / 256), 256, 0, st>>>(P, eps);
    else smooth_layout_kernel<<<(unsigned)((P.npad + 255) / 256), 256, 0, st>>>(P, eps);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)gx, (unsigned)P.nsplit);
    if (P.norm == LIP_L1) pass_norm<LIP_L1>(P, grid, st);
    else if (P.norm == LIP_L2) pass_norm<LIP_L2>(P, grid, st);
    else pass_norm<LIP_LINF>(P, grid, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    smooth_finish_kernel<<<RED_BLOCKS, 256, 0, st>>>(P, eps, grad, block_sums);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    smooth_total_kernel<<<1, 32, 0, st>>>(block_sums, RED_BLOCKS, P.p, out);
    return cudaGetLastError();
}

cudaError_t launch_vec_reduce(const double* a, const double* b, int64_t n, int op, double* partial, double* out,
                              cudaStream_t st) {
    vec_reduce_kernel<<<RED_BLOCKS, 256, 0, st>>>(a, b, n, op, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    vec_reduce_final_kernel<<<1, 256, 0, st>>>(partial, RED_BLOCKS, op, out);
    return cudaGetLastError();
}

cudaError_t launch_vec_axpy(double* out, const double* a, double alpha, const double* b, int64_t n, cudaStream_t st) {
    vec_axpy_kernel<<<RED_BLOCKS, 256, 0, st>>>(out, a, alpha, b, n);
    return cudaGetLastError();
}

cudaError_t launch_vec_scale(double* out, const double* a, double alpha, int64_t n, cudaStream_t st) {
    vec_scale_kernel<<<RED_BLOCKS, 256, 0, st>>>(out, a, alpha, n);
    return cudaGetLastError();
}

cudaError_t launch_apply_eps(void* y0, int es, const double* eps, int64_t n, cudaStream_t st) {
    apply_eps_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(y0, es, eps, n);
    return cudaGetLastError();
}

}  // namespace lip
