// Gradient of L = sum_q gbar_q g(q) through the saved argmin u_q / argmax l_q
// (g = (H_up + H_lo)/2, Sec. 3 Eq. (eq:g); piecewise smooth, differentiable almost
// everywhere, Table 1):
//   dL/dq_i   = gbar M/2 ( d dist_up(q, x^u)/dq_i - d dist_lo(q, x^l)/dq_i )
//   dL/dy^k   = 1/2 sum_q gbar_q ([u_q = k] + [l_q = k])
//   dL/dM     = 1/2 sum_q gbar_q ( dist_up(q, x^u) - dist_lo(q, x^l) )
// One thread per query, in the caller's coordinates, arithmetic in the handle's
// element type, all in one launch: dL/dy is added straight into the caller's grad_y with
// atomics of the element type (or, in the deterministic mode, summed as 64-bit fixed point
// scaled by a power of two from max |grad_g|, whose integer atomics give the same bits in
// any order, then added in a second pass), and dL/dM is a fixed-shape two-level FP64 reduction
// finished by the last block to arrive (bitwise reproducible); the per-query terms and the
// warp sums are in the element type, the block and grid sums in FP64.
#include <algorithm>

#include "launch.h"

namespace lip {

constexpr int BWD_THREADS = 256;

// Magnitude v and dv/dt' of one coordinate of the upper (side > 0) or lower (side < 0)
// distance vector, t' = sign_i w_i (q_i - x_i).
template <typename T>
__device__ __forceinline__ void coord_part(T t, bool constrained, int side, T& v, T& dv) {
    if (constrained) {
        if (side > 0) { v = t > 0 ? t : (T)0; dv = t > 0 ? (T)1 : (T)0; }
        else { v = t < 0 ? -t : (T)0; dv = t < 0 ? (T)-1 : (T)0; }
    } else {
        v = t < 0 ? -t : t;
        dv = t > 0 ? (T)1 : (t < 0 ? (T)-1 : (T)0);
    }
}


// 2^e with the largest sum of contributions, nq * max|grad_g| / 2 per datum, below 2^60.
__device__ __forceinline__ double fix_scale(const unsigned* maxbits, int64_t nq) {
    const double bound = 0.5 * (double)__uint_as_float(*maxbits) * (double)(nq > 0 ? nq : 1);
    int e;
    frexp(bound > 0.0 ? bound : 1.0, &e);            // bound < 2^e
    return ldexp(1.0, 60 - e);
}

template <typename T>
__global__ void __launch_bounds__(256) grad_max_kernel(const T* gb, int64_t n, unsigned* maxbits) {
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf((float)gb[i]) * (1.f + 1e-6f));   // float rounding of a double grad_g
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(maxbits, __float_as_uint(m));   // |.| orders as its bits
}

template <typename T>
__global__ void grad_y_fix_kernel(const unsigned long long* fix, const unsigned* maxbits, int64_t nq, int64_t N,
                                  T* grad_y) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const double v = (double)(long long)fix[k] / fix_scale(maxbits, nq);
    grad_y[k] = (T)((double)grad_y[k] + v);
}

// DM: register arrays for up to DM coordinates (16, or 32 for the widest handles)
template <typename T, int DM>
__global__ void __launch_bounds__(BWD_THREADS) backward_kernel(const BwdParams P) {
    const int64_t qi = (int64_t)blockIdx.x * BWD_THREADS + threadIdx.x;
    T gm = 0;
    if (qi < P.nq) {
        const T* q = static_cast<const T*>(P.Q) + qi * P.d;
        const T gb = static_cast<const T*>(P.gbar)[qi];
        const int u = P.iu[qi], l = P.il[qi];
        T* gq = P.grad_Q ? static_cast<T*>(P.grad_Q) + qi * P.d : nullptr;
        if (u < 0 || l < 0) {
            if (gq) for (int i = 0; i < P.d; ++i) gq[i] = 0;
        } else {
            const T* X0 = static_cast<const T*>(P.X0);
            const T* xu = X0 + (int64_t)u * P.d;
            const T* xl = X0 + (int64_t)l * P.d;
            // the query and both data rows once, in registers, with dt'/dq_i = sign_i w_i
            T qv[DM], tu[DM], tl[DM], sq[DM];
#pragma unroll
            for (int i = 0; i < DM; ++i) {
                if (i < P.d) {
                    sq[i] = sizeof(T) == 4 ? (T)P.sqf[i] : (P.mon[i] < 0 ? (T)-1 : (T)1) * (T)P.w[i];
                    qv[i] = q[i];
                    tu[i] = (qv[i] - xu[i]) * sq[i];
                    tl[i] = (qv[i] - xl[i]) * sq[i];
                }
            }
            // pass 1: the two distances (and the Linf arg-max coordinates, lowest on ties)
            T au = 0, al = 0;
            int mu = -1, ml = -1;
#pragma unroll
            for (int i = 0; i < DM; ++i) {
                if (i >= P.d) break;
                T vu, vl, dv;
                const bool c = P.mon[i] != 0;
                coord_part<T>(tu[i], c, +1, vu, dv);
                coord_part<T>(tl[i], c, -1, vl, dv);
                if (P.norm == LIP_L1) { au += vu; al += vl; }
                else if (P.norm == LIP_L2) { au += vu * vu; al += vl * vl; }
                else {
                    if (vu > au) { au = vu; mu = i; }
                    if (vl > al) { al = vl; ml = i; }
                }
            }
            const T du = P.norm == LIP_L2 ? sqrt(au) : au;
            const T dl = P.norm == LIP_L2 ? sqrt(al) : al;
            // pass 2: d dist / d q_i for both sides, then dL/dq_i
            if (gq) {
                const T hm = (T)(0.5 * P.M) * gb;
                const T ru = du > 0 ? (T)1 / du : (T)0, rl = dl > 0 ? (T)1 / dl : (T)0;
#pragma unroll
                for (int i = 0; i < DM; ++i) {
                    if (i >= P.d) break;
                    T vu, vl, dvu, dvl;
                    const bool c = P.mon[i] != 0;
                    coord_part<T>(tu[i], c, +1, vu, dvu);
                    coord_part<T>(tl[i], c, -1, vl, dvl);
                    T gu = 0, gl = 0;
                    if (P.norm == LIP_L1) {
                        gu = dvu * sq[i];
                        gl = dvl * sq[i];
                    } else if (P.norm == LIP_L2) {
                        gu = dvu * sq[i] * vu * ru;
                        gl = dvl * sq[i] * vl * rl;
                    } else {
                        if (i == mu && du > 0) gu = dvu * sq[i];
                        if (i == ml && dl > 0) gl = dvl * sq[i];
                    }
                    gq[i] = hm * (gu - gl);
                }
            }
            if (P.gy_fix) {
                const double c = 0.5 * (double)gb * fix_scale(P.gb_maxbits, P.nq);
                const unsigned long long f = (unsigned long long)__double2ll_rn(c);   // two's complement
                atomicAdd(P.gy_fix + u, f);
                atomicAdd(P.gy_fix + l, f);
            } else if (P.grad_y) {
                T* gy = static_cast<T*>(P.grad_y);
                atomicAdd(gy + u, (T)0.5 * gb);
                atomicAdd(gy + l, (T)0.5 * gb);
            }
            gm = (T)0.5 * gb * (du - dl);
        }
    }
    // fixed-shape block reduction of dL/dM
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) gm += __shfl_xor_sync(0xffffffffu, gm, off);   // warp sum in T
    __shared__ double red[BWD_THREADS / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)gm;
    __syncthreads();
    __shared__ bool last;
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < BWD_THREADS / 32; ++w) s += red[w];
        P.gm_part[blockIdx.x] = s;
        __threadfence();                                   // the partial is visible before the count
        last = atomicAdd(P.arrived, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || !P.grad_M) return;
    // the last block sums every block's partial in block order: the same shape every call
    __threadfence();
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += BWD_THREADS) s += P.gm_part[b];
    __shared__ double red2[BWD_THREADS];
    red2[threadIdx.x] = s;
    __syncthreads();
    for (int w = BWD_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red2[threadIdx.x] += red2[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *P.grad_M = red2[0];
}

int backward_blocks(int64_t nq) { return (int)((nq + BWD_THREADS - 1) / BWD_THREADS); }

cudaError_t launch_grad_max(int elem_bytes, const void* gbar, int64_t nq, unsigned* maxbits, cudaStream_t st) {
    const unsigned g = (unsigned)std::min<int64_t>(1024, (nq + 255) / 256 > 0 ? (nq + 255) / 256 : 1);
    if (elem_bytes == 8) grad_max_kernel<double><<<g, 256, 0, st>>>(static_cast<const double*>(gbar), nq, maxbits);
    else grad_max_kernel<float><<<g, 256, 0, st>>>(static_cast<const float*>(gbar), nq, maxbits);
    return cudaGetLastError();
}

cudaError_t launch_grad_y_fix(int elem_bytes, const unsigned long long* gy_fix, const unsigned* maxbits, int64_t nq,
                              int64_t N, void* grad_y, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    const unsigned g = (unsigned)((N + 255) / 256);
    if (elem_bytes == 8) grad_y_fix_kernel<double><<<g, 256, 0, st>>>(gy_fix, maxbits, nq, N, static_cast<double*>(grad_y));
    else grad_y_fix_kernel<float><<<g, 256, 0, st>>>(gy_fix, maxbits, nq, N, static_cast<float*>(grad_y));
    return cudaGetLastError();
}

cudaError_t launch_backward(int elem_bytes, const BwdParams& P, cudaStream_t st) {
    const int nb = backward_blocks(P.nq);
    if (nb > 0) {
        const bool wide = P.d > 16;
        if (elem_bytes == 8) {
            if (wide) backward_kernel<double, 32><<<nb, BWD_THREADS, 0, st>>>(P);
            else backward_kernel<double, 16><<<nb, BWD_THREADS, 0, st>>>(P);
        } else {
            if (wide) backward_kernel<float, 32><<<nb, BWD_THREADS, 0, st>>>(P);
            else backward_kernel<float, 16><<<nb, BWD_THREADS, 0, st>>>(P);
        }
    }
    return cudaGetLastError();
}

}  // namespace lip
