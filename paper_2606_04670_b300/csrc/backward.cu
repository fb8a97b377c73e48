// Gradient of L = sum_q gbar_q g(q) through the saved argmin u_q / argmax l_q
// (g = (H_up + H_lo)/2, Sec. 3 Eq. (eq:g); piecewise smooth, differentiable almost
// everywhere, Table 1):
//   dL/dq_i   = gbar M/2 ( d dist_up(q, x^u)/dq_i - d dist_lo(q, x^l)/dq_i )
//   dL/dy^k   = 1/2 sum_q gbar_q ([u_q = k] + [l_q = k])
//   dL/dM     = 1/2 sum_q gbar_q ( dist_up(q, x^u) - dist_lo(q, x^l) )
// One thread per query, in the caller's coordinates, arithmetic in the handle's
// element type, all in one launch: dL/dy is added straight into the caller's grad_y with
// atomics of the element type, and dL/dM is a fixed-shape two-level FP64 reduction
// finished by the last block to arrive (bitwise reproducible); the per-query terms and the
// warp sums are in the element type, the block and grid sums in FP64.
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


template <typename T>
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
            T qv[D_MAX], tu[D_MAX], tl[D_MAX], sq[D_MAX];
#pragma unroll
            for (int i = 0; i < D_MAX; ++i) {
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
            for (int i = 0; i < D_MAX; ++i) {
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
                for (int i = 0; i < D_MAX; ++i) {
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
            if (P.grad_y) {
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

cudaError_t launch_backward(int elem_bytes, const BwdParams& P, cudaStream_t st) {
    const int nb = backward_blocks(P.nq);
    if (nb > 0) {
        if (elem_bytes == 8) backward_kernel<double><<<nb, BWD_THREADS, 0, st>>>(P);
        else backward_kernel<float><<<nb, BWD_THREADS, 0, st>>>(P);
    }
    return cudaGetLastError();
}

}  // namespace lip
