// Gradient of L = sum_q gbar_q g(q) through the saved argmin u_q / argmax l_q
// (g = (H_up + H_lo)/2, Sec. 3 Eq. (eq:g); piecewise smooth, differentiable almost
// everywhere, Table 1):
//   dL/dq_i   = gbar M/2 ( d dist_up(q, x^u)/dq_i - d dist_lo(q, x^l)/dq_i )
//   dL/dy^k   = 1/2 sum_q gbar_q ([u_q = k] + [l_q = k])
//   dL/dM     = 1/2 sum_q gbar_q ( dist_up(q, x^u) - dist_lo(q, x^l) )
// One thread per query, in the caller's coordinates, arithmetic in the handle's
// element type; dL/dy is accumulated with FP64 atomics in scratch, dL/dM by a
// fixed-shape two-level FP64 reduction (bitwise reproducible).
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
__device__ __forceinline__ T coord_t(const BwdParams& P, const T* q, const T* x, int i, T& sq) {
    sq = (P.mon[i] < 0 ? (T)-1 : (T)1) * (T)P.w[i];   // dt'/dq_i
    return (q[i] - x[i]) * sq;
}

template <typename T>
__global__ void __launch_bounds__(BWD_THREADS) backward_kernel(const BwdParams P) {
    const int64_t qi = (int64_t)blockIdx.x * BWD_THREADS + threadIdx.x;
    double gm = 0.0;
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
            // pass 1: the two distances (and the Linf arg-max coordinates, lowest on ties)
            T au = 0, al = 0;
            int mu = -1, ml = -1;
            for (int i = 0; i < P.d; ++i) {
                T sq, vu, vl, dv;
                const bool c = P.mon[i] != 0;
                coord_part<T>(coord_t<T>(P, q, xu, i, sq), c, +1, vu, dv);
                coord_part<T>(coord_t<T>(P, q, xl, i, sq), c, -1, vl, dv);
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
                for (int i = 0; i < P.d; ++i) {
                    T sq, vu, vl, dvu, dvl;
                    const bool c = P.mon[i] != 0;
                    coord_part<T>(coord_t<T>(P, q, xu, i, sq), c, +1, vu, dvu);
                    coord_part<T>(coord_t<T>(P, q, xl, i, sq), c, -1, vl, dvl);
                    T gu = 0, gl = 0;
                    if (P.norm == LIP_L1) {
                        gu = dvu * sq;
                        gl = dvl * sq;
                    } else if (P.norm == LIP_L2) {
                        if (du > 0) gu = dvu * sq * vu / du;
                        if (dl > 0) gl = dvl * sq * vl / dl;
                    } else {
                        if (i == mu && du > 0) gu = dvu * sq;
                        if (i == ml && dl > 0) gl = dvl * sq;
                    }
                    gq[i] = hm * (gu - gl);
                }
            }
            if (P.gy64) {
                atomicAdd(P.gy64 + u, 0.5 * (double)gb);
                atomicAdd(P.gy64 + l, 0.5 * (double)gb);
            }
            gm = 0.5 * (double)gb * ((double)du - (double)dl);
        }
    }
    // fixed-shape block reduction of dL/dM
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) gm += __shfl_xor_sync(0xffffffffu, gm, off);
    __shared__ double red[BWD_THREADS / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = gm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < BWD_THREADS / 32; ++w) s += red[w];
        P.gm_part[blockIdx.x] = s;
    }
}

__global__ void sum_partials_kernel(const double* part, int n, double* out) {
    __shared__ double red[1024];
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) s += part[k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

template <typename T>
__global__ void add_grad_y_kernel(const double* gy64, int64_t n, T* grad_y) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) grad_y[k] = (T)((double)grad_y[k] + gy64[k]);
}

int backward_blocks(int64_t nq) { return (int)((nq + BWD_THREADS - 1) / BWD_THREADS); }

cudaError_t launch_backward(int elem_bytes, const BwdParams& P, int64_t N, void* grad_y, double* grad_M,
                            cudaStream_t st) {
    const int nb = backward_blocks(P.nq);
    if (nb > 0) {
        if (elem_bytes == 8) backward_kernel<double><<<nb, BWD_THREADS, 0, st>>>(P);
        else backward_kernel<float><<<nb, BWD_THREADS, 0, st>>>(P);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (grad_M) {
        sum_partials_kernel<<<1, 1024, 0, st>>>(P.gm_part, nb, grad_M);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (grad_y && P.gy64 && N > 0) {
        const unsigned g = (unsigned)((N + 255) / 256);
        if (elem_bytes == 8) add_grad_y_kernel<double><<<g, 256, 0, st>>>(P.gy64, N, static_cast<double*>(grad_y));
        else add_grad_y_kernel<float><<<g, 256, 0, st>>>(P.gy64, N, static_cast<float*>(grad_y));
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace lip
