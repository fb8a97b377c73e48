// Throughput of the special-function pipe (MUFU) for sqrt.approx.ftz.f32 and
// rsqrt.approx.ftz.f32: eight independent dependency chains per thread, 8 blocks of 256
// threads per SM, 4096 steps.  Prints one line per timed launch with the results per SM
// per clock at the device's maximum SM clock.  Used by tests/test_gpu_mufu_rate.py to check
// the MUFU roof the benchmark divides by (16 results per SM per clock).
#include <cstdio>
#include <cuda_runtime.h>

template <int OP>
__global__ void __launch_bounds__(256) chains(float* out, int iters, float c) {
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = 1.0f + threadIdx.x * 1e-3f + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float r;
            if (OP == 0) asm volatile("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[k]));
            else asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[k]));
            a[k] = r + c;
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // index < gridDim.x * blockDim.x
}

int main() {
    int sms = 0, khz = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess ||
        cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, 0) != cudaSuccess) {
        printf("no device\n");
        return 1;
    }
    const int blocks = sms * 8, threads = 256, iters = 4096;
    float* out = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(float)) != cudaSuccess) return 1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int op = 0; op < 2; ++op) {
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0);
            if (op == 0) chains<0><<<blocks, threads>>>(out, iters, 0.5f);
            else chains<1><<<blocks, threads>>>(out, iters, 0.5f);
            cudaEventRecord(e1);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double ops = (double)blocks * threads * iters * 8;
            printf("%s %d %.4f %.4f\n", op == 0 ? "sqrt" : "rsqrt", rep, ms,
                   ops / (ms * 1e-3) / sms / (khz * 1e3));
        }
    }
    cudaError_t e = cudaDeviceSynchronize();
    cudaFree(out);
    printf("status %s\n", cudaGetErrorString(e));
    return e == cudaSuccess ? 0 : 1;
}
