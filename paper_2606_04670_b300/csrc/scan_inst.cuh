// Instantiation table of the exact-shape scan kernels for one norm (SCAN_NORM).
#pragma once
#include <utility>

#include "scan.cuh"

namespace lip {

template <int NORM, int C, int U, int V>
cudaError_t launch_scan_exact(const ScanParams& P, int gx, int gy, cudaStream_t st) {
    constexpr int R = rows_for_variant(C + U, V);
    constexpr int FSR = fsr_for_variant(V);
    constexpr int NCH = ExactShape<NORM, C, U>::NCH;
    auto kern = scan_exact_kernel<NORM, C, U, R, FSR>;
    const size_t smem = (size_t)SCAN_STAGES * P.tile_groups * NCH * sizeof(float4);
    static cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   SCAN_STAGES * TILE_GROUPS_MAX * NCH * (int)sizeof(float4));
    if (attr != cudaSuccess) return attr;
    kern<<<dim3(gx, gy), SCAN_THREADS, smem, st>>>(P);
    return cudaGetLastError();
}

template <int NORM>
struct ExactTable {
    ScanKernelInfo tab[EXACT_DMAX + 1][EXACT_DMAX + 1][SCAN_VARIANTS];
    template <int C, int U, int V>
    void fill_variant() {
        ScanKernelInfo& e = tab[C][U][V];
        e.launch = &launch_scan_exact<NORM, C, U, V>;
        e.kernel = reinterpret_cast<const void*>(
            &scan_exact_kernel<NORM, C, U, rows_for_variant(C + U, V), fsr_for_variant(V)>);
        e.rows = rows_for_variant(C + U, V);
        e.nch = ExactShape<NORM, C, U>::NCH;
    }
    template <int K>
    void fill_one() {
        constexpr int C = K / (EXACT_DMAX + 1), U = K % (EXACT_DMAX + 1);
        if constexpr (exact_shape_available(C, U)) {
            fill_variant<C, U, 0>();
            fill_variant<C, U, 1>();
            if constexpr (fma_sqrt_shape(NORM, C, U)) {
                fill_variant<C, U, 2>();
                fill_variant<C, U, 3>();
                fill_variant<C, U, 4>();
                fill_variant<C, U, 5>();
            } else {
                for (int v = 2; v < SCAN_VARIANTS; ++v) tab[C][U][v] = tab[C][U][v & 1];
            }
        }
    }
    template <int... K>
    void fill(std::integer_sequence<int, K...>) { (fill_one<K>(), ...); }
    ExactTable() { fill(std::make_integer_sequence<int, (EXACT_DMAX + 1) * (EXACT_DMAX + 1)>{}); }
};

}  // namespace lip
