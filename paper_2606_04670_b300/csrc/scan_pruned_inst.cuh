// Instantiation table of the pruned scan kernels for one norm (scan_pruned.cuh).
#pragma once
#include <utility>

#include "scan_pruned.cuh"

namespace lip {

// variant 6: half the exact kernel's queries per thread; variant 7: the full count
__host__ __device__ constexpr int pruned_rows(int D, int v) { return rows_for_variant(D, v == 6 ? 1 : 0); }

template <int NORM, int C, int U, int R>
cudaError_t launch_scan_pruned(const PrunedParams& P, int gx, cudaStream_t st) {
    constexpr int NCH = ExactShape<NORM, C, U, true>::NCH;
    auto kern = scan_pruned_kernel<NORM, C, U, R>;
    constexpr int NB4 = pruned_box_f4(C + U);
    constexpr int RECS = TILE_GROUPS_MAX / PRUNED_CG;        // chunk records a stage holds
    const size_t smem = (size_t)PRUNED_STAGES * (P.S.tile_groups * NCH + RECS * NB4) * sizeof(float4);
    static cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   PRUNED_STAGES * (TILE_GROUPS_MAX * NCH + RECS * NB4) * (int)sizeof(float4));
    if (attr != cudaSuccess) return attr;
    kern<<<gx, SCAN_THREADS, smem, st>>>(P);
    return cudaGetLastError();
}

template <int NORM>
struct PrunedTable {
    PrunedKernelInfo tab[PRUNED_DMAX + 1][PRUNED_UMAX + 1][2];
    template <int C, int U, int V>
    void fill_variant() {
        constexpr int R = pruned_rows(C + U, V);
        PrunedKernelInfo& e = tab[C][U][V - 6];
        e.launch = &launch_scan_pruned<NORM, C, U, R>;
        e.kernel = reinterpret_cast<const void*>(&scan_pruned_kernel<NORM, C, U, R>);
        e.rows = R;
        e.nch = ExactShape<NORM, C, U, true>::NCH;
    }
    template <int K>
    void fill_one() {
        constexpr int C = K / (PRUNED_UMAX + 1), U = K % (PRUNED_UMAX + 1);
        if constexpr (pruned_shape_available(C, U)) {
            fill_variant<C, U, 6>();
            fill_variant<C, U, 7>();
        }
    }
    template <int... K>
    void fill(std::integer_sequence<int, K...>) { (fill_one<K>(), ...); }
    PrunedTable() { fill(std::make_integer_sequence<int, (PRUNED_DMAX + 1) * (PRUNED_UMAX + 1)>{}); }
};

}  // namespace lip
