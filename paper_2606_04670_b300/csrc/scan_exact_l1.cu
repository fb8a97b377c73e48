// Exact-shape FP32 scan kernels for the L1 norm.
#include "scan_inst.cuh"

namespace lip {
ScanKernelInfo scan_exact_info_l1(int C, int U, int v) {
    static ExactTable<LIP_L1> t;
    if (C < 0 || U < 0 || C > EXACT_DMAX || U > EXACT_DMAX || v < 0 || v >= SCAN_VARIANTS) return {};
    return t.tab[C][U][v];
}
}  // namespace lip
