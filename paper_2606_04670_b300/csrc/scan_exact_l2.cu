// Exact-shape FP32 scan kernels for the L2 norm.
#include "scan_inst.cuh"

namespace lip {
ScanKernelInfo scan_exact_info_l2(int C, int U, int v) {
    static ExactTable<LIP_L2> t;
    if (C < 0 || U < 0 || C > EXACT_DMAX || U > EXACT_DMAX || v < 0 || v >= SCAN_VARIANTS) return {};
    return t.tab[C][U][v];
}
}  // namespace lip
