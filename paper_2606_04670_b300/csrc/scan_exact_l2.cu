// Exact-shape FP32 scan kernels for the L2 norm.
#include "scan_inst.cuh"

namespace lip {
ScanKernelInfo scan_exact_info_l2(int C, int U) {
    static ExactTable<LIP_L2> t;
    if (C < 0 || U < 0 || C > D_MAX || U > D_MAX) return {};
    return t.tab[C][U];
}
}  // namespace lip
