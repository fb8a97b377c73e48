// Pruned scan kernels (chunk bounds over the data in spatial order) for the L2 norm.
#include "scan_pruned_inst.cuh"

namespace lip {
PrunedKernelInfo scan_pruned_info_l2(int C, int U, int v) {
    static PrunedTable<LIP_L2> t;
    if (C < 0 || U < 0 || C > PRUNED_DMAX || U > PRUNED_UMAX || (v != 6 && v != 7)) return {};
    return t.tab[C][U][v - 6];
}
}  // namespace lip
