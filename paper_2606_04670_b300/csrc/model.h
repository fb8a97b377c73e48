// Private header of the library's host code: the handle behind lip_handle and the
// helpers that the C ABI's source files share.  Not part of the interface.
#pragma once
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "launch.h"

namespace lip {

// Records a one-line message for lip_last_error and returns s.
lip_status fail(lip_status s, const char* fmt, ...);
// The lip_status (and message) for a failed CUDA call.
lip_status cuda_fail(cudaError_t e, const char* what);
// Adds to the count of the library's kernel launches (lip_kernel_launches).
void count_launches(uint64_t n);
// cudaMalloc for every device buffer the library owns.  lip_debug_fail_alloc can make it
// report cudaErrorMemoryAllocation (without allocating) to test the OOM paths.
cudaError_t dev_malloc(void** p, size_t bytes);

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

#define CUDA_TRY(expr)                                              \
    do {                                                            \
        cudaError_t e_ = (expr);                                    \
        if (e_ != cudaSuccess) return lip::cuda_fail(e_, #expr);    \
    } while (0)

#define LIP_TRY(expr)                                               \
    do {                                                            \
        lip_status s_ = (expr);                                     \
        if (s_ != LIP_OK) return s_;                                \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Device buffer that only grows; freed with the handle.
struct Scratch {
    void* p = nullptr;
    size_t bytes = 0;
    lip_status ensure(size_t need, const char* what) {
        if (need <= bytes) return LIP_OK;
        if (p) {
            cudaError_t e = cudaFree(p);   // implicit device synchronisation: no user in flight
            p = nullptr;
            bytes = 0;
            if (e != cudaSuccess) return cuda_fail(e, what);
        }
        size_t sz = std::max<size_t>(need, 256);
        sz = (sz + 255) & ~size_t(255);
        cudaError_t e = dev_malloc(&p, sz);
        if (e != cudaSuccess) { p = nullptr; return cuda_fail(e, what); }
        bytes = sz;
        return LIP_OK;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
};

}  // namespace lip

using namespace lip;

struct lip_model {
    int device = 0;
    int sms = 148;
    int d = 0, C = 0, norm = LIP_L2, prec = LIP_FP32, esize = 4;
    double M = 0.0;
    int8_t mon[D_MAX] = {};
    double w[D_MAX] = {};
    int perm[D_MAX] = {};
    double sgnw[D_MAX] = {};
    bool exact = false;
    int dl = 0, nch = 0, aux = 0;
    int64_t N = 0, cap = 0, cap_pad = 0;
    void* X0 = nullptr;
    void* y0 = nullptr;
    void* hot = nullptr;
    unsigned* status = nullptr;       // [0]: runtime error bits, [1]: finiteness check
    ScanKernelInfo kinfo;
    int occ_blocks = 1;
    int tile_groups = 32;             // groups per shared-memory tile (8, 16, 32 or 64)
    int splits = 0;                   // 0 = automatic
    int last_splits = 0;
    int variant = 0;
    // fault injection for tests (lip_debug_scan_fault): the exact scan's wait limit and the
    // data tile whose bulk copy it does not issue
    unsigned long long dbg_wait_ns = 0;   // 0: the default limit
    int dbg_skip_tile = -1;               // -1: none
    Scratch partial, est, bwd, io;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
    cudaEvent_t ev_scan0 = nullptr, ev_scan1 = nullptr;   // caller's timing events
    // tensor-core forms (LIP_TC_TF32, LIP_TC_BF16, LIP_TC_FP16)
    // FP64 handles: a float copy of the layout for the FP32 screen of the exact FP64 scan
    void* hot32 = nullptr;
    int dl32 = 0, nch32 = 0, aux32 = 0;
    bool exact32 = false, s32_dirty = true;
    int fp64_mode = 0;                 // 0: FP32 screen + FP64 candidates; 1: FP64 scan throughout
    ScanKernelInfo kinfo32;
    int occ32 = 1;
    unsigned* s32_max = nullptr;       // [2] largest |scaled coordinate| and |y| (float bits)
    Scratch s64;                       // float queries and the FP32 pass's partials
    bool tc = false, tc_dirty = true;
    int tc_fmt = 0;                    // TC_TF32, TC_BF16 or TC_FP16 (operand split)
    int tc_variant = 0;                // 0: 16 epilogue warps, 1: 8
    int64_t tc_ntiles_cap = 0;
    char* tc_btiles = nullptr;
    unsigned* tc_maxbits = nullptr;    // [2] max |x^|, max |y| (float bits)
    Scratch tc_q;
    Scratch tc_order;                  // the data's spatial order and position-ordered copies
    int64_t tc_window = 0;              // lip_set_tc_window (0: the library's default)
    bool pruned = false;                // variants 6 / 7: the pruned scan (scan_pruned.cuh)
    PrunedKernelInfo pinfo;
    Scratch sp_data, sp_q;              // position-ordered layout and chunk records; query order
    bool sp_dirty = true;               // the position-ordered layout needs a rebuild
    int64_t sp_total = -1;              // (row, chunk) pairs of the last pruned scan, -1 if none
    int64_t sp_tiles = -1;              // its blocks x data tiles
    int est_form = 0;                   // lip_estimate_M: 0 pruned from N = 32768, 1 always full, 2 pruned where available
    int64_t est_work[3] = {-1, -1, -1};   // lip_last_estimate_work
    // lip_estimate_M_async: the result (4 doubles) and the pruned form's work counters are
    // copied to est_back (pinned) and est_done is recorded after the copy
    unsigned char* est_back = nullptr;  // 64 bytes
    cudaEvent_t est_done = nullptr;
    int est_pending = 0;                // 0 none, 1 queued on the device, 2 known on the host
    double est_host_res[4] = {0, -1, -1, -1};   // the result when est_pending == 2
    int64_t est_pending_total = -1;     // est_work[2] of the queued estimate (-1: full form)
    int* tc_fb_count = nullptr;         // device count of the last tensor-core lip_eval's fallback
    // local Lipschitz constants (Sec. 4.3), valid until the data change
    bool loc_valid = false;
    bool loc_bucket = true;            // the evaluation's bucket lookup applies (else binary search)
    float loc_scale = 0.f;
    int32_t loc_over = 0, loc_max_cand = 0;   // statistics of the last table fit
    int loc_m = 0;
    double loc_T[LOC_KNOTS] = {};
    Scratch loc_buf, loc_tmp;          // layout and tables; sampled distances and bounds
    char* loc_small = nullptr;         // knots (FP64, raw, float roundings) and LocMeta
    // penalty smoothing (Sec. 4.4): pair-pass layout and partials, L-BFGS vectors, scalars
    Scratch sm_rec, sm_part, sm_vec, sm_small;
};

namespace lip {

void fill_scan_params(const lip_model* h, ScanParams& P);
void fill_hot_params(const lip_model* h, HotParams& P, int64_t k0, int64_t k1);
// Number of N-splits: enough blocks to fill the GPU in nearly whole waves.
int choose_splits(const lip_model* h, int64_t gx, int64_t tiles);

}  // namespace lip
