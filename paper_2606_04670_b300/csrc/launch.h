// Parameter blocks and host launchers shared between the kernel units and the C ABI.
#pragma once
#include <cmath>
#include <utility>

#include "scan.cuh"

namespace lip {

// The estimate's norm weights (Sec. 5 M_est, weighted norm): a power of two scales the
// layout's coordinate exactly; any other weight is applied to the FP32 coordinate
// differences in the pair kernels instead, because rounding w x into the layout leaves an
// error of the order of the difference of two points one FP32 unit apart.
inline bool est_weighted(const double* w, int d) {
    for (int j = 0; j < d; ++j) {
        int e;
        if (std::frexp(w[j], &e) != 0.5) return true;
    }
    return false;
}
// Layout scale of coordinate j: the weight when it is applied exactly there, else 1.
inline double est_layout_scale(const double* w, int j, bool weighted) { return weighted ? 1.0 : w[j]; }

struct EstParams {
    const float4* lay;    // layout: coordinates times est_layout_scale, nch = D + 1 channels per group
    int64_t N;
    int nb;               // tiles per side
    float4* cand;         // [nb * nb]: {ratio^2, bits(i), bits(j), valid}
    // block-cyclic share of the tile pairs: pair (I, J >= I) belongs to part
    // (I nb + J) mod nparts; a launch covers the pairs of `part` only
    int part = 0, nparts = 1;
    bool weighted = false;   // est_weighted: the pair kernels multiply differences by w
    float w[D_MAX] = {};     // the weights in FP32 (read only when weighted)
};

// Device words of the exact selection that follows the FP32 screen: q* (bits of the
// largest FP32 squared ratio, -1 without a pair), the number of tile pairs listed for the
// FP64 passes, R* (bits of the largest FP64 ratio among the pairs near q*, starting at +0)
// and the smallest key i << 32 | j attaining R*.
struct EstExactState {
    int q;
    int count;
    unsigned long long ratio;
    unsigned long long key;
};

struct EstFinalParams {
    const float4* cand;
    int nb;
    const void* X0;
    const void* y0;
    int d, norm, elem_bytes;
    double w[D_MAX];
    double* out;          // [3]: M_est, i, j (as doubles); [4] with write_key
    int part = 0, nparts = 1;   // the tile pairs whose candidates are read (as EstParams)
    int write_key = 0;    // out[3] = the FP64 ratio again, the key that orders parts (-1 without a pair)
    // the exact selection: the screen's layout (positions), its weighting, the position ->
    // data index map (nullptr: the identity), the list of tile pairs I << 16 | J to visit
    // (capacity: every tile pair) and the device words
    const float4* lay = nullptr;
    int64_t N = 0;
    bool weighted = false;
    const int* perm = nullptr;
    unsigned* list = nullptr;
    EstExactState* state = nullptr;
};

struct BwdParams {
    const void* Q;
    int64_t nq;
    int d, norm;
    double M;
    int8_t mon[D_MAX];
    double w[D_MAX];
    float sqf[D_MAX];        // sign_i w_i in float (FP32 handles)
    const void* X0;
    const int32_t* iu;
    const int32_t* il;
    const void* gbar;
    void* grad_Q;            // nullable, [nq][d]
    void* grad_y;            // nullable, [N], accumulated
    double* grad_M;          // nullable, overwritten
    double* gm_part;         // [backward_blocks(nq)] per-block partial sums of dL/dM
    unsigned* arrived;       // blocks done (zeroed before the launch)
    // deterministic grad_y: contributions summed as 64-bit fixed point (integer atomics
    // are associative), then added to grad_y
    unsigned long long* gy_fix;   // nullable, [N], zeroed before the launch
    const unsigned* gb_maxbits;   // largest |grad_g| (float bits), for the fixed-point scale
};

// Exact FP64 envelopes of FP64 handles from a float copy of the layout (screen64.cu).
struct Screen64Params {
    const double* Q;                  // caller's queries [nq][d]
    int64_t nq;
    int C, dl, nch;                   // the float layout
    int perm[D_MAX];
    double scale[D_MAX];              // M * sign_j * w_j
    const void* hot32;
    int64_t ngroups, groups_per_split;
    int nsplit1;                      // splits of the FP32 pass
    const PartialRec<float>* partial1;
    const unsigned* maxbits;          // [2]: largest |scaled coordinate| and |y| (float bits)
    MergeParams M;                    // d, norm, mon, w, M, X0, y0 for the FP64 values
    PartialRec<double>* partial2;     // [gridDim.y][nq]
};

int screen64_threads();
cudaError_t launch_build_hot32(const HotParams& P, unsigned* maxbits, cudaStream_t st);
cudaError_t launch_to_float(const double* a, int64_t n, float* out, cudaStream_t st);
cudaError_t launch_screen64(int norm, const Screen64Params& P, int gx, int gy, cudaStream_t st);

cudaError_t launch_merge(int elem_bytes, const MergeParams& P, cudaStream_t st);
cudaError_t launch_sqrt_fma(const float* s, float* out, int64_t n, cudaStream_t st);

// data-sharded evaluation (shard.cu)
cudaError_t launch_shard_keys(int elem_bytes, const void* partial, int nsplit, int64_t nq, const void* Q, int d,
                              int64_t index_base, int64_t* key_up, int64_t* key_lo, cudaStream_t st);
cudaError_t launch_shard_reeval(int elem_bytes, const MergeParams& P, int64_t index_base, int64_t N,
                                const int64_t* key_up, const int64_t* key_lo, double* hi64, double* lo64,
                                cudaStream_t st);
cudaError_t launch_shard_finish(int elem_bytes, int64_t nq, const int64_t* key_up, const int64_t* key_lo,
                                const double* hi64, const double* lo64, void* g, void* lo, void* hi, int32_t* idx_up,
                                int32_t* idx_lo, cudaStream_t st);
cudaError_t launch_build_hot(int elem_bytes, const HotParams& P, cudaStream_t st);
cudaError_t launch_pad_hot(int elem_bytes, void* hot, int64_t k0, int64_t k1, int nch, int dl, cudaStream_t st);

int estimate_tile_points();
cudaError_t launch_estimate_layout(int elem_bytes, const HotParams& P, cudaStream_t st);
cudaError_t launch_estimate(int norm, int d, const EstParams& P, cudaStream_t st);
// After launch_estimate: q* of the part and the list of its tile pairs whose screen
// maximum reaches q* (1 - 2^-16), then launch_estimate_exact.
cudaError_t launch_estimate_final(const EstFinalParams& P, cudaStream_t st);
constexpr int ESTIMATE_FINAL_LAUNCHES = 4;
// The exact selection over the listed tile pairs (state->q, state->count and P.list set):
// R*, then the lowest pair attaining it, then out.  Three launches.
cudaError_t launch_estimate_exact(const EstFinalParams& P, cudaStream_t st);
constexpr int ESTIMATE_EXACT_LAUNCHES = 3;

// tensor-core operand formats
constexpr int TC_TF32 = 0, TC_BF16 = 1, TC_FP16 = 2;
size_t tc_tile_bytes_for(int d, int fmt);
size_t tc_a_bytes_for(int d, int fmt);
size_t tc_rec_bytes();
// Spatial order of n points (row-major [n][d]): perm[position] = index, by a 16-bit Hilbert
// key of the first min(d, 16) coordinates and a stable radix sort (deterministic).
size_t spatial_order_scratch(int64_t n);
// bounds (nullable): [d] (min, max) of each coordinate's finite values, (0, 0) when none.
cudaError_t spatial_order(const float* X, int64_t n, int d, int* perm, float2* bounds, void* scratch,
                          cudaStream_t st);
int spatial_order_launches();
// The tensor-core form's data in spatial order (spatial_order of the data): tiles are
// built in position order, and the rescreen reads the position-ordered copies.
struct TcDataOrder {
    int* dperm;                      // [N] position -> data index
    float* Xs;                       // [N][d] the data rows in position order
    float* ys;                       // [N]
    float2* bounds;                  // [D_MAX] the data's bounding box, the centring of the pieces
    void* scratch;                   // spatial_order_scratch(N)
};
struct TcQueryOrder {
    int* qperm;                      // [nq] position -> query index
    void* scratch;                   // spatial_order_scratch(nq)
};
cudaError_t tc_prepare_data(const float* X0, const float* y0, int64_t N, int d, const double* scale,
                            unsigned* maxbits, char* tiles, int64_t ntiles, int fmt, const TcDataOrder& O,
                            cudaStream_t st);
cudaError_t tc_eval_launch(const float* Q, int64_t nq, int d, const double* scale, int64_t N,
                           const unsigned* maxbits, const char* btiles, int64_t ntiles, char* atiles, float4* qc,
                           void* rec, const double* w, double M, const float* X0, const float* y0, float* g, float* lo,
                           float* hi, int32_t* iu, int32_t* il, int* fb_count, int* fb_list, void* fb_state,
                           int* arrive, int64_t window, unsigned* err, int variant, int fmt,
                           const TcDataOrder& O, const TcQueryOrder& QO, cudaEvent_t ev0, cudaEvent_t ev1,
                           cudaStream_t st);
// Scratch of the scan's soft lockstep counters for nq queries against ntiles data tiles.
size_t tc_arrive_bytes(int64_t nq, int64_t ntiles);
// Deferred finiteness check of rows [n0, n0 + n) of X0 / y0 (element size es): records
// ERRBIT_NONFINITE in *err and replaces non-finite rows by a finite one (sanitize.cu).
// first_ok: one unsigned of scratch.
cudaError_t launch_sanitize(int es, void* X0, void* y0, int64_t n0, int64_t n, int d, unsigned* err,
                            unsigned* first_ok, cudaStream_t st);
// ------------------------------------------------ pruned scan (scan_pruned.cuh)
// Variants 6 and 7 of the exact FP32 scan: the data in spatial order with a box and value
// range per 32-point chunk, chunks skipped when they cannot change a query's extrema.
struct PrunedParams {
    ScanParams S;                 // hot: the layout in position order; partial: [nq] records
    const int* qperm;             // [nq] query position -> query index (spatial order)
    const int* dperm;             // [N] data position -> data index
    const float4* box;            // [nchunks][pruned_box_f4(D)] chunk records
    const float4* sbox;           // [nchunks / PRUNED_CPS][pruned_box_f4(D)]: records of 64 groups
    int64_t nchunks;
    unsigned long long* work;     // nullable: [0] evaluated (row, chunk) pairs, [1] tiles copied,
                                  // [2] (warp, chunk) pairs passing the warp-box test, per launch
};
// Chunk record: lo[D], hi[D] (layout coordinates), ylo (smallest y), yhv (largest value of
// the lower bound's channel: y, or the aux channel where the layout has one).
__host__ __device__ constexpr int pruned_box_f4(int D) { return (2 * D + 2 + 3) / 4; }
// Largest dimension with a pruned instantiation.
constexpr int PRUNED_DMAX = 8;
// The pruned scan's chunks: 16 points (4 groups), 16 of them to a 64-group super-chunk.
constexpr int PRUNED_CG = 4;
constexpr int PRUNED_CPS = 64 / PRUNED_CG;
// Unconstrained shapes (C = 0) have a pruned instantiation up to this many coordinates.
constexpr int PRUNED_UMAX = 16;
__host__ __device__ constexpr bool pruned_shape_available(int C, int U) {
    return C + U >= 1 && (C + U <= PRUNED_DMAX || (C == 0 && U <= PRUNED_UMAX));
}
using PrunedLaunchFn = cudaError_t (*)(const PrunedParams&, int gx, cudaStream_t);
struct PrunedKernelInfo {
    PrunedLaunchFn launch = nullptr;
    const void* kernel = nullptr;
    int rows = 0;
    int nch = 0;
};
PrunedKernelInfo scan_pruned_info(int norm, int C, int U, int variant);
// The records of the pruned scan's 16-point chunks of the position-ordered layout `hot`
// (N real points), then the records of every PRUNED_CPS consecutive chunks (sbox,
// nchunks a multiple of PRUNED_CPS).
cudaError_t launch_pruned_boxes(const void* hot, int64_t N, int64_t nchunks, int D, int nch, bool aux, void* box,
                                void* sbox, cudaStream_t st);
// The records of every `cpts`-point chunk of a layout (as above, without the unions).
cudaError_t launch_chunk_records(const void* hot, int64_t N, int64_t nchunks, int D, int nch, bool aux, void* box,
                                 cudaStream_t st, int cpts = 32);
// The union of every `per` consecutive records of `box` (nsuper of them) into sbox.
cudaError_t launch_record_union(const void* box, int64_t nsuper, int per, int D, void* sbox, cudaStream_t st);

// ------------------------------------------------ pruned estimate (estimate_pruned.cu)
// M_est over the data in spatial order: the screen pass finds the largest FP32 squared
// ratio q*, skipping tile pairs and 32-point chunks whose exact FP32 bound stays below
// the largest value found so far (with the selection's 2^-16 margin), and records each
// tile pair's largest value; the select kernel lists the tile pairs that reach
// q* (1 - 2^-16) for the exact selection (launch_estimate_exact).
struct EstPrunedParams {
    const float4* lay;            // the estimate layout in position order
    int64_t N;
    int nb;                       // 512-point tiles
    const float4* cbox;           // [nb * 16][pruned_box_f4(d)] chunk records
    const float4* tbox;           // [nb][pruned_box_f4(d)] tile records
    int* gbest;                   // bits of the largest FP32 squared ratio q*, -1 none
    float* bq;                    // [nb (nb + 1) / 2] each tile pair's largest value (-1: none, skipped)
    bool weighted = false;        // as EstParams
    float w[PRUNED_DMAX] = {};
    // optional counters: tile pairs entered, (warp, chunk) pairs evaluated
    unsigned long long* work = nullptr;
};
cudaError_t launch_estimate_pruned(int norm, int d, const EstPrunedParams& P, cudaStream_t st);
bool estimate_pruned_available(int d);
// q* from P.gbest and the list of tile pairs whose P.bq reaches q* (1 - 2^-16), into F.state / F.list.
cudaError_t launch_estimate_pruned_select(const EstPrunedParams& P, const EstFinalParams& F, cudaStream_t st);

// Scratch of the device-side fallback for nq queries (fb_state above).
size_t tc_fallback_state_bytes(int64_t nq);

struct TopkParams {
    const void* Q;
    int64_t nq;
    int d, C, dl, nch;
    int perm[D_MAX];
    double scale[D_MAX];
    const void* hot;
    int64_t ngroups, groups_per_split;
    void* partial;           // [nsplit][nq][2][K]: values then indices
};

struct TopkMergeParams {
    const void* Q;
    int64_t nq;
    int d, k, K, nsplit, norm;
    double M;
    int8_t mon[D_MAX];
    double w[D_MAX];
    double wk[8];
    const void* X0;
    const void* y0;
    const void* partial;
    void *g, *lo, *hi;
    int32_t *idx_up, *idx_lo;   // [nq][k]
};

int topk_threads();
cudaError_t launch_topk(int elem_bytes, int norm, int K, const TopkParams& P, int gx, int gy, const TopkMergeParams& M,
                        cudaStream_t st);

int backward_blocks(int64_t nq);
cudaError_t launch_backward(int elem_bytes, const BwdParams& P, cudaStream_t st);
cudaError_t launch_grad_max(int elem_bytes, const void* gbar, int64_t nq, unsigned* maxbits, cudaStream_t st);
cudaError_t launch_grad_y_fix(int elem_bytes, const unsigned long long* gy_fix, const unsigned* maxbits, int64_t nq,
                              int64_t N, void* grad_y, cudaStream_t st);

// ------------------------------------------------ local Lipschitz constants (Sec. 4.3)

constexpr int LOC_KNOTS = 32;        // table stride: up to 31 knots and the last segment
constexpr int LOC_BUCKETS = 2048;    // knot-lookup buckets of the evaluation scan

struct LocMeta {
    int npos;                        // positive sampled distances
    int m;                           // distinct knots
    unsigned rbits;                  // largest |scaled coordinate| (float bits)
    int bucket_ok;                   // 1 if no lookup bucket holds two knots
    float scale;                     // lookup buckets per unit distance
    int n_over;                      // data whose table candidate list overflowed
    int max_cand;                    // longest candidate list that did not
    int pad;
};

struct LocalParams {
    const void* X0;                  // caller's data [N][d], float or double (es bytes)
    const void* y0;
    int es;
    int64_t N, npad;
    int d, dp, pr, norm, m;          // dp: d rounded up to 4; m: knots requested or given
    double w[D_MAX];
    // monotone coordinates (one-sided distances; the records hold sign * w * x)
    int mono;                        // 1 if some coordinate is constrained
    unsigned cmask;                  // bit i: coordinate i is constrained
    int8_t mon[D_MAX];
    int64_t S;                       // sampled pairs
    uint64_t seed;
    float* rec;                      // [npad][pr = dp + 4]: w-scaled coordinates (0-padded to dp),
                                     // y, d1 (float), F (float), 0
    float* mt;                       // [npad][LOC_KNOTS]: FP32 table (the screen's lower bounds until the table)
    double* mt64;                    // [N][LOC_KNOTS]: exact table
    double* d1;                      // [N]
    double* F;                       // [N]
    double* T64;                     // [LOC_KNOTS] knots, +inf padded
    float* Tf;                       // [3][LOC_KNOTS] knots rounded to nearest, down, up
    double* raw;                     // [LOC_KNOTS] quantile picks (or the given knots)
    double* sample;                  // [S] sampled distances
    int* counts;                     // [2][S] samples below / at most each sample
    float* ubound;                   // [N] the screen's upper bounds of d1
    unsigned* bpack;                 // [LOC_BUCKETS] bucket table: bits of the knot inside the
                                     // bucket (+inf if none), low 5 bits replaced by the count below
    int* cand;                       // [N][local_candidates()] table candidate lists
    int* ncand;                      // [N] their lengths
    int* over;                       // [N] data whose list overflowed
    LocMeta* meta;
};

struct LocalScanParams {
    const void* Q;                   // float or double (es bytes)
    int es;
    int64_t nq;
    int d, dp;
    double w[D_MAX];                 // the query's scaling (sign * w with monotone coordinates)
    int mono;
    unsigned cmask;
    const float* rec;
    const float* mt;
    const float* Tf;
    const unsigned* bpack;           // packed bucket table (LocalParams::bpack)
    float scale;
    int bucket_ok;                   // the bucket lookup applies (else binary search)
    int64_t npad, points_per_split;
    void* partial;                   // [nsplit][nq] PartialRec<float>
};

struct LocalMergeParams {
    const void* Q;                   // float or double (es bytes), as X0, y0 and the outputs
    int es;
    int64_t nq;
    int d, norm, m, nsplit;
    double w[D_MAX];
    int mono;
    int8_t mon[D_MAX];
    const void* X0;
    const void* y0;
    const double* d1;
    const double* F;
    const double* mt64;
    const double* T64;
    const void* partial;
    void *g, *lo, *hi;
    int32_t *idx_up, *idx_lo;
};

struct LocalTopkWeights {
    double wk[8];
};

int local_dim_pad(int d);
int local_queries_per_block_mono();
int local_topk_threads();
cudaError_t launch_local_eval_k(int norm, int k, int K, const LocalScanParams& S, int gx, int nsplit,
                                const LocalMergeParams& M, const LocalTopkWeights& W, cudaStream_t st);
int local_record_floats(int d);
int64_t local_pad(int64_t N);
int local_scan_tile();
int local_queries_per_block(int d);
cudaError_t launch_local_layout(const LocalParams& P, cudaStream_t st);
cudaError_t launch_local_knots(const LocalParams& P, bool sampled, cudaStream_t st);
int local_candidates();
// m: the distinct knots the knots kernel kept (sizes the screen's shared memory)
cudaError_t launch_local_table(const LocalParams& P, bool bucket_ok, int m, cudaStream_t st);
cudaError_t launch_local_eval(int norm, const LocalScanParams& S, int gx, int nsplit, bool bucket,
                              const LocalMergeParams& M, cudaStream_t st);

// ------------------------------------------------ penalty smoothing (Sec. 4.4)

struct SmoothParams {
    const void* X0;                  // caller's data [N][d], float or double (es bytes)
    const void* y0;
    int es;
    int64_t N, npad;
    int d, dp, C, norm;              // dp: d rounded up to 4; C: constrained coordinates (first)
    int perm[D_MAX];
    double scale[D_MAX];             // M * w * sign, in layout order
    double p;                        // penalty weight of Eq. (optim)
    float* rec;                      // [npad][dp + 4]: scaled coordinates, z = y + eps, 0, 0, 0
    double* rec64;                   // FP64 handles: [npad][dp + 2] scaled coordinates, z, 0 (FP64 pass)
    double* partial;                 // [nsplit][N][2]: R - C and S per split (row side)
    unsigned long long* colfix;      // [N]: R - C of the column side, signed fixed point
    unsigned* zbits;                 // [2]: largest z and -z (order-preserving bits)
    int nsplit;
    int64_t points_per_split;
};

int smooth_tile();
int smooth_rows_per_block(int es);
int smooth_reduce_blocks();
cudaError_t launch_smooth_objective(const SmoothParams& P, const double* eps, double* grad, double* block_sums,
                                    double* out, int gx, cudaStream_t st);
cudaError_t launch_vec_reduce(const double* a, const double* b, int64_t n, int op, double* partial, double* out,
                              cudaStream_t st);
cudaError_t launch_vec_axpy(double* out, const double* a, double alpha, const double* b, int64_t n, cudaStream_t st);
cudaError_t launch_vec_scale(double* out, const double* a, double alpha, int64_t n, cudaStream_t st);
cudaError_t launch_apply_eps(void* y0, int es, const double* eps, int64_t n, cudaStream_t st);

}  // namespace lip
