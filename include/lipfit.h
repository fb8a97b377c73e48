/*
 * lipfit.h -- C ABI of liblipfit.so: optimal Lipschitz interpolation on a B300 (sm_103a).
 *
 * What it computes (G. Beliakov, "Fitting scattered data with optional monotonicity
 * constraints on GPU: LipFit package"):
 *
 *   H_up(x) = min_k ( y^k + M dist_up(x, x^k) )   Sec. 3, Eq. (upperlower)
 *   H_lo(x) = max_k ( y^k - M dist_lo(x, x^k) )   Sec. 3, Eq. (upperlower)
 *   g(x)    = ( H_up(x) + H_lo(x) ) / 2           Sec. 3, Eq. (eq:g)
 *
 * dist is the L1, L2 or Linf norm of the weighted coordinate differences
 * w_i (x_i - x^k_i).  Coordinates in which the function is increasing use the
 * positive part (x_i - x^k_i)_+ in dist_up and (x^k_i - x_i)_+ in dist_lo
 * (Sec. 4.1, Eq. (distmon) and the bounds g <= y^k for x below x^k, g >= y^k for x
 * above x^k stated there); decreasing coordinates are mirrored.  Unconstrained
 * coordinates use |x_i - x^k_i| in both.  Ties in the min/max go to the lowest k.
 *
 * Conventions for every call:
 *  - Array pointers are DEVICE pointers owned by the caller, unless the function name
 *    ends in _host (then they are host pointers; page-locked memory gives the fastest
 *    copies).  Matrices are row-major and dense: X is [N][d], Q is [nq][d].
 *  - Element type: float for LIP_FP32 / LIP_TC_* handles, double for LIP_FP64 handles
 *    (X, y, Q and the g/lo/hi outputs alike).  Indices are int32 (N < 2^31).
 *  - Calls are ordered on the given CUDA stream (NULL = legacy default stream) and
 *    return before the GPU work finishes, except where a call says it synchronises.
 *  - A handle is used by one host thread and one stream at a time; its scratch memory
 *    is reused by the next call on it.
 *  - No C++ exception, abort or exit crosses this interface.  Every failure is a
 *    lip_status; lip_last_error() returns a one-line explanation (thread-local).
 *  - Argument errors are detected on the host before any GPU work is queued, so they
 *    leave the handle and the stream untouched.
 */
#ifndef LIPFIT_H
#define LIPFIT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Symbols of this interface are exported from liblipfit.so; everything else is hidden. */
#if defined(__GNUC__)
#define LIP_API __attribute__((visibility("default")))
#else
#define LIP_API
#endif

typedef enum {
    LIP_OK = 0,
    LIP_ERR_ARG = 1,          /* bad argument: null pointer, size out of range, M < 0 ...   */
    LIP_ERR_NONFINITE = 2,    /* NaN or Inf in the data X or y                              */
    LIP_ERR_OOM = 3,          /* device or host allocation failed                          */
    LIP_ERR_CUDA = 4,         /* a CUDA runtime call failed (detail in lip_last_error)      */
    LIP_ERR_CAPACITY = 5,     /* lip_add beyond the reserved capacity                       */
    LIP_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up (see lip_check)         */
    LIP_ERR_UNSUPPORTED = 7,  /* valid request this build does not handle                  */
    LIP_ERR_NO_DEVICE = 8,    /* no CUDA device visible                                     */
    LIP_ERR_STATE = 9         /* call out of order (lip_eval_local before lip_local_fit)    */
} lip_status;

typedef enum { LIP_L1 = 1, LIP_L2 = 2, LIP_LINF = 3 } lip_norm;

typedef enum {
    LIP_FP32 = 0,      /* FP32 arithmetic in the all-pairs scan, FP64 re-evaluation of winners */
    LIP_FP64 = 1,      /* FP64 data and results: FP32 screen, FP64 values (see lip_set_tuning) */
    LIP_TC_BF16 = 2,   /* L2 only: tensor-core cross term (bf16 split), exact FP64 rescreen  */
    LIP_TC_TF32 = 3,   /* L2 only: tensor-core cross term (tf32 split), exact FP64 rescreen  */
    LIP_TC_FP16 = 4    /* L2 only: tensor-core cross term (fp16 split), exact FP64 rescreen  */
    /* The tensor-core precisions need the L2 norm and no monotone coordinates (the squared
     * distance is then a cross product plus the two squared norms, which one more MMA adds).
     * TF32: each operand split into a TF32 head and an FP32 tail, three kind::tf32
     * products.  BF16: each operand split into three bf16 pieces, six kind::f16 products.
     * FP16: each operand scaled by a power of two (from the data's bounding box) and split
     * into two fp16 pieces, three kind::f16 products; a query farther than 2^14 / 2^7 times
     * the box's half-diagonal from its centre in some coordinate (outside the fp16 range)
     * goes to the fallback.  The returned bounds are the exact FP64 envelopes rounded once
     * (see the kernel's error bound); queries with too many near-ties go to a device-side
     * fallback (an FP32 screen of all points, then FP64 on the survivors) that gives the
     * same exact envelopes.  lip_eval does not synchronise on these handles either. */
} lip_precision;

/* Largest dimension d accepted by lip_fit / lip_reserve. */
#define LIP_D_MAX 32

/* Fitting parameters (Sec. 5, setparams(mon, a, b, w)).  All pointers are HOST pointers
 * that are read during the call only.
 *   norm       lip_norm of dist.
 *   precision  lip_precision of the evaluation.
 *   mon        d entries in {-1, 0, 1}: decreasing / unconstrained / increasing in that
 *              coordinate (Sec. 5, mon in {-1,0,1}^dim).  NULL = no monotonicity
 *              (the paper's model=0).
 *   w          d norm weights > 0: dist uses w_i (x_i - x^k_i).  NULL = all ones.  (These
 *              are weights of the norm; they are unrelated to the k-neighbour weights
 *              of Sec. 5 "Extra features".)                                              */
typedef struct lip_params {
    int32_t norm;
    int32_t precision;
    const int8_t* mon;
    const double* w;
} lip_params;

typedef struct lip_model* lip_handle;

/* ---------------------------------------------------------------- data (Sec. 5) */

/* Copy N data points into a new handle (Sec. 5: add() copies the data into GPU memory).
 *   X [N][d], y [N]: device arrays, read during the call's stream work only; the caller
 *   may reuse them once the stream has passed this call.
 *   M: Lipschitz constant (>= 0, finite) used by lip_eval until lip_set_M.
 * Errors: LIP_ERR_ARG (N < 1, N >= 2^31, d < 1, d > LIP_D_MAX, M < 0 or not finite,
 *   bad norm/precision/mon/w), LIP_ERR_UNSUPPORTED (tensor-core precision with a norm
 *   other than L2), LIP_ERR_NONFINITE (NaN/Inf in X or y; this is the only call that
 *   synchronises the stream, to read that check back), LIP_ERR_OOM, LIP_ERR_CUDA.
 * On error *out is NULL and nothing is leaked. */
LIP_API lip_status lip_fit(const void* X, const void* y, int64_t N, int32_t d, double M,
                   const lip_params* p, void* stream, lip_handle* out);

/* Same as lip_fit with X and y in host memory (copied to the device inside the call). */
LIP_API lip_status lip_fit_host(const void* X, const void* y, int64_t N, int32_t d, double M,
                        const lip_params* p, void* stream, lip_handle* out);

/* Empty handle with room for `capacity` points (Sec. 5: LipFit(reservedata, dim) reserves
 * space so that data can be added later without extra copies). */
LIP_API lip_status lip_reserve(int64_t capacity, int32_t d, double M, const lip_params* p,
                       lip_handle* out);

/* Append n points (device X [n][d], y [n]) after the current ones (Sec. 5: new data can
 * be added at any time and values() uses them).  Synchronises the stream to check the
 * new points are finite.  LIP_ERR_CAPACITY if N + n exceeds the capacity; the handle is
 * unchanged on any error. */
LIP_API lip_status lip_add(lip_handle h, const void* X, const void* y, int64_t n, void* stream);

/* lip_add with X and y in host memory. */
LIP_API lip_status lip_add_host(lip_handle h, const void* X, const void* y, int64_t n, void* stream);

/* lip_add / lip_add_host without waiting for the GPU: the finiteness check of the new
 * points runs on the device.  A point holding NaN or Inf is replaced on the device by a
 * copy of a finite point (the handle's first point if it already held data, else the
 * first finite new point, else x = 0, y = 0) so that no kernel reads a non-finite
 * datum, and the next lip_check returns LIP_ERR_NONFINITE; the results computed in
 * between are those of the data with the replaced points (lip_clear starts over).  The
 * points count as added either way.  Argument errors (LIP_ERR_ARG, LIP_ERR_CAPACITY)
 * are returned at once and leave the handle unchanged.  X and y must stay valid until the
 * stream has passed this call (for lip_add_host_async, pinned host memory keeps the copy
 * asynchronous). */
LIP_API lip_status lip_add_async(lip_handle h, const void* X, const void* y, int64_t n, void* stream);
LIP_API lip_status lip_add_host_async(lip_handle h, const void* X, const void* y, int64_t n, void* stream);

/* Remove every point (Sec. 5: clear()).  The capacity is kept. */
LIP_API lip_status lip_clear(lip_handle h, void* stream);

/* Number of points currently held, or -1 for a NULL handle. */
LIP_API int64_t lip_size(lip_handle h);

/* Change M (Sec. 5 passes the Lipschitz constant to each values() call).  Re-scales the
 * handle's internal copy on `stream`. */
LIP_API lip_status lip_set_M(lip_handle h, double M, void* stream);

/* ---------------------------------------------------------------- evaluation */

/* Evaluate the interpolant at nq query points (Sec. 5: values(query, LC, model, k=1)).
 *   Q [nq][d]         device, element type of the handle.
 *   g, lo, hi [nq]    device outputs (element type of the handle): g = (H_up + H_lo)/2,
 *                     lo = H_lo, hi = H_up.  Any of them may be NULL.
 *   idx_up, idx_lo    device int32 [nq]: the data index attaining H_up (argmin) and
 *                     H_lo (argmax), lowest index on exact ties.  May be NULL.
 * nq = 0 is a no-op.  A query with a NaN/Inf coordinate gives NaN outputs and index -1.
 * With a handle that holds no points (after lip_clear) every output is NaN / -1.
 * FP32 handles: the all-pairs scan runs in FP32, then the two selected data points are
 * re-evaluated in FP64, so lo/hi/g are exact up to the choice of index, which can only
 * differ from the exact one where two candidates are within FP32 rounding.
 * Errors: LIP_ERR_ARG, LIP_ERR_OOM (scratch growth), LIP_ERR_CUDA. */
LIP_API lip_status lip_eval(lip_handle h, const void* Q, int64_t nq, void* g, void* lo, void* hi,
                    int32_t* idx_up, int32_t* idx_lo, void* stream);

/* k > 1 neighbours (Sec. 5, "extra features" 2: values(query, LC, model, k) with the
 * neighbour weights of setparams).  Replaces the minimum and the maximum by weighted sums
 * of the k best bounds:
 *   H_up^k(q) = sum_j wk[j] v_(j),  v_(1) <= ... <= v_(k) the k smallest y^i + M dist_up(q, x^i),
 *   H_lo^k(q) = sum_j wk[j] v_[j],  v_[1] >= ... >= v_[k] the k largest  y^i - M dist_lo(q, x^i),
 *   g = (H_up^k + H_lo^k) / 2,  hi = H_up^k, lo = H_lo^k.
 * Equal values are ordered by data index.  1 <= k <= 8; wk: host array of k finite
 * weights >= 0 (the paper takes them to sum to 1; this is not enforced).
 * idx_up / idx_lo: device int32 [nq][k], the data indices in the order of the bounds.
 * Any output may be NULL.  Fewer than k data points (or a non-finite query) give NaN and
 * index -1.  The selection runs in the handle's scan precision (FP32 for FP32 and
 * tensor-core handles), the k selected bounds are re-evaluated in FP64. */
LIP_API lip_status lip_eval_k(lip_handle h, const void* Q, int64_t nq, int32_t k, const double* wk,
                              void* g, void* lo, void* hi, int32_t* idx_up, int32_t* idx_lo,
                              void* stream);

/* lip_eval with Q and the outputs in host memory: the queries are copied in, evaluated
 * and the results copied out in chunks (2^19 queries; 2^23 with the pruned scan, which
 * prunes better on all the queries at once), with copies overlapping the kernels of
 * other chunks.  Synchronises the stream before returning (the outputs are then valid). */
LIP_API lip_status lip_eval_host(lip_handle h, const void* Q, int64_t nq, void* g, void* lo, void* hi,
                         int32_t* idx_up, int32_t* idx_lo, void* stream);

/* lip_eval_host without the final synchronisation: returns once the copies (on the
 * handle's own copy stream) and the kernels (on `stream`) are queued.  Q and the outputs
 * must stay valid, and the outputs unread, until lip_check(h, stream) has returned (it
 * waits for the handle's copies); pinned host memory keeps the copies asynchronous.  The
 * copies of one handle's call overlap the kernels queued before it on `stream`, so calls
 * on several handles overlap one another's transfers and kernels.  The handle's next
 * host-path call reuses its staging buffers in order. */
LIP_API lip_status lip_eval_host_async(lip_handle h, const void* Q, int64_t nq, void* g, void* lo, void* hi,
                                       int32_t* idx_up, int32_t* idx_lo, void* stream);

/* Lipschitz constant of the data (Sec. 5: lipschitz_constant()): the maximum over pairs
 * i < j of |y^i - y^j| / dist(x^i, x^j) with the symmetric weighted norm of the handle
 * (monotonicity does not enter).  N^2/2 work and no pair matrix is stored (Sec. 5).
 * Pairs with dist = 0 and equal y are skipped; dist = 0 with different y gives +Inf.
 * The result is the FP64 definition's, exactly: each pair's ratio in plain IEEE double
 * arithmetic (|x^i_k - x^j_k| w_k per coordinate, summed / squared and summed / the
 * largest, the square root for L2, then |y^i - y^j| / dist), the largest of them, the
 * lowest (i, j) among equal values.  An FP32 screen finds the largest FP32 squared ratio
 * q*; every pair whose FP32 squared ratio reaches q* (1 - 2^-16) is re-evaluated in FP64
 * (the screen's relative error, (2d + 16) 2^-24 for FP32 data, keeps the exact maximum
 * among them).  Norm weights that are not powers of two multiply the FP32 coordinate
 * differences, so points a few FP32 units apart keep their exact difference.  FP64
 * handles screen the data rounded to FP32: pairs closer than FP32 resolution are outside
 * the bound there.
 * Outputs (host): *M_out, and the pair (*i_out < *j_out).  *i_out = *j_out = -1 with
 * *M_out = 0 only when no pair has a defined ratio: N < 2, or every pair is a repeated
 * point (dist = 0) with equal y.  Data at distinct points with constant y give M = 0 with
 * a real pair, the lowest (i, j) at positive distance.  Synchronises the stream. */
LIP_API lip_status lip_estimate_M(lip_handle h, double* M_out, int64_t* i_out, int64_t* j_out,
                          void* stream);

/* lip_estimate_M without the wait: queues the same computation on `stream` (the result's
 * 48 bytes are copied to pinned memory the handle owns) and returns; lip_estimate_M_result
 * waits for that copy and gives the result, the same as lip_estimate_M's bit for bit.  So
 * the estimates of several handles, each on its own stream, run side by side.  One estimate
 * per handle is outstanding: a second call (or lip_estimate_M) first waits for the copy of
 * the first and drops its result.  The data must stay unchanged until the result is read.
 * LIP_ERR_ARG for a NULL handle, LIP_ERR_OOM when the 64 pinned bytes cannot be had. */
LIP_API lip_status lip_estimate_M_async(lip_handle h, void* stream);

/* The result of the estimate lip_estimate_M_async queued on h (outputs as lip_estimate_M),
 * after waiting for it; lip_last_estimate_work then reports its work.  LIP_ERR_STATE when
 * none is outstanding (never queued, or already read), LIP_ERR_ARG for NULL pointers. */
LIP_API lip_status lip_estimate_M_result(lip_handle h, double* M_out, int64_t* i_out, int64_t* j_out);

/* Form of lip_estimate_M on this handle.  0 (the default): FP32 handles with d <= 8 and
 * N >= 32768 take the pruned form (below that the full screen is cheaper than the pruned
 * form's setup); 2: the pruned form wherever available (FP32, d <= 8); 1: always the full
 * kernel.  The pruned form puts the data in spatial order with a box and y range per
 * 16-point chunk and per 512-point tile, and its FP32 screen skips the tile pairs and
 * chunks whose exact FP32 upper bound (box gaps with the pair arithmetic's own operations,
 * rcp.approx with a 2^-18 margin) is below (1 - 2^-16) times the largest value already
 * found.  Other handles, and lip_estimate_M_part, screen all pairs.  Both forms are
 * followed by the same FP64 selection over the tile pairs whose screen maximum reaches
 * q* (1 - 2^-16), and give the same result bit for bit.  LIP_ERR_ARG for a NULL handle
 * or another value. */
LIP_API lip_status lip_set_estimate_full(lip_handle h, int32_t full);

/* ------------------------------------------------ several GPUs (one process per GPU) */
/* The paper computes every bound and the estimate as one reduction over all data (Sec. 5:
 * O(N) work per query, N^2 for the Lipschitz constant, no pair matrix); these calls split
 * that reduction across GPUs.  The collectives between them are the caller's (the Python
 * package uses torch.distributed, NCCL on GPUs); each call runs on this process's GPU.
 *
 * Data-sharded evaluation: rank r holds the contiguous slice of the data starting at
 * global index index_base_r in its own handle (same d, M, norm, mon, w and precision on
 * every rank).  Per call:
 *   1. lip_shard_scan       on every rank: packed keys key_up, key_lo [nq] (device int64);
 *   2. all-reduce MIN of key_up and key_lo over the ranks;
 *   3. lip_shard_reeval     on every rank: hi64, lo64 [nq] (device double);
 *   4. all-reduce MIN of hi64 and MAX of lo64 over the ranks;
 *   5. lip_shard_finish     on any rank that wants the outputs.
 * The results equal lip_eval's on one handle holding all the data, bit for bit (the keys
 * order the ranks' FP32 scan extrema exactly as lip_eval's split merge does, and the
 * winners are re-evaluated in FP64 by the rank that holds them).  FP32 and tensor-core
 * handles (the plain FP32 scan runs on either); LIP_ERR_UNSUPPORTED for FP64 handles. */

/* Step 1: the all-pairs scan of this rank's data.  key_up[q] (key_lo[q]) = (the FP32 scan's
 * smallest upper (largest lower) bound value v made order-preserving as an unsigned 32-bit
 * integer, of -v for the lower bound) << 31 | (index_base + local index of its datum), the
 * lowest index on ties; INT64_MAX when the handle holds no points or the query is not
 * finite.  The MIN over ranks of these keys is the single-GPU choice.
 *   Q [nq][d] device, handle element type; index_base >= 0 with index_base + capacity
 *   <= 2^31 (LIP_ERR_ARG otherwise).  Asynchronous on `stream`. */
LIP_API lip_status lip_shard_scan(lip_handle h, const void* Q, int64_t nq, int64_t index_base, int64_t* key_up,
                                  int64_t* key_lo, void* stream);

/* Step 3: for every query whose merged key names a datum of this rank (global index in
 * [index_base, index_base + N)), its exact FP64 bound y + M dist_up (hi64) and
 * y - M dist_lo (lo64), computed as lip_eval's merge does; +Inf (hi64) and -Inf (lo64)
 * for the others, the neutral values of step 4.  Asynchronous on `stream`. */
LIP_API lip_status lip_shard_reeval(lip_handle h, const void* Q, int64_t nq, int64_t index_base,
                                    const int64_t* key_up, const int64_t* key_lo, double* hi64, double* lo64,
                                    void* stream);

/* Step 5: g = (hi + lo) / 2 (in FP64, rounded once to the handle's element type), lo, hi
 * and the global indices idx_up, idx_lo from the merged keys and values; NaN and -1 where
 * a key is INT64_MAX.  Any output may be NULL.  Asynchronous on `stream`. */
LIP_API lip_status lip_shard_finish(lip_handle h, int64_t nq, const int64_t* key_up, const int64_t* key_lo,
                                    const double* hi64, const double* lo64, void* g, void* lo, void* hi,
                                    int32_t* idx_up, int32_t* idx_lo, void* stream);

/* The Lipschitz-constant estimate over one block-cyclic share of the pairs, for ranks that
 * all hold the same data: the N^2/2 pairs are cut into tile pairs (I, J >= I) of 512
 * points, and part p of nparts takes the tile pairs with (I * tiles + J) mod nparts = p.
 * out (host double[4]) = {M over the part's pairs (lip_estimate_M's exact FP64 selection
 * restricted to them), i, j, M again as the ordering key}, or {0, -1, -1, -1} when the
 * part has no pair with a defined ratio.  The estimate over all pairs is the part whose
 * key is largest, the lowest (i, j) on ties (lip_estimate_M's result, bit for bit).
 * 0 <= part < nparts, else LIP_ERR_ARG.  Synchronises the stream. */
LIP_API lip_status lip_estimate_M_part(lip_handle h, int32_t part, int32_t nparts, double* out, void* stream);

/* Largest N accepted by lip_estimate_M_noalloc. */
#define LIP_NOALLOC_N_MAX 32768

/* lip_estimate_M for callers that cannot allocate device memory.  The paper has no
 * counterpart; this is a convenience of this library.  It is meant for code that must
 * not call cudaMalloc: a plugin whose host application has already reserved the GPU's
 * memory in its own allocator, or a latency-bound loop that cannot absorb the
 * device-wide synchronisation cudaFree implies.  It needs no handle, allocates nothing,
 * and keeps its working memory in one fixed array of about 4.4 MB inside the library,
 * which every GPU that loads liblipfit.so holds until the process exits.
 *   X [N][d], y [N]  device, float, finite (not checked); read only.
 *   N                1 <= N <= LIP_NOALLOC_N_MAX, else LIP_ERR_ARG (fixed capacity).
 *   d, norm, w       as for lip_fit (w: host array of d weights > 0, or NULL).
 *   out              device double[3], written with {M_est, i, j} (i < j as doubles),
 *                    the definition, kernels and results of lip_estimate_M, including
 *                    its rule for -1 / -1 (no pair with a defined ratio).
 * The call is asynchronous on `stream` (it does not synchronise).  The first call on
 * each device looks up the array's device address (cudaGetSymbolAddress); make that
 * first call before any stream capture.  The address is kept per device and CUDA
 * context, so after a cudaDeviceReset the next call looks it up again in the new
 * context (that call, too, must come before any capture).  Every call on a device shares the one array,
 * which keeps the last call's contents (each call writes everything it later reads, so
 * nothing needs clearing): calls whose GPU work overlaps -- on different streams, or
 * from several host threads -- race and give wrong results, so order them on one
 * stream. */
LIP_API lip_status lip_estimate_M_noalloc(const float* X, const float* y, int64_t N, int32_t d,
                                          int32_t norm, const double* w, double* out, void* stream);

/* ------------------------------------------------ local Lipschitz constants (Sec. 4.3) */
/* compute_local_lipschitz() and values_local(query, model, k = 1) of Sec. 5.
 *
 * Every datum x^k gets a non-decreasing step function M_k(t) of the distance t from x^k,
 * and the bounds of Eq. (upperlower) use it in place of M:
 *   H_up(q) = min_k ( y^k + M_k(t_k) t_k ),  H_lo(q) = max_k ( y^k - M_k(t_k) t_k ),
 *   t_k = dist(q, x^k),  g = (H_up + H_lo) / 2.
 * M_k(t) = F_k for t <= d1_k, where d1_k is the distance to the nearest other datum and
 * F_k = |y^k - y^(1)| / d1_k (the largest such ratio over data tied at d1_k).  Beyond d1_k,
 * M_k(t) = Mtab_k[s] with s = #{i : T_i < t} and
 *   Mtab_k[s] = max( F_k, max { |y^k - y^j| / d_kj : 0 < d_kj <= T_{s+1} } ),  T_{m+1} = +inf:
 * the largest ratio over the data no farther than the next knot.  The knots T_1 < ... <
 * T_m are common to all data.  dist is the symmetric weighted norm of the handle
 * (|x_i - x'_i| w_i; L1, L2 or Linf).  Pairs at distance 0 are skipped.  The result
 * interpolates the data.
 * Handles with monotone coordinates (Sec. 5: values_local follows values()'s monotonicity
 * convention) use the one-sided distances of Sec. 4.1 Eq. (distmon): the upper bound takes
 * M_k(dist_up(q, x^k)) dist_up(q, x^k), the lower M_k(dist_lo(q, x^k)) dist_lo(q, x^k), and
 * datum k's table is built from the two events each other datum j gives it -- the distance
 * dist_up(x^j, x^k) with ratio (y^j - y^k)_+ / dist (what its upper bound needs to
 * interpolate x^j) and dist_lo(x^j, x^k) with (y^k - y^j)_+ / dist -- in place of the pairs
 * above (d1_k is the smallest positive event distance, F_k the largest ratio there); the
 * knots are quantiles of the sampled pairs' dist_up(x^a, x^b).  Data consistent with the
 * monotonicity are interpolated, and the envelopes are monotone in those coordinates.
 *
 * The table is exact: every distance and ratio that decides an entry is the IEEE double
 * result of the definition above (each operation rounded once, coordinates in order),
 * found by an FP32 screen with a rigorous error bound and FP64 re-computation of every
 * pair the bound cannot rule out.  Handles: any precision, with or without monotone
 * coordinates (FP64 handles: float or double arrays as for lip_eval).  Adding or clearing data invalidates
 * the table (LIP_ERR_STATE until the next fit).  N^2 work per fit: one screening scan that
 * lists, per datum, the pairs its running bounds cannot rule out (a second scan for the data
 * whose list overflows). */

/* Largest number of knots. */
#define LIP_LOCAL_KNOTS_MAX 31
/* Largest number of sampled pairs. */
#define LIP_LOCAL_SAMPLE_MAX (1 << 20)

/* Knots from a sample (Sec. 4.3: quantiles of the distribution of interpoint
 * distances, approximated from a sample).  sample_pairs pairs (a_s, b_s) are drawn with
 * SplitMix64 (Steele, Lea and Flood 2014): output c of the generator seeded with `seed`
 * is mix(seed + (c + 1) * 0x9E3779B97F4A7C15), a_s = out(2s) mod N, b_s = out(2s + 1) mod N.
 * Their positive distances, sorted, D_(1) <= ... <= D_(S'), give T_i = D_(ceil(i S' / nknots)),
 * i = 1..nknots, with repeated values dropped (so m <= nknots; m = 0 when S' = 0).
 * 0 <= nknots <= LIP_LOCAL_KNOTS_MAX, 0 <= sample_pairs <= LIP_LOCAL_SAMPLE_MAX.
 * Synchronises the stream.  Errors: LIP_ERR_ARG (ranges, no data), LIP_ERR_UNSUPPORTED,
 * LIP_ERR_OOM, LIP_ERR_CUDA. */
LIP_API lip_status lip_local_fit(lip_handle h, int32_t nknots, int64_t sample_pairs, uint64_t seed,
                                 void* stream);

/* The same with the caller's knots: host array of nknots finite values > 0, strictly
 * increasing (else LIP_ERR_ARG).  Synchronises the stream. */
LIP_API lip_status lip_local_fit_knots(lip_handle h, const double* knots, int32_t nknots, void* stream);

/* The knots in use (host array of at least LIP_LOCAL_KNOTS_MAX doubles; may be NULL) and
 * their number m.  LIP_ERR_STATE without a current table. */
LIP_API lip_status lip_local_knots(lip_handle h, double* knots, int32_t* nknots);

/* Copies the exact table to device double arrays (each may be NULL): d1 [N], F [N]
 * (d1 = +Inf and F = 0 for a datum without a neighbour at positive distance) and
 * Mtab [N][m + 1], row-major.  Ordered on the stream. */
LIP_API lip_status lip_local_table(lip_handle h, double* d1, double* F, double* Mtab, void* stream);

/* Statistics of the last table fit (each pointer may be NULL): the number of data whose
 * candidate list overflowed (their rows took the second scan) and the longest list that
 * did not.  Diagnostics only.  LIP_ERR_STATE without a current table. */
LIP_API lip_status lip_local_stats(lip_handle h, int32_t* overflow_rows, int32_t* max_candidates);

/* The envelopes with the local constants.  Arguments, outputs and NaN handling as for
 * lip_eval (element type of the handle, device).  The scan runs in FP32 and picks the winning data; their
 * bounds are then recomputed in FP64 with the exact table, so hi/lo are the exact values
 * of the selected data.  The selection can differ from the exact one where two values are
 * within FP32 rounding, or where a distance lies within FP32 rounding of one of the
 * datum's knots (M_k jumps there).  LIP_ERR_STATE without a current table. */
LIP_API lip_status lip_eval_local(lip_handle h, const void* Q, int64_t nq, void* g, void* lo, void* hi,
                                  int32_t* idx_up, int32_t* idx_lo, void* stream);

/* values_local(query, model, k) with k > 1 (Sec. 5): lip_eval_k's weighted sums of the k
 * best bounds, each bound with the local constant of its datum.  k, wk, the outputs (float,
 * device; idx_up / idx_lo [nq][k]) and the ordering of equal values as for lip_eval_k;
 * the k selected bounds are re-evaluated in FP64 with the exact table.  LIP_ERR_STATE
 * without a current table. */
LIP_API lip_status lip_eval_local_k(lip_handle h, const void* Q, int64_t nq, int32_t k, const double* wk,
                                    void* g, void* lo, void* hi, int32_t* idx_up, int32_t* idx_lo, void* stream);

/* ------------------------------------------------ penalty smoothing (Sec. 4.4) */
/* smooth_lipschitz(LC, model) of Sec. 5: changes eps to the data values minimising
 *
 *   Phi(eps) = (1/p) ||eps||^2
 *            + sum_{i != k} ((y_i - y_k - M d+_ik - (eps_k - eps_i))_+)^2      Eq. (const1)
 *            + sum_{i != k} ((y_k - y_i - M d-_ik + eps_k - eps_i)_+)^2        Eq. (const2)
 *
 * (Eq. (optim)), d+_ik = dist_up(x^i, x^k) and d-_ik = dist_lo(x^i, x^k) of the handle's
 * norm, weights and monotone coordinates (both the symmetric distance without them).
 * One evaluation is a fused pass over the N (N - 1) / 2 unordered pairs (each pair's two
 * terms at once) in FP32 with FP64 sums (in FP64 throughout on FP64 handles); nothing
 * pairwise is stored, and the terms owed to the second datum of a violating pair are summed
 * in 64-bit fixed point, so an evaluation is reproducible bit for bit.  Any handle with
 * N >= 1; M finite >= 0, p finite > 0. */

/* Phi and its gradient at eps (device double [N]): *f_out (host), grad (device double [N],
 * may be NULL).  Synchronises the stream. */
LIP_API lip_status lip_smooth_objective(lip_handle h, double M, double p, const double* eps, double* f_out,
                                        double* grad, void* stream);

/* Minimise Phi with L-BFGS from eps = 0 (Nocedal and Wright, Algorithms 7.4/7.5: history
 * pairs 1..64, backtracking Armijo line search from step 1), stopping when max |dPhi/deps|
 * <= gtol or after max_iter iterations.  Then, as the paper's package does, the handle's
 * values become y + eps (rounded to float) and its constant becomes M, so lip_eval
 * evaluates the smoothed interpolant at once (y + eps stays FP64 on FP64 handles); a local
 * Lipschitz table is invalidated.
 * eps_out (device double [N]) may be NULL; *f_out = Phi at the result, *iters_out = the
 * iterations taken, *evals_out = the objective evaluations (host, each may be NULL).  Synchronises the stream many times (the line
 * search reads Phi).  Errors: LIP_ERR_ARG, LIP_ERR_UNSUPPORTED, LIP_ERR_OOM, LIP_ERR_CUDA. */
LIP_API lip_status lip_smooth(lip_handle h, double M, double p, int32_t max_iter, int32_t history, double gtol,
                              double* eps_out, double* f_out, int32_t* iters_out, int32_t* evals_out,
                              void* stream);

/* ---------------------------------------------------------------- differentiation */

/* Gradient of L = sum_q grad_g[q] * g(q) through the saved argmin/argmax (g is piecewise
 * smooth and differentiable almost everywhere, Table 1):
 *   grad_Q [nq][d] (overwritten)   dL/dq  = M/2 (grad dist_up(q, x^u) - grad dist_lo(q, x^l))
 *   grad_y [N]     (ACCUMULATED)   dL/dy^k = 1/2 sum_q grad_g[q] ([u_q = k] + [l_q = k])
 *   grad_M [1]     (overwritten)   dL/dM  = 1/2 sum_q grad_g[q] (dist_up - dist_lo)
 * with the subgradient 0 at a zero distance and, for Linf, the lowest coordinate on a
 * tie of the maximum.  Q, idx_up, idx_lo are those given to / returned by lip_eval;
 * grad_g is [nq].  All device pointers; element type of the handle for Q, grad_g,
 * grad_Q, grad_y; grad_M is double.  Any of grad_Q, grad_y, grad_M may be NULL.
 * deterministic = 0: one kernel launch; grad_y receives atomic additions of the element
 * type, so its last bits may change with the order of the atomics.  deterministic != 0:
 * the contributions to grad_y are summed as 64-bit fixed point (scale 2^(60 - e) with
 * nq max|grad_g| / 2 < 2^e), which integer atomics add exactly in any order, and then added
 * to grad_y, so grad_y is bitwise reproducible (three launches).  grad_M uses a
 * fixed-order two-level reduction (finished by the last block) and is always bitwise
 * reproducible. */
LIP_API lip_status lip_backward(lip_handle h, const void* Q, int64_t nq, const int32_t* idx_up,
                        const int32_t* idx_lo, const void* grad_g, void* grad_Q, void* grad_y,
                        double* grad_M, int32_t deterministic, void* stream);

/* ---------------------------------------------------------------- many data sets */

/* One independent data set of a batch (Sec. 6: instance-based models with no training
 * phase; many small ones are evaluated at once).  Device pointers are the caller's;
 * X and y are copied by lip_batch_create, Q and the outputs are used by every
 * lip_batch_eval (so refill Q in place to evaluate new queries).
 *   X [N][d], y [N]   device float, 1 <= N < 2^31, 1 <= d <= LIP_D_MAX (sets with d <= 10
 *                     take the exact-shape bodies, wider ones a plain-load body).
 *   norm, M, mon, w   as for lip_fit (mon, w: host arrays of d entries, or NULL).
 *   Q [nq][d]         device float (nq may be 0).
 *   g, lo, hi [nq], idx_up, idx_lo [nq]   device outputs, each may be NULL.
 *   tile_groups       shared-memory tile of this set (8, 16, 32, 64; 0 = automatic). */
typedef struct lip_batch_set {
    const float* X;
    const float* y;
    int64_t N;
    int32_t d;
    int32_t norm;
    double M;
    const int8_t* mon;
    const double* w;
    const float* Q;
    int64_t nq;
    float* g;
    float* lo;
    float* hi;
    int32_t* idx_up;
    int32_t* idx_lo;
    int32_t tile_groups;
    int32_t reserved;
} lip_batch_set;

/* Launch-shape options of a batch (what the autotuner sets; results do not depend on it).
 *   tile_groups      tile for sets with N > 512 when the set gives none (0 = 32).
 *   items_per_block  work items per resident thread block that the data splitting aims
 *                    at (0 = 8): more items balance the tail, fewer cost less merging.
 *   waves            persistent grid = SMs x resident blocks per SM x waves (0 = 1). */
typedef struct lip_batch_options {
    int32_t tile_groups;
    int32_t items_per_block;
    int32_t waves;
    int32_t reserved;
} lip_batch_options;

typedef struct lip_batch_model* lip_batch;

/* Copy and transform every set (the lip_fit transform), cut the work into
 * (set, query block, data split) items sorted largest first, and allocate all scratch.
 * opt may be NULL.  Synchronises the stream once, to check that X and y are finite.
 * Errors: LIP_ERR_ARG (naming the first bad set), LIP_ERR_NONFINITE, LIP_ERR_OOM,
 * LIP_ERR_CUDA; on error *out is NULL. */
LIP_API lip_status lip_batch_create(const lip_batch_set* sets, int32_t nsets, const lip_batch_options* opt,
                                    void* stream, lip_batch* out);

/* Evaluate every set at its queries: one persistent scan launch over the work list, then
 * one merge launch that re-evaluates each query's two winners in FP64 and writes the
 * outputs.  Only enqueues a 4-byte memset and the two kernels on `stream`: no allocation
 * and no synchronisation.  Results equal lip_eval on each set. */
LIP_API lip_status lip_batch_eval(lip_batch b, void* stream);

/* The same call under the name of the batched evaluation in the design notes. */
LIP_API lip_status lip_eval_batched(lip_batch b, void* stream);

/* Sizes of a batch: sum over sets of nq * N, sum of nq, work items, persistent grid. */
LIP_API lip_status lip_batch_info(lip_batch b, double* total_pairs, int64_t* total_queries,
                                  int64_t* n_items, int32_t* grid);

/* Optional caller events recorded around the persistent scan kernel of every
 * lip_batch_eval (NULL, NULL turns this off), as lip_set_timing_events. */
LIP_API lip_status lip_batch_set_timing_events(lip_batch b, void* ev_before_scan, void* ev_after_scan);

/* Synchronise and report LIP_ERR_TIMEOUT if a bounded wait in the batched kernel gave up. */
LIP_API lip_status lip_batch_check(lip_batch b, void* stream);

LIP_API void lip_batch_free(lip_batch b);

/* ---------------------------------------------------------------- launch shape */

/* Launch shape of lip_eval on this handle (what the autotuner sets).  tile_groups, splits
 * and variants 0 / 1 do not change the results.
 *   tile_groups  groups of 4 data points staged per shared-memory tile: 8, 16, 32 or 64
 *                (0 keeps the current value).  Ignored by the generic kernel.
 *   splits       number of slices of the data scanned by separate thread blocks and
 *                merged afterwards; 0 = chosen per call to fill the GPU in whole waves.
 *   variant      scan kernel variant: 0 holds the default number of queries per thread,
 *                1 half as many (more resident warps); -1 keeps the current one.
 *                2 / 3 and 4 / 5 are 0 / 1 with one in eight (2, 3) or one in sixteen
 *                (4, 5) of the square roots of the L2 scans with monotone coordinates
 *                (two roots per pair, which load the special-function unit) computed on
 *                the FMA pipe (Lomont's seed and three Newton steps, a few ulps); their
 *                FP32 values differ in the last bits, so the selected index can differ
 *                where two bound values are that close (the bounds returned are the FP64
 *                values of the selected data either way); other shapes run 0 / 1.
 *                6 / 7 (FP32 handles, exact shapes with d <= 8): the pruned scan, with half /
 *                all of variant 0's queries per thread.  The data are kept in a spatial order
 *                with a bounding box and value range per 32-point chunk, the queries are put
 *                in spatial order per call, and a warp skips every chunk that provably cannot
 *                lower H_up or raise H_lo of any of its queries (the test repeats the pair
 *                arithmetic's FP32 operations on the box, so it is exact); the scan starts
 *                near the block's queries and runs over all the data in one split.  The
 *                extrema are those of the full scan; among data with exactly equal FP32
 *                values the one met first in that order is chosen (the returned bounds are
 *                its FP64 values).  Other shapes run 6 / 7 as 0 / 1.
 *                Ignored by the generic kernel.  For tensor-core handles (0 to 5): bit 0
 *                runs the tensor-core epilogue on 8 warps instead of 16; 0 / 1 run one
 *                persistent CTA per SM whose data sweeps keep a soft lockstep (the CTAs
 *                of a round read each data tile at about the same time, so it comes from
 *                L2), 2 / 3 the same without the lockstep, 4 / 5 one CTA per query tile;
 *                the results do not depend on the variant.  For LIP_FP64 handles: 0 (the
 *                default) scans a float copy of the layout and recomputes in FP64 only
 *                the pairs within the FP32 error bound of the extremum, 1 scans in FP64
 *                throughout (0 or 1); both return the FP64 envelopes.
 * LIP_ERR_ARG for other values. */
LIP_API lip_status lip_set_tuning(lip_handle h, int32_t tile_groups, int32_t splits, int32_t variant);

/* The library's own autotuner: times lip_eval on Q (device, nq >= 1) for every variant x
 * tile_groups {8, 16, 32, 64} x splits {0 (automatic), 1, 2, 3, 4, 6, 8, 12, 16} with CUDA
 * events on the stream (median of reps runs after one warm-up run), applies the fastest
 * with lip_set_tuning and returns it (host outputs, each may be NULL; *ms_out in ms).  The
 * results of lip_eval do not depend on the choice.  Allocates and frees its own output
 * buffers and synchronises the stream.  The Python package adds a JSON cache keyed by
 * shape (paper_2606_04670_b300/autotune.py). */
LIP_API lip_status lip_autotune(lip_handle h, const void* Q, int64_t nq, int32_t reps, int32_t* tile_groups_out,
                                int32_t* splits_out, int32_t* variant_out, double* ms_out, void* stream);

/* Current launch shape: tile_groups, the configured splits (0 = automatic), the splits
 * used by the last lip_eval, the queries held per thread by the scan kernel and the
 * variant.  Any output pointer may be NULL. */
LIP_API lip_status lip_get_tuning(lip_handle h, int32_t* tile_groups, int32_t* splits,
                                  int32_t* last_splits, int32_t* queries_per_thread, int32_t* variant);

/* ---------------------------------------------------------------- measurement */

/* Optional CUDA events (cudaEvent_t, created by the caller) that lip_eval records on its
 * stream immediately before and after its all-pairs scan kernel, so that the kernel can
 * be timed alone on the stream it runs on.  NULL, NULL turns this off. */
LIP_API lip_status lip_set_timing_events(lip_handle h, void* ev_before_scan, void* ev_after_scan);

/* After a pruned scan (lip_set_tuning variants 6 / 7): *evaluated = the (row, chunk)
 * pairs the last scan of this handle evaluated, *total = all its (row, chunk) pairs (rows
 * of 32 consecutive queries of the spatial order x 32-point chunks, each 1,024 query-point
 * pairs); *evaluated = *total = -1 when the last scan was not pruned.
 * Synchronises the device to read the count. */
LIP_API lip_status lip_last_scan_work(lip_handle h, int64_t* evaluated, int64_t* total);

/* The same and more (host int64[5]): out[0] evaluated and out[1] all (row, chunk) pairs as
 * lip_last_scan_work, out[2] the data tiles the blocks copied to shared memory, out[3]
 * blocks x data tiles, out[4] the (warp, chunk) pairs of the copied tiles that passed the
 * warp-box test (and went to the per-query tests); all -1 when the last scan was not
 * pruned.
 * Synchronises the device.  LIP_ERR_ARG for NULL. */
LIP_API lip_status lip_last_scan_stats(lip_handle h, int64_t* out);

/* After a pruned lip_estimate_M: out (host int64[3]) = the tile pairs that passed the tile
 * bound test, the (row, chunk) pairs the screen evaluated (a row holds 32 consecutive
 * points of the spatial order, a chunk 16 column points), and the total (row, chunk)
 * pairs of the tile triangle; all -1
 * when the last estimate of this handle did not take the pruned form.  Reads what the
 * estimate (which synchronises) left on the host.  LIP_ERR_ARG for NULL. */
LIP_API lip_status lip_last_estimate_work(lip_handle h, int64_t* out);

/* Tensor-core handles, variants 0 / 1 of lip_set_tuning: the data bytes over which the
 * persistent CTAs of one round may spread their sweeps of the data tiles (a producer runs
 * at most that far ahead of the slowest CTA of its round, and waits at most 2 ms for it).
 * Smaller windows keep the tiles a round reads in L2 for less DRAM traffic; larger ones let
 * the CTAs absorb differences in their speed.  0 (the default) selects 32 MB.  Ignored by
 * other handles and variants; the results do not depend on it.  LIP_ERR_ARG if bytes < 0. */
LIP_API lip_status lip_set_tc_window(lip_handle h, int64_t bytes);

/* Tensor-core handles (LIP_TC_*): number of queries of the last lip_eval whose candidate
 * lists overflowed (or, for LIP_TC_FP16, that lay outside the fp16 range) and were settled
 * by the device-side fallback (0 when the tensor-core form and its exact rescreen settled
 * every query, and for other handles); -1 for a NULL handle or a CUDA error.  The count
 * stays on the device during lip_eval: this call synchronises the device to read it. */
LIP_API int64_t lip_last_fallback(lip_handle h);

/* Number of kernels this library has launched in this process (all handles). */
LIP_API uint64_t lip_kernel_launches(void);

/* ---------------------------------------------------------------- status */

/* Synchronise the stream and report a failure recorded by the device since the last
 * lip_check on this handle (it also waits for lip_eval_host_async's copies):
 * LIP_ERR_TIMEOUT if a bounded wait inside a kernel gave up
 * (the kernel then skipped its work and returned), LIP_ERR_NONFINITE if a lip_add_async /
 * lip_add_host_async met NaN or Inf (TIMEOUT is reported first when both happened),
 * LIP_ERR_CUDA for a CUDA error.  The recorded failures are cleared. */
LIP_API lip_status lip_check(lip_handle h, void* stream);

LIP_API void lip_free(lip_handle h);

LIP_API const char* lip_status_string(lip_status s);

/* Copies the calling thread's last error message into buf (always NUL-terminated when
 * len > 0) and returns its full length. */
LIP_API size_t lip_last_error(char* buf, size_t len);

/* The same as lip_last_error. */
LIP_API size_t lip_last_error_detail(char* buf, size_t len);

/* Library version, e.g. "0.1.0 sm_103a". */
LIP_API const char* lip_version(void);

/* ---------------------------------------------------------------- fault injection (tests) */
/* The paper has no counterpart: these two calls let tests reach the library's failure
 * paths without a real device fault. */

/* Makes the n-th device allocation the library attempts from now on (counting from 1, on
 * any handle or thread) fail as if the device were out of memory: it returns
 * LIP_ERR_OOM through the usual path, without calling cudaMalloc.  n = 0 turns this off.
 * Allocations after the failing one succeed again.  LIP_ERR_ARG for n < 0. */
LIP_API lip_status lip_debug_fail_alloc(int64_t n);

/* The square root the exact scan's variants 2-5 compute on the FMA pipe (lip_set_tuning),
 * element by element: out[i] = sqrt(s[i]) for device float arrays of n entries (tests;
 * asynchronous on `stream`).  The paper has no counterpart. */
LIP_API lip_status lip_debug_sqrt_fma(const float* s, float* out, int64_t n, void* stream);

/* Fault injection for the exact FP32 scan kernel of handle h (FP32 handles whose shape has
 * an exact instantiation; other kernels ignore it):
 *   wait_limit_ns  limit of the kernel's bounded waits on its data tiles, in ns of the GPU's
 *                  global timer (0 = the default, 2 s; at most the default).
 *   skip_tile      every thread block leaves out the bulk copy of its data tile number
 *                  skip_tile (0 = its first), so its wait for that tile runs out: the block
 *                  records the timeout in the handle's status word, waits for the copies it
 *                  did issue, writes NaN / index -1 for its queries and returns.  lip_check
 *                  then reports LIP_ERR_TIMEOUT.  -1 = no tile left out.
 * The handle stays usable: lip_debug_scan_fault(h, 0, -1) restores normal evaluation.
 * LIP_ERR_ARG for a NULL handle, skip_tile < -1 or a limit above the default. */
LIP_API lip_status lip_debug_scan_fault(lip_handle h, uint64_t wait_limit_ns, int32_t skip_tile);

#ifdef __cplusplus
}
#endif
#endif /* LIPFIT_H */
