// Many independent data sets in one persistent launch (instance-based evaluation of
// many small models at once, Sec. 6): every set is fitted exactly as lip_fit does,
// the work is cut into (set, query block, data split) items, sorted largest first,
// and one persistent kernel pulls items from an atomic counter.  Each item runs the
// same scan body as lip_eval (scan_block), dispatched on the set's shape
// (norm, constrained, free coordinates).  A batched merge then re-evaluates every
// query's winners in FP64.  lip_batch_eval only enqueues a memset and two kernels,
// with no allocation and no synchronisation.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "launch.h"

namespace lip {
lip_status set_error(lip_status s, const char* msg);
cudaError_t dev_malloc(void** p, size_t bytes);
}

using namespace lip;

namespace {

constexpr int B_DMAX = 10;   // shapes with exact bodies: C + U <= 10

struct BatchItem {
    int32_t set, split;
    int64_t qblock;
};

struct BatchParams {
    const ScanParams* sets;     // [nsets], device
    const int32_t* shape;       // [nsets]: (norm - 1) * 121 + C * 11 + U
    const BatchItem* items;     // [n_items], largest first
    int64_t n_items;
    int* counter;
};

// Queries per thread of the batched bodies: all shapes share the kernel's register
// budget (128 at 4 resident blocks per SM), so wider shapes hold fewer queries.
__host__ __device__ constexpr int batch_rows(int D) { return D <= 4 ? 8 : (D <= 6 ? 4 : 2); }

template <int NORM, int C, int U>
__device__ __noinline__ void item_body(const ScanParams& P, int64_t qblock, int split, float4* tiles, uint64_t* bars,
                                       bool reinit) {
    scan_block<NORM, C, U, batch_rows(C + U)>(P, qblock, split, tiles, bars, reinit);
}

constexpr bool batch_shape_ok(int C, int U) { return C >= 0 && U >= 0 && C + U >= 1 && C + U <= B_DMAX; }

template <int K>
__device__ __forceinline__ bool try_body(int shape, const ScanParams& P, int64_t qb, int sp, float4* tiles,
                                         uint64_t* bars, bool reinit) {
    constexpr int NORM = K / 121 + 1, C = (K % 121) / 11, U = K % 11;
    if constexpr (batch_shape_ok(C, U)) {
        if (shape == K) {
            item_body<NORM, C, U>(P, qb, sp, tiles, bars, reinit);
            return true;
        }
    }
    return false;
}

template <int... K>
__device__ __forceinline__ void dispatch(int shape, const ScanParams& P, int64_t qb, int sp, float4* tiles,
                                         uint64_t* bars, bool reinit, std::integer_sequence<int, K...>) {
    (try_body<K>(shape, P, qb, sp, tiles, bars, reinit) || ...);
}

// Sets wider than the exact bodies (d = 11 .. LIP_D_MAX, any number of constrained
// coordinates): one query per thread against the set's layout (constrained coordinates
// first, mirrored and scaled; y after the d coordinates; the L1 auxiliary channel is not
// needed), read with plain loads, the index tracked per pair with strict comparisons (so
// the lowest index on ties), in the arithmetic of the generic scan kernel.
constexpr int WIDE_SHAPE0 = 3 * 121;       // shape ids WIDE_SHAPE0 + norm - 1
constexpr int WIDE_ROWS = 1;

template <int NORM>
__device__ __noinline__ void wide_item_body(const ScanParams& P, int64_t qblock, int split) {
    const int64_t qi = qblock * SCAN_THREADS + threadIdx.x;
    if (qi >= P.nq) return;
    const float* Q = static_cast<const float*>(P.Q);
    const float4* hot = static_cast<const float4*>(P.hot);
    float q[D_MAX];
#pragma unroll
    for (int j = 0; j < D_MAX; ++j) q[j] = j < P.d ? (float)(P.scale[j] * (double)Q[qi * P.d + P.perm[j]]) : 0.f;
    float mu = __int_as_float(0x7f800000), ml = -mu;
    int iu = -1, il = -1;
    const int64_t g0 = (int64_t)split * P.groups_per_split;
    const int64_t g1 = g0 + P.groups_per_split < P.ngroups ? g0 + P.groups_per_split : P.ngroups;
    for (int64_t g = g0; g < g1; ++g) {
        float au[4] = {0.f, 0.f, 0.f, 0.f}, al[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < D_MAX; ++j) {
            if (j >= P.dl) break;
            const float4 xv = hot[g * P.nch + j];
            const float xe[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float t = q[j] - xe[e];
                float u, l;
                if (j < P.C) { u = fmaxf(t, 0.f); l = fmaxf(-t, 0.f); }
                else { u = fabsf(t); l = u; }
                if (NORM == LIP_L1) { au[e] += u; al[e] += l; }
                else if (NORM == LIP_L2) { au[e] = fmaf(u, u, au[e]); al[e] = fmaf(l, l, al[e]); }
                else { au[e] = fmaxf(au[e], u); al[e] = fmaxf(al[e], l); }
            }
        }
        const float4 yv = hot[g * P.nch + P.dl];
        const float ye[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float du = NORM == LIP_L2 ? sqrtf(au[e]) : au[e];
            const float dl = NORM == LIP_L2 ? sqrtf(al[e]) : al[e];
            const float vu = ye[e] + du, vl = ye[e] - dl;      // NaN (padding) fails both tests
            const int k = (int)(g * GROUP + e);
            if (vu < mu) { mu = vu; iu = k; }
            if (vl > ml) { ml = vl; il = k; }
        }
    }
    static_cast<PartialRec<float>*>(P.partial)[(int64_t)split * P.nq + qi] = PartialRec<float>{mu, iu, ml, il};
}

__global__ void __launch_bounds__(SCAN_THREADS, 4) batch_scan_kernel(const BatchParams B) {
    extern __shared__ __align__(128) float4 tiles[];
    __shared__ __align__(8) uint64_t bars[SCAN_STAGES];
    __shared__ int64_t s_item;
    bool reinit = false;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(B.counter, 1);
        __syncthreads();
        const int64_t it = s_item;
        __syncthreads();
        if (it >= B.n_items) break;
        const BatchItem item = B.items[it];
        const int shape = B.shape[item.set];
        if (shape >= WIDE_SHAPE0) {
            if (shape == WIDE_SHAPE0) wide_item_body<LIP_L1>(B.sets[item.set], item.qblock, item.split);
            else if (shape == WIDE_SHAPE0 + 1) wide_item_body<LIP_L2>(B.sets[item.set], item.qblock, item.split);
            else wide_item_body<LIP_LINF>(B.sets[item.set], item.qblock, item.split);
        } else {
            dispatch(shape, B.sets[item.set], item.qblock, item.split, tiles, bars, reinit,
                     std::make_integer_sequence<int, 3 * 121>{});
            reinit = true;                 // the barriers have been initialised once
        }
        __syncthreads();
    }
}

__global__ void batch_merge_kernel(const MergeParams* mp, const int64_t* qprefix, int nsets, int64_t total_q) {
    const int64_t qg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (qg >= total_q) return;
    int lo = 0, hi = nsets - 1;   // last set with qprefix[set] <= qg
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (qprefix[mid] <= qg) lo = mid;
        else hi = mid - 1;
    }
    merge_one<float>(mp[lo], qg - qprefix[lo]);
}

// Algorithmic FP32 lane operations per pair of the survey's count, used to weigh items.
double pair_cost(int norm, int C, int U) {
    const int d = C + U;
    if (norm == LIP_L1) return 2.0 * (d - C) + 4.0 * C + 2 + 4;
    if (norm == LIP_L2) return 2.0 * (d - C) + 5.0 * C + 2 + 4 + (C > 0 ? 8.0 : 4.0);   // sqrt on MUFU
    return 2.0 * (d - C) + 3.0 * C + 2 + 4;
}

lip_status cfail(cudaError_t e, const char* what) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return set_error(LIP_ERR_OOM, buf);
    }
    return set_error(e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver ? LIP_ERR_NO_DEVICE : LIP_ERR_CUDA, buf);
}

#define B_TRY(expr)                                          \
    do {                                                     \
        cudaError_t e_ = (expr);                             \
        if (e_ != cudaSuccess) return cfail(e_, #expr);      \
    } while (0)

#define LIP_BATCH_TRY(expr)                                  \
    do {                                                     \
        lip_status s_ = (expr);                              \
        if (s_ != LIP_OK) return s_;                         \
    } while (0)

inline int64_t rup(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

struct lip_batch_model {
    int device = 0;
    int nsets = 0;
    int64_t total_q = 0;
    double total_pairs = 0;
    int64_t n_items = 0;
    int grid = 0;
    size_t smem = 0;
    std::vector<void*> allocs;
    ScanParams* d_sp = nullptr;
    MergeParams* d_mp = nullptr;
    int32_t* d_shape = nullptr;
    BatchItem* d_items = nullptr;
    int64_t* d_qprefix = nullptr;
    int* d_counter = nullptr;
    unsigned* d_status = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

static void batch_free(lip_batch_model* b) {
    if (!b) return;
    for (void* p : b->allocs) cudaFree(p);
    delete b;
}

static lip_status balloc(lip_batch_model* b, void** p, size_t n, const char* what) {
    cudaError_t e = dev_malloc(p, std::max<size_t>(n, 16));
    if (e != cudaSuccess) {
        *p = nullptr;
        return cfail(e, what);
    }
    b->allocs.push_back(*p);
    return LIP_OK;
}

static lip_status batch_create(const lip_batch_set* sets, int32_t nsets, const lip_batch_options* opt,
                               cudaStream_t st, lip_batch_model* b) {
    // ---- validation (host only, before any device work)
    char msg[256];
    for (int s = 0; s < nsets; ++s) {
        const lip_batch_set& x = sets[s];
        const char* bad = nullptr;
        if (x.N < 1 || x.N >= ((int64_t)1 << 31)) bad = "N outside [1, 2^31)";
        else if (x.d < 1 || x.d > D_MAX) bad = "d outside [1, LIP_D_MAX]";
        else if (x.norm < LIP_L1 || x.norm > LIP_LINF) bad = "norm is not L1/L2/Linf";
        else if (!(x.M >= 0.0) || !std::isfinite(x.M)) bad = "M must be finite and >= 0";
        else if (!x.X || !x.y) bad = "X or y is NULL";
        else if (x.nq < 0 || (x.nq > 0 && !x.Q)) bad = "nq < 0 or Q is NULL";
        else if (x.tile_groups != 0 && x.tile_groups != 8 && x.tile_groups != 16 && x.tile_groups != 32 &&
                 x.tile_groups != 64)
            bad = "tile_groups is not 0, 8, 16, 32 or 64";
        if (!bad && x.mon)
            for (int i = 0; i < x.d; ++i)
                if (x.mon[i] < -1 || x.mon[i] > 1) bad = "mon entries must be -1, 0 or 1";
        if (!bad && x.w)
            for (int i = 0; i < x.d; ++i)
                if (!(x.w[i] > 0.0) || !std::isfinite(x.w[i])) bad = "w entries must be finite and > 0";
        if (bad) {
            snprintf(msg, sizeof msg, "set %d: %s", s, bad);
            return set_error(LIP_ERR_ARG, msg);
        }
    }
    B_TRY(cudaGetDevice(&b->device));
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    b->nsets = nsets;

    // ---- per-set layout and sizes
    std::vector<ScanParams> sp(nsets);
    std::vector<MergeParams> mp(nsets);
    std::vector<int32_t> shape(nsets);
    std::vector<int64_t> x_off(nsets), y_off(nsets), hot_off(nsets), part_off(nsets), qprefix(nsets + 1, 0);
    std::vector<int> tg(nsets), rows(nsets), nch(nsets), aux(nsets), cset(nsets);
    std::vector<int64_t> ngroups(nsets);
    int64_t xs = 0, ys = 0, hs = 0;
    size_t smem = 0;
    for (int s = 0; s < nsets; ++s) {
        const lip_batch_set& x = sets[s];
        int C = 0;
        for (int i = 0; i < x.d; ++i) C += (x.mon && x.mon[i] != 0) ? 1 : 0;
        const int U = x.d - C;
        cset[s] = C;
        const bool wide = x.d > B_DMAX;
        shape[s] = wide ? WIDE_SHAPE0 + x.norm - 1 : (x.norm - 1) * 121 + C * 11 + U;
        aux[s] = (x.norm == LIP_L1 && C > 0) ? 1 : 0;
        nch[s] = x.d + 1 + aux[s];
        rows[s] = wide ? WIDE_ROWS : batch_rows(x.d);
        int t = x.tile_groups;
        if (t == 0) t = x.N <= 128 ? 8 : (x.N <= 512 ? 16 : (opt && opt->tile_groups ? opt->tile_groups : 32));
        tg[s] = t;
        ngroups[s] = rup(cdiv(x.N, GROUP), t);
        // the wide body reads its set with plain loads: no shared-memory tiles
        if (!wide) smem = std::max(smem, (size_t)SCAN_STAGES * t * nch[s] * sizeof(float4));
        x_off[s] = xs;
        xs += x.N * x.d;
        y_off[s] = ys;
        ys += x.N;
        hot_off[s] = hs;               // in float4 units
        hs += ngroups[s] * nch[s];
        qprefix[s + 1] = qprefix[s] + x.nq;
        b->total_pairs += (double)x.nq * (double)x.N;
    }
    b->total_q = qprefix[nsets];
    b->smem = smem;

    // ---- persistent grid: resident blocks per SM of the batched kernel
    if (smem > 48 * 1024)
        B_TRY(cudaFuncSetAttribute(batch_scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_scan_kernel, SCAN_THREADS, smem) != cudaSuccess ||
        occ < 1) {
        cudaGetLastError();
        occ = 1;
    }
    b->grid = sms * occ * (opt && opt->waves > 0 ? opt->waves : 1);

    // ---- work items: split large sets so that items stay well below the per-block share
    double weighted = 0;
    for (int s = 0; s < nsets; ++s) {
        const int C = cset[s], U = sets[s].d - C;
        weighted += (double)sets[s].nq * sets[s].N * pair_cost(sets[s].norm, C, U);
    }
    const int per_block = opt && opt->items_per_block > 0 ? opt->items_per_block : 8;
    const double target = std::max(1.0, weighted / ((double)b->grid * per_block));
    struct HostItem { double cost; BatchItem it; };
    std::vector<HostItem> hi;
    std::vector<int> nsplit(nsets);
    int64_t ps = 0;
    for (int s = 0; s < nsets; ++s) {
        const lip_batch_set& x = sets[s];
        const int C = cset[s], U = sets[s].d - C;
        const double pc = pair_cost(x.norm, C, U);
        const int64_t qb = (int64_t)SCAN_THREADS * rows[s];
        const int64_t tiles = ngroups[s] / tg[s];
        int64_t spl = (int64_t)std::ceil((double)std::min<int64_t>(qb, std::max<int64_t>(x.nq, 1)) * x.N * pc / target);
        spl = std::max<int64_t>(1, std::min(spl, tiles));
        const int64_t gps = rup(cdiv(ngroups[s], spl), tg[s]);
        spl = cdiv(ngroups[s], gps);
        nsplit[s] = (int)spl;
        part_off[s] = ps;
        ps += spl * x.nq;
        for (int64_t q = 0; q * qb < x.nq; ++q) {
            const int64_t nqb = std::min(qb, x.nq - q * qb);
            for (int64_t k = 0; k < spl; ++k) {
                const int64_t gk = std::min(gps, ngroups[s] - k * gps);
                hi.push_back({(double)nqb * gk * GROUP * pc, BatchItem{s, (int32_t)k, q}});
            }
        }
        ScanParams& P = sp[s];
        std::memset(&P, 0, sizeof P);
        P.wait_ns = WAIT_LIMIT_NS;
        P.skip_tile = -1;
        P.nq = x.nq;
        P.d = x.d;
        P.C = C;
        P.dl = x.d;
        P.nch = nch[s];
        int j = 0;
        for (int pass = 0; pass < 2; ++pass)
            for (int i = 0; i < x.d; ++i) {
                const int8_t m = x.mon ? x.mon[i] : 0;
                if ((pass == 0) != (m != 0)) continue;
                P.perm[j] = i;
                P.scale[j] = x.M * (m < 0 ? -1.0 : 1.0) * (x.w ? x.w[i] : 1.0);
                ++j;
            }
        P.Q = x.Q;
        P.ngroups = ngroups[s];
        P.groups_per_split = gps;
        P.tile_groups = tg[s];
        MergeParams& M = mp[s];
        std::memset(&M, 0, sizeof M);
        M.Q = x.Q;
        M.nq = x.nq;
        M.d = x.d;
        M.nsplit = (int)spl;
        M.M = x.M;
        M.norm = x.norm;
        for (int i = 0; i < x.d; ++i) {
            M.mon[i] = x.mon ? x.mon[i] : 0;
            M.w[i] = x.w ? x.w[i] : 1.0;
        }
        M.g = x.g;
        M.lo = x.lo;
        M.hi = x.hi;
        M.idx_up = x.idx_up;
        M.idx_lo = x.idx_lo;
    }
    std::stable_sort(hi.begin(), hi.end(), [](const HostItem& a, const HostItem& c) { return a.cost > c.cost; });
    std::vector<BatchItem> items(hi.size());
    for (size_t k = 0; k < hi.size(); ++k) items[k] = hi[k].it;
    b->n_items = (int64_t)items.size();

    // ---- device memory
    void *x0, *y0, *hot, *part;
    LIP_BATCH_TRY(balloc(b, &x0, (size_t)xs * 4, "batch data copy"));
    LIP_BATCH_TRY(balloc(b, &y0, (size_t)ys * 4, "batch value copy"));
    LIP_BATCH_TRY(balloc(b, &hot, (size_t)hs * 16, "batch scan layout"));
    LIP_BATCH_TRY(balloc(b, &part, (size_t)std::max<int64_t>(ps, 1) * sizeof(PartialRec<float>), "batch partials"));
    LIP_BATCH_TRY(balloc(b, (void**)&b->d_sp, nsets * sizeof(ScanParams), "batch set table"));
    LIP_BATCH_TRY(balloc(b, (void**)&b->d_mp, nsets * sizeof(MergeParams), "batch merge table"));
    LIP_BATCH_TRY(balloc(b, (void**)&b->d_shape, nsets * sizeof(int32_t), "batch shapes"));
    LIP_BATCH_TRY(balloc(b, (void**)&b->d_items, items.size() * sizeof(BatchItem), "batch work list"));
    LIP_BATCH_TRY(balloc(b, (void**)&b->d_qprefix, (nsets + 1) * sizeof(int64_t), "batch query offsets"));
    LIP_BATCH_TRY(balloc(b, (void**)&b->d_counter, sizeof(int), "batch counter"));
    LIP_BATCH_TRY(balloc(b, (void**)&b->d_status, 2 * sizeof(unsigned), "batch status"));
    B_TRY(cudaMemsetAsync(b->d_status, 0, 2 * sizeof(unsigned), st));

    // ---- copy and transform every set (the same kernels as lip_fit / lip_add)
    for (int s = 0; s < nsets; ++s) {
        const lip_batch_set& x = sets[s];
        float* xd = static_cast<float*>(x0) + x_off[s];
        float* yd = static_cast<float*>(y0) + y_off[s];
        float4* hd = static_cast<float4*>(hot) + hot_off[s];
        B_TRY(cudaMemcpyAsync(xd, x.X, (size_t)x.N * x.d * 4, cudaMemcpyDeviceToDevice, st));
        B_TRY(cudaMemcpyAsync(yd, x.y, (size_t)x.N * 4, cudaMemcpyDeviceToDevice, st));
        B_TRY(launch_pad_hot(4, hd, x.N, ngroups[s] * GROUP, nch[s], x.d, st));
        HotParams H;
        std::memset(&H, 0, sizeof H);
        H.X0 = xd;
        H.y0 = yd;
        H.k0 = 0;
        H.k1 = x.N;
        H.d = x.d;
        H.C = sp[s].C;
        H.dl = x.d;
        H.nch = nch[s];
        H.aux = aux[s];
        for (int j = 0; j < D_MAX; ++j) {
            H.perm[j] = sp[s].perm[j];
            H.scale[j] = sp[s].scale[j];
        }
        H.hot = hd;
        H.err = b->d_status + 1;
        B_TRY(launch_build_hot(4, H, st));
        sp[s].hot = hd;
        sp[s].partial = static_cast<PartialRec<float>*>(part) + part_off[s];
        sp[s].err = b->d_status;
        mp[s].X0 = xd;
        mp[s].y0 = yd;
        mp[s].partial = sp[s].partial;
    }
    B_TRY(cudaMemcpyAsync(b->d_sp, sp.data(), nsets * sizeof(ScanParams), cudaMemcpyHostToDevice, st));
    B_TRY(cudaMemcpyAsync(b->d_mp, mp.data(), nsets * sizeof(MergeParams), cudaMemcpyHostToDevice, st));
    B_TRY(cudaMemcpyAsync(b->d_shape, shape.data(), nsets * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    B_TRY(cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice, st));
    B_TRY(cudaMemcpyAsync(b->d_qprefix, qprefix.data(), (nsets + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    unsigned bad = 0;
    B_TRY(cudaMemcpyAsync(&bad, b->d_status + 1, sizeof bad, cudaMemcpyDeviceToHost, st));
    B_TRY(cudaStreamSynchronize(st));
    if (bad & ERRBIT_NONFINITE) return set_error(LIP_ERR_NONFINITE, "a set's X or y holds NaN or Inf");
    return LIP_OK;
}

extern "C" {

lip_status lip_batch_create(const lip_batch_set* sets, int32_t nsets, const lip_batch_options* opt, void* stream,
                            lip_batch* out) {
    if (!out) return set_error(LIP_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!sets || nsets < 1) return set_error(LIP_ERR_ARG, "sets is NULL or nsets < 1");
    if (opt && (opt->tile_groups != 0 && opt->tile_groups != 8 && opt->tile_groups != 16 && opt->tile_groups != 32 &&
                opt->tile_groups != 64))
        return set_error(LIP_ERR_ARG, "options: tile_groups is not 0, 8, 16, 32 or 64");
    if (opt && (opt->items_per_block < 0 || opt->items_per_block > 1024 || opt->waves < 0 || opt->waves > 64))
        return set_error(LIP_ERR_ARG, "options: items_per_block or waves out of range");
    lip_batch_model* b = new (std::nothrow) lip_batch_model();
    if (!b) return set_error(LIP_ERR_OOM, "host allocation failed");
    const lip_status s = batch_create(sets, nsets, opt, static_cast<cudaStream_t>(stream), b);
    if (s != LIP_OK) {
        batch_free(b);
        return s;
    }
    *out = b;
    return LIP_OK;
}

lip_status lip_batch_eval(lip_batch b, void* stream) {
    if (!b) return set_error(LIP_ERR_ARG, "batch is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    B_TRY(cudaMemsetAsync(b->d_counter, 0, sizeof(int), st));
    BatchParams P{b->d_sp, b->d_shape, b->d_items, b->n_items, b->d_counter};
    if (b->ev0) B_TRY(cudaEventRecord(b->ev0, st));
    batch_scan_kernel<<<b->grid, SCAN_THREADS, b->smem, st>>>(P);
    B_TRY(cudaGetLastError());
    if (b->ev1) B_TRY(cudaEventRecord(b->ev1, st));
    if (b->total_q > 0) {
        batch_merge_kernel<<<(unsigned)cdiv(b->total_q, 256), 256, 0, st>>>(b->d_mp, b->d_qprefix, b->nsets,
                                                                             b->total_q);
        B_TRY(cudaGetLastError());
    }
    return LIP_OK;
}

lip_status lip_batch_info(lip_batch b, double* total_pairs, int64_t* total_queries, int64_t* n_items,
                          int32_t* grid) {
    if (!b) return set_error(LIP_ERR_ARG, "batch is NULL");
    if (total_pairs) *total_pairs = b->total_pairs;
    if (total_queries) *total_queries = b->total_q;
    if (n_items) *n_items = b->n_items;
    if (grid) *grid = b->grid;
    return LIP_OK;
}

lip_status lip_batch_check(lip_batch b, void* stream) {
    if (!b) return set_error(LIP_ERR_ARG, "batch is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned bits = 0;
    B_TRY(cudaMemcpyAsync(&bits, b->d_status, sizeof bits, cudaMemcpyDeviceToHost, st));
    B_TRY(cudaStreamSynchronize(st));
    if (bits & ERRBIT_TIMEOUT) {
        B_TRY(cudaMemsetAsync(b->d_status, 0, sizeof bits, st));
        B_TRY(cudaStreamSynchronize(st));
        return set_error(LIP_ERR_TIMEOUT, "a bounded wait in the batched kernel gave up");
    }
    return LIP_OK;
}

lip_status lip_batch_set_timing_events(lip_batch b, void* ev_before_scan, void* ev_after_scan) {
    if (!b) return set_error(LIP_ERR_ARG, "batch is NULL");
    if ((ev_before_scan == nullptr) != (ev_after_scan == nullptr)) return set_error(LIP_ERR_ARG, "give both events or neither");
    b->ev0 = static_cast<cudaEvent_t>(ev_before_scan);
    b->ev1 = static_cast<cudaEvent_t>(ev_after_scan);
    return LIP_OK;
}

void lip_batch_free(lip_batch b) { batch_free(b); }

}  // extern "C"
