// C ABI of liblipfit (declared in include/lipfit.h): handles, validation, data, the
// envelope evaluation in every precision, the estimate, the backward pass, launch shapes
// and status.  Local constants are in api_local.cu, smoothing in api_smooth.cu.
#include "model.h"

namespace lip {

namespace {
thread_local std::string g_err;
std::atomic<uint64_t> g_launches{0};
}  // namespace

lip_status fail(lip_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

lip_status cuda_fail(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(LIP_ERR_OOM, "%s: out of device memory", what);
    }
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver)
        return fail(LIP_ERR_NO_DEVICE, "%s: %s", what, cudaGetErrorString(e));
    return fail(LIP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {
// > 0: the device allocation that brings this to 0 fails (lip_debug_fail_alloc)
std::atomic<int64_t> g_fail_alloc_countdown{0};
}  // namespace

cudaError_t dev_malloc(void** p, size_t bytes) {
    int64_t c = g_fail_alloc_countdown.load(std::memory_order_relaxed);
    while (c > 0 && !g_fail_alloc_countdown.compare_exchange_weak(c, c - 1, std::memory_order_relaxed)) {
    }
    if (c == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

// Records an error for lip_last_error from other translation units of the library.
lip_status set_error(lip_status s, const char* msg) { return fail(s, "%s", msg); }

uint64_t launches_total() { return g_launches.load(std::memory_order_relaxed); }

const std::string& last_error_text() { return g_err; }

}  // namespace lip

namespace lip {

lip_status check_params(int32_t d, double M, const lip_params* p) {
    if (!p) return fail(LIP_ERR_ARG, "params is NULL");
    if (d < 1 || d > D_MAX) return fail(LIP_ERR_ARG, "d = %d is outside [1, %d]", d, D_MAX);
    if (!(M >= 0.0) || !std::isfinite(M)) return fail(LIP_ERR_ARG, "M = %g must be finite and >= 0", M);
    if (p->norm < LIP_L1 || p->norm > LIP_LINF) return fail(LIP_ERR_ARG, "norm = %d is not L1/L2/Linf", p->norm);
    if (p->precision < LIP_FP32 || p->precision > LIP_TC_FP16)
        return fail(LIP_ERR_ARG, "precision = %d is not a lip_precision", p->precision);
    if (p->mon)
        for (int i = 0; i < d; ++i)
            if (p->mon[i] < -1 || p->mon[i] > 1) return fail(LIP_ERR_ARG, "mon[%d] = %d is not -1/0/1", i, p->mon[i]);
    if (p->w)
        for (int i = 0; i < d; ++i)
            if (!(p->w[i] > 0.0) || !std::isfinite(p->w[i]))
                return fail(LIP_ERR_ARG, "w[%d] = %g must be finite and > 0", i, p->w[i]);
    if (p->precision == LIP_TC_BF16 || p->precision == LIP_TC_TF32 || p->precision == LIP_TC_FP16) {
        if (p->norm != LIP_L2) return fail(LIP_ERR_UNSUPPORTED, "tensor-core precision needs the L2 norm");
        if (p->mon)
            for (int i = 0; i < d; ++i)
                if (p->mon[i] != 0)
                    return fail(LIP_ERR_UNSUPPORTED, "the tensor-core form needs the symmetric distance (no mon)");
    }
    return LIP_OK;
}

void fill_scan_params(const lip_model* h, ScanParams& P) {
    P.d = h->d;
    P.C = h->C;
    P.dl = h->dl;
    P.nch = h->nch;
    for (int j = 0; j < D_MAX; ++j) {
        P.perm[j] = h->perm[j];
        P.scale[j] = h->M * h->sgnw[j];
    }
    P.hot = h->hot;
    P.err = h->status;
    P.wait_ns = h->dbg_wait_ns ? h->dbg_wait_ns : WAIT_LIMIT_NS;
    P.skip_tile = h->dbg_skip_tile;
}

void fill_hot_params(const lip_model* h, HotParams& P, int64_t k0, int64_t k1) {
    P.X0 = h->X0;
    P.y0 = h->y0;
    P.k0 = k0;
    P.k1 = k1;
    P.d = h->d;
    P.C = h->C;
    P.dl = h->dl;
    P.nch = h->nch;
    P.aux = h->aux;
    for (int j = 0; j < D_MAX; ++j) {
        P.perm[j] = h->perm[j];
        P.scale[j] = h->M * h->sgnw[j];
    }
    P.hot = h->hot;
    P.err = h->status + 1;
}

void free_model(lip_model* h) {
    if (!h) return;
    DeviceGuard g(h->device);
    if (h->X0) cudaFree(h->X0);
    if (h->y0) cudaFree(h->y0);
    if (h->hot) cudaFree(h->hot);
    if (h->hot32) cudaFree(h->hot32);
    if (h->s32_max) cudaFree(h->s32_max);
    h->s64.release();
    if (h->status) cudaFree(h->status);
    h->partial.release();
    h->est.release();
    h->bwd.release();
    h->io.release();
    h->tc_q.release();
    h->sp_data.release();
    h->sp_q.release();
    h->tc_order.release();
    if (h->tc_btiles) cudaFree(h->tc_btiles);
    if (h->tc_maxbits) cudaFree(h->tc_maxbits);
    h->loc_buf.release();
    h->loc_tmp.release();
    h->sm_rec.release();
    h->sm_part.release();
    h->sm_vec.release();
    h->sm_small.release();
    if (h->loc_small) cudaFree(h->loc_small);
    for (int b = 0; b < 2; ++b) {
        if (h->ev_in[b]) cudaEventDestroy(h->ev_in[b]);
        if (h->ev_out[b]) cudaEventDestroy(h->ev_out[b]);
    }
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    if (h->est_done) {
        if (h->est_pending == 1) cudaEventSynchronize(h->est_done);   // the result's copy
        cudaEventDestroy(h->est_done);
    }
    if (h->est_back) cudaFreeHost(h->est_back);
    delete h;
}

lip_status create_model(int64_t cap, int32_t d, double M, const lip_params* p, cudaStream_t st, lip_model** out) {
    *out = nullptr;
    LIP_TRY(check_params(d, M, p));
    if (cap < 1 || cap >= (int64_t)1 << 31) return fail(LIP_ERR_ARG, "capacity %lld is outside [1, 2^31)", (long long)cap);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    lip_model* h = new (std::nothrow) lip_model();
    if (!h) return fail(LIP_ERR_OOM, "host allocation of the handle failed");
    h->device = dev;
    cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev);
    h->d = d;
    h->norm = p->norm;
    h->prec = p->precision;
    h->esize = p->precision == LIP_FP64 ? 8 : 4;
    h->M = M;
    // Layout coordinate order: constrained coordinates first, then the rest, each in
    // the caller's order; decreasing coordinates are mirrored (sign -1).
    int j = 0;
    for (int pass = 0; pass < 2; ++pass)
        for (int i = 0; i < d && i < D_MAX; ++i) {             // d <= D_MAX (checked above)
            const int8_t m = p->mon ? p->mon[i] : 0;
            if ((pass == 0) != (m != 0)) continue;
            h->perm[j] = i;
            h->sgnw[j] = (m < 0 ? -1.0 : 1.0) * (p->w ? p->w[i] : 1.0);
            ++j;
        }
    for (int i = 0; i < d && i < D_MAX; ++i) {
        h->mon[i] = p->mon ? p->mon[i] : 0;
        h->w[i] = p->w ? p->w[i] : 1.0;
        if (h->mon[i] != 0) h->C++;
    }
    const int U = d - h->C;
    h->tc = h->prec == LIP_TC_TF32 || h->prec == LIP_TC_BF16 || h->prec == LIP_TC_FP16;
    h->tc_fmt = h->prec == LIP_TC_BF16 ? TC_BF16 : (h->prec == LIP_TC_FP16 ? TC_FP16 : TC_TF32);
    if ((h->prec == LIP_FP32 || h->tc) && exact_shape_available(h->C, U)) {
        h->exact = true;
        h->dl = d;
        h->aux = (h->norm == LIP_L1 && h->C > 0) ? 1 : 0;
        h->nch = d + 1 + h->aux;
        h->kinfo = scan_exact_info(h->norm, h->C, U);
    } else {
        h->exact = false;
        h->dl = generic_dim(d);
        h->aux = 0;
        h->nch = h->dl + 1;
        h->kinfo = scan_generic_info(h->esize, h->norm, h->dl);
    }
    if (!h->kinfo.launch) {
        free_model(h);
        return fail(LIP_ERR_UNSUPPORTED, "no scan kernel for norm %d, %d constrained + %d free coordinates", p->norm, h->C, U);
    }
    const size_t smem = h->exact ? (size_t)SCAN_STAGES * h->tile_groups * h->nch * 16 : 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&h->occ_blocks, h->kinfo.kernel, SCAN_THREADS, smem) != cudaSuccess ||
        h->occ_blocks < 1) {
        cudaGetLastError();
        h->occ_blocks = 1;
    }
    if (h->esize == 8) {
        // the float layout of the FP32 screen: the FP32 handles' choice of kernel
        if (exact_shape_available(h->C, U)) {
            h->exact32 = true;
            h->dl32 = d;
            h->aux32 = (h->norm == LIP_L1 && h->C > 0) ? 1 : 0;
            h->nch32 = d + 1 + h->aux32;
            h->kinfo32 = scan_exact_info(h->norm, h->C, U);
        } else {
            h->dl32 = generic_dim(d);
            h->nch32 = h->dl32 + 1;
            h->kinfo32 = scan_generic_info(4, h->norm, h->dl32);
        }
        if (!h->kinfo32.launch) {
            free_model(h);
            return fail(LIP_ERR_UNSUPPORTED, "no FP32 screen kernel for norm %d, %d + %d coordinates", p->norm, h->C, U);
        }
        const size_t smem32 = h->exact32 ? (size_t)SCAN_STAGES * h->tile_groups * h->nch32 * 16 : 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&h->occ32, h->kinfo32.kernel, SCAN_THREADS, smem32) !=
                cudaSuccess || h->occ32 < 1) {
            cudaGetLastError();
            h->occ32 = 1;
        }
    }
    h->cap = cap;
    h->cap_pad = round_up(cap, PAD_POINTS);
    struct { void** p; size_t n; const char* what; } allocs[] = {
        {&h->X0, (size_t)cap * d * h->esize, "data copy"},
        {&h->y0, (size_t)cap * h->esize, "value copy"},
        {&h->hot, (size_t)h->cap_pad * h->nch * h->esize, "scan layout"},
        {reinterpret_cast<void**>(&h->status), 4 * sizeof(unsigned), "status word"},
    };
    for (auto& a : allocs) {
        e = dev_malloc(a.p, a.n);
        if (e != cudaSuccess) {
            *a.p = nullptr;
            free_model(h);
            return cuda_fail(e, a.what);
        }
    }
    if (h->tc) {
        h->tc_ntiles_cap = ceil_div(cap, 256);
        struct { void** p; size_t n; const char* what; } tca[] = {
            {reinterpret_cast<void**>(&h->tc_btiles), (size_t)h->tc_ntiles_cap * tc_tile_bytes_for(d, h->tc_fmt),
             "tensor-core data tiles"},
            {reinterpret_cast<void**>(&h->tc_maxbits), 2 * sizeof(unsigned), "tensor-core bounds"},
        };
        for (auto& a : tca) {
            e = dev_malloc(a.p, a.n);
            if (e != cudaSuccess) {
                *a.p = nullptr;
                free_model(h);
                return cuda_fail(e, a.what);
            }
        }
    }
    if (h->esize == 8) {
        struct { void** p; size_t n; const char* what; } s32[] = {
            {&h->hot32, (size_t)h->cap_pad * h->nch32 * 4, "float screen layout"},
            {reinterpret_cast<void**>(&h->s32_max), 2 * sizeof(unsigned), "screen bounds"},
        };
        for (auto& a : s32) {
            e = dev_malloc(a.p, a.n);
            if (e != cudaSuccess) {
                *a.p = nullptr;
                free_model(h);
                return cuda_fail(e, a.what);
            }
        }
    }
    e = cudaMemsetAsync(h->status, 0, 4 * sizeof(unsigned), st);
    if (e == cudaSuccess) e = launch_pad_hot(h->esize, h->hot, 0, h->cap_pad, h->nch, h->dl, st);
    count_launches(1);
    if (e != cudaSuccess) {
        free_model(h);
        return cuda_fail(e, "handle initialisation");
    }
    *out = h;
    return LIP_OK;
}

// Copy n points after the current ones and build their scan layout.  Synchronises to read
// the finiteness check back, unless `deferred`: then the check and the replacement of
// non-finite points run on the device (sanitize.cu) and lip_check reports them.
lip_status add_points(lip_model* h, const void* X, const void* y, int64_t n, cudaStream_t st, cudaMemcpyKind kind,
                      bool deferred = false) {
    if (n < 0) return fail(LIP_ERR_ARG, "n = %lld < 0", (long long)n);
    if (n == 0) return LIP_OK;
    if (!X || !y) return fail(LIP_ERR_ARG, "X or y is NULL");
    if (h->N + n > h->cap)
        return fail(LIP_ERR_CAPACITY, "%lld + %lld points exceed the capacity %lld", (long long)h->N, (long long)n,
                    (long long)h->cap);
    const size_t es = h->esize;
    CUDA_TRY(cudaMemcpyAsync(static_cast<char*>(h->X0) + (size_t)h->N * h->d * es, X, (size_t)n * h->d * es, kind, st));
    CUDA_TRY(cudaMemcpyAsync(static_cast<char*>(h->y0) + (size_t)h->N * es, y, (size_t)n * es, kind, st));
    if (deferred) {
        CUDA_TRY(launch_sanitize(h->esize, h->X0, h->y0, h->N, n, h->d, h->status, h->status + 2, st));
        count_launches(2);
    }
    CUDA_TRY(cudaMemsetAsync(h->status + 1, 0, sizeof(unsigned), st));
    HotParams P;
    fill_hot_params(h, P, h->N, h->N + n);
    CUDA_TRY(launch_build_hot(h->esize, P, st));
    count_launches(1);
    if (deferred) {                     // every new point is finite now
        h->N += n;
        h->tc_dirty = true;
        h->s32_dirty = true;
        h->sp_dirty = true;
        h->loc_valid = false;
        return LIP_OK;
    }
    unsigned bad = 0;
    CUDA_TRY(cudaMemcpyAsync(&bad, h->status + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (bad & ERRBIT_NONFINITE) {
        CUDA_TRY(launch_pad_hot(h->esize, h->hot, h->N, h->N + n, h->nch, h->dl, st));
        count_launches(1);
        CUDA_TRY(cudaStreamSynchronize(st));
        return fail(LIP_ERR_NONFINITE, "X or y holds NaN or Inf");
    }
    h->N += n;
    h->tc_dirty = true;
    h->s32_dirty = true;
    h->sp_dirty = true;
    h->loc_valid = false;
    return LIP_OK;
}

lip_status fit_common(const void* X, const void* y, int64_t N, int32_t d, double M, const lip_params* p, void* stream,
                      lip_handle* out, cudaMemcpyKind kind) {
    if (!out) return fail(LIP_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!X || !y) return fail(LIP_ERR_ARG, "X or y is NULL");
    if (N < 1 || N >= (int64_t)1 << 31) return fail(LIP_ERR_ARG, "N = %lld is outside [1, 2^31)", (long long)N);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    lip_model* h = nullptr;
    LIP_TRY(create_model(N, d, M, p, st, &h));
    DeviceGuard g(h->device);
    lip_status s = add_points(h, X, y, N, st, kind);
    if (s != LIP_OK) {
        free_model(h);
        return s;
    }
    *out = h;
    return LIP_OK;
}

// Number of N-splits: enough blocks to fill the GPU in nearly whole waves.
int choose_splits(const lip_model* h, int64_t gx, int64_t tiles) {
    if (h->splits > 0) return (int)std::max<int64_t>(1, std::min<int64_t>(h->splits, tiles));
    const int64_t wave = (int64_t)h->sms * h->occ_blocks;
    // up to 64 slices, more when a few query blocks could not fill a wave otherwise (the
    // tensor-core fallback's handful of queries)
    const int64_t cap = std::max<int64_t>(64, wave / std::max<int64_t>(gx, 1));
    const int64_t smax = std::max<int64_t>(1, std::min<int64_t>(cap, tiles / 2));
    int best = 1;
    double best_eff = 0.0;
    for (int64_t s = 1; s <= smax; ++s) {
        const int64_t blocks = gx * s;
        const double eff = (double)blocks / (double)(ceil_div(blocks, wave) * wave);
        if (eff > best_eff + 1e-9) { best_eff = eff; best = (int)s; }
        if (eff >= 0.9) break;
    }
    return best;
}

// The pruned scan (variants 6 / 7, scan_pruned.cuh): the data in spatial order with the
// chunk records (rebuilt lazily after the data or M change), the queries in spatial order,
// one launch over all the data (one split).
lip_status scan_partials_pruned(lip_model* h, const void* Q, int64_t nq, cudaStream_t st, int* nsplit_out) {
    const int64_t N = h->N;
    const int64_t npad = round_up(N, PAD_POINTS), ngroups = npad / GROUP, nchunks = ngroups / PRUNED_CG;
    const int D = h->dl;
    h->last_splits = ngroups > 0 ? 1 : 0;
    *nsplit_out = 0;
    if (ngroups == 0) return LIP_OK;
    const int64_t gx = ceil_div(nq, (int64_t)SCAN_THREADS * h->pinfo.rows);
    if (gx > 0x7fffffff) return fail(LIP_ERR_ARG, "nq = %lld is too large", (long long)nq);
    const int pnch = h->pinfo.nch;                   // the pruned layout: no aux channel
    const size_t perm_b = round_up(N * 4, 256), hot_b = round_up(ngroups * pnch * 16, 256),
                 box_b = round_up(nchunks * pruned_box_f4(D) * 16, 256), bnd_b = round_up(D_MAX * 8, 256),
                 cnt_b = 256, sbox_b = round_up(nchunks / PRUNED_CPS * pruned_box_f4(D) * 16, 256);
    LIP_TRY(h->sp_data.ensure(perm_b + hot_b + box_b + bnd_b + cnt_b + sbox_b + spatial_order_scratch(N),
                              "pruned scan data"));
    char* base = static_cast<char*>(h->sp_data.p);
    int* dperm = reinterpret_cast<int*>(base);
    void* shot = base + perm_b;
    void* box = base + perm_b + hot_b;
    float2* bounds = reinterpret_cast<float2*>(base + perm_b + hot_b + box_b);
    unsigned long long* work = reinterpret_cast<unsigned long long*>(base + perm_b + hot_b + box_b + bnd_b);
    void* sbox = base + perm_b + hot_b + box_b + bnd_b + cnt_b;
    void* oscratch = base + perm_b + hot_b + box_b + bnd_b + cnt_b + sbox_b;
    if (h->sp_dirty) {
        CUDA_TRY(spatial_order(static_cast<const float*>(h->X0), N, h->d, dperm, bounds, oscratch, st));
        HotParams Hp;
        fill_hot_params(h, Hp, 0, N);
        Hp.hot = shot;
        Hp.gather = dperm;
        Hp.nch = pnch;
        Hp.aux = 0;
        Hp.err = h->status + 3;                         // the data were checked when added
        CUDA_TRY(launch_build_hot(4, Hp, st));
        CUDA_TRY(launch_pad_hot(4, shot, N, npad, pnch, h->dl, st));
        CUDA_TRY(launch_pruned_boxes(shot, N, nchunks, D, pnch, false, box, sbox, st));
        count_launches(4 + spatial_order_launches());
        h->sp_dirty = false;
    }
    const size_t qp_b = round_up(nq * 4, 256);
    LIP_TRY(h->sp_q.ensure(qp_b + spatial_order_scratch(nq), "pruned scan query order"));
    int* qperm = static_cast<int*>(h->sp_q.p);
    CUDA_TRY(spatial_order(static_cast<const float*>(Q), nq, h->d, qperm, nullptr,
                           static_cast<char*>(h->sp_q.p) + qp_b, st));
    count_launches(spatial_order_launches());
    LIP_TRY(h->partial.ensure(std::max<size_t>(1, (size_t)nq * sizeof(PartialRec<float>)), "scan scratch"));
    PrunedParams PP{};
    fill_scan_params(h, PP.S);
    PP.S.Q = Q;
    PP.S.nq = nq;
    PP.S.hot = shot;
    PP.S.ngroups = ngroups;
    PP.S.groups_per_split = ngroups;
    PP.S.tile_groups = h->tile_groups;
    PP.S.partial = h->partial.p;
    PP.qperm = qperm;
    PP.dperm = dperm;
    PP.box = static_cast<const float4*>(box);
    PP.sbox = static_cast<const float4*>(sbox);
    PP.nchunks = nchunks;
    PP.work = work;
    CUDA_TRY(cudaMemsetAsync(work, 0, 3 * sizeof(unsigned long long), st));
    if (h->ev_scan0) CUDA_TRY(cudaEventRecord(h->ev_scan0, st));
    CUDA_TRY(h->pinfo.launch(PP, (int)gx, st));
    if (h->ev_scan1) CUDA_TRY(cudaEventRecord(h->ev_scan1, st));
    count_launches(1);
    h->sp_total = gx * (SCAN_THREADS / 32) * h->pinfo.rows * nchunks;   // (32-query row, 16-point chunk) pairs
    h->sp_tiles = gx * (ngroups / h->tile_groups);                       // blocks x tiles of the data
    *nsplit_out = 1;
    return LIP_OK;
}

// The all-pairs scan of the plain layout into per-split partial records (h->partial);
// *nsplit_out receives the number of splits (0 when the handle holds no points).
lip_status scan_partials(lip_model* h, const void* Q, int64_t nq, cudaStream_t st, int* nsplit_out) {
    if (h->pruned) return scan_partials_pruned(h, Q, nq, st, nsplit_out);
    h->sp_total = -1;
    const int64_t ngroups = round_up(h->N, PAD_POINTS) / GROUP;
    const int tg = h->exact ? h->tile_groups : 1;
    const int64_t gx = ceil_div(nq, (int64_t)SCAN_THREADS * h->kinfo.rows);
    int nsplit = 0;
    int64_t gps = 0;
    if (ngroups > 0) {
        const int64_t tiles = ngroups / (h->exact ? tg : TILE_GROUPS_MAX);
        const int s = choose_splits(h, gx, tiles);
        const int64_t unit = h->exact ? tg : TILE_GROUPS_MAX;
        gps = round_up(ceil_div(ngroups, s), unit);
        nsplit = (int)ceil_div(ngroups, gps);
    }
    h->last_splits = nsplit;
    if (gx > 0x7fffffff) return fail(LIP_ERR_ARG, "nq = %lld is too large", (long long)nq);
    const size_t rec = h->esize == 8 ? sizeof(PartialRec<double>) : sizeof(PartialRec<float>);
    LIP_TRY(h->partial.ensure(std::max<size_t>(1, (size_t)nsplit * nq * rec), "scan scratch"));
    if (nsplit > 0) {
        ScanParams P;
        fill_scan_params(h, P);
        P.Q = Q;
        P.nq = nq;
        P.ngroups = ngroups;
        P.groups_per_split = gps;
        P.tile_groups = tg;
        P.partial = h->partial.p;
        if (h->ev_scan0) CUDA_TRY(cudaEventRecord(h->ev_scan0, st));
        CUDA_TRY(h->kinfo.launch(P, (int)gx, nsplit, st));
        if (h->ev_scan1) CUDA_TRY(cudaEventRecord(h->ev_scan1, st));
        count_launches(1);
    }
    *nsplit_out = nsplit;
    return LIP_OK;
}

// The handle's parameters of the FP64 re-evaluation (split merge and shard re-evaluation).
void fill_merge_params(const lip_model* h, const void* Q, int64_t nq, MergeParams& Mp) {
    Mp.Q = Q;
    Mp.nq = nq;
    Mp.d = h->d;
    Mp.M = h->M;
    Mp.norm = h->norm;
    for (int i = 0; i < D_MAX; ++i) {
        Mp.mon[i] = h->mon[i];
        Mp.w[i] = h->w[i];
    }
    Mp.X0 = h->X0;
    Mp.y0 = h->y0;
}

lip_status eval_plain(lip_model* h, const void* Q, int64_t nq, void* g, void* lo, void* hi, int32_t* iu, int32_t* il,
                      cudaStream_t st) {
    int nsplit = 0;
    LIP_TRY(scan_partials(h, Q, nq, st, &nsplit));
    MergeParams Mp;
    Mp.Q = Q;
    Mp.nq = nq;
    Mp.d = h->d;
    Mp.nsplit = nsplit;
    Mp.M = h->M;
    Mp.norm = h->norm;
    for (int i = 0; i < D_MAX; ++i) {
        Mp.mon[i] = h->mon[i];
        Mp.w[i] = h->w[i];
    }
    Mp.X0 = h->X0;
    Mp.y0 = h->y0;
    Mp.partial = h->partial.p;
    Mp.g = g;
    Mp.lo = lo;
    Mp.hi = hi;
    Mp.idx_up = iu;
    Mp.idx_lo = il;
    CUDA_TRY(launch_merge(h->esize, Mp, st));
    count_launches(1);
    return LIP_OK;
}

// Tensor-core form: prepare the data tiles if the data or M changed, then build the
// query tiles, scan on the tensor cores, rescreen candidates in FP64, and settle the
// queries whose candidate lists overflowed with the device-side fallback passes (their
// count stays on the device: no synchronisation).
lip_status eval_tc(lip_model* h, const void* Q, int64_t nq, void* g, void* lo, void* hi, int32_t* iu, int32_t* il,
                   cudaStream_t st) {
    const int d = h->d;
    double scale[D_MAX];
    for (int j = 0; j < D_MAX; ++j) scale[j] = j < d ? h->M * h->w[j] : 0.0;
    const int64_t ntiles = ceil_div(h->N, 256);
    // the data's spatial order and its position-ordered copies (kept with the handle)
    const size_t p_b = round_up(h->N * 4, 256), x_b = round_up(h->N * d * 4, 256), y_b = round_up(h->N * 4, 256),
                 b_b = round_up(D_MAX * 8, 256);
    LIP_TRY(h->tc_order.ensure(p_b + x_b + y_b + b_b + spatial_order_scratch(h->N), "tensor-core data order"));
    char* ob = static_cast<char*>(h->tc_order.p);
    TcDataOrder O{};
    O.dperm = reinterpret_cast<int*>(ob);
    O.Xs = reinterpret_cast<float*>(ob + p_b);
    O.ys = reinterpret_cast<float*>(ob + p_b + x_b);
    O.bounds = reinterpret_cast<float2*>(ob + p_b + x_b + y_b);
    O.scratch = ob + p_b + x_b + y_b + b_b;
    if (h->tc_dirty) {
        CUDA_TRY(tc_prepare_data(static_cast<const float*>(h->X0), static_cast<const float*>(h->y0), h->N, d, scale,
                                 h->tc_maxbits, h->tc_btiles, ntiles, h->tc_fmt, O, st));
        count_launches(2 + spatial_order_launches());
        h->tc_dirty = false;
    }
    const int64_t nqt = ceil_div(nq, 128);
    const size_t a_b = round_up((int64_t)(nqt * tc_a_bytes_for(d, h->tc_fmt)), 256), eps_b = round_up(nq * 16, 256),
                 rec_b = round_up((int64_t)(nq * tc_rec_bytes()), 256), list_b = round_up(nq * 4 + 4, 256),
                 qp_b = round_up(nq * 4, 256), fb_b = round_up((int64_t)tc_fallback_state_bytes(nq), 256),
                 ar_b = round_up((int64_t)tc_arrive_bytes(nq, ntiles), 256);
    h->tc_fb_count = nullptr;
    LIP_TRY(h->tc_q.ensure(a_b + eps_b + rec_b + list_b + qp_b + fb_b + ar_b + spatial_order_scratch(nq),
                           "tensor-core query scratch"));
    char* base = static_cast<char*>(h->tc_q.p);
    int* fb_list = reinterpret_cast<int*>(base + a_b + eps_b + rec_b);
    int* fb_count = fb_list + nq;
    TcQueryOrder QO{};
    QO.qperm = reinterpret_cast<int*>(base + a_b + eps_b + rec_b + list_b);
    void* fb_state = base + a_b + eps_b + rec_b + list_b + qp_b;
    int* arrive = reinterpret_cast<int*>(base + a_b + eps_b + rec_b + list_b + qp_b + fb_b);
    QO.scratch = base + a_b + eps_b + rec_b + list_b + qp_b + fb_b + ar_b;
    CUDA_TRY(tc_eval_launch(static_cast<const float*>(Q), nq, d, scale, h->N, h->tc_maxbits, h->tc_btiles,
                            ntiles, base, reinterpret_cast<float4*>(base + a_b), base + a_b + eps_b, h->w, h->M,
                            static_cast<const float*>(h->X0), static_cast<const float*>(h->y0), static_cast<float*>(g),
                            static_cast<float*>(lo), static_cast<float*>(hi), iu, il, fb_count, fb_list, fb_state,
                            arrive, h->tc_window, h->status, h->tc_variant, h->tc_fmt, O, QO, h->ev_scan0, h->ev_scan1, st));
    count_launches(7 + spatial_order_launches());
    h->tc_fb_count = fb_count;          // read back by lip_last_fallback only
    return LIP_OK;
}

// FP64 handles: the FP32 screen (float copy of the layout, the FP32 kernels), then the
// candidate pass with FP64 values, then the usual merge (screen64.cu).
lip_status eval_screen64(lip_model* h, const void* Q, int64_t nq, void* g, void* lo, void* hi, int32_t* iu,
                         int32_t* il, cudaStream_t st) {
    const int64_t npad = round_up(h->N, PAD_POINTS);
    if (h->s32_dirty) {
        HotParams Hp;
        fill_hot_params(h, Hp, 0, h->N);
        Hp.hot = h->hot32;
        Hp.dl = h->dl32;
        Hp.nch = h->nch32;
        Hp.aux = h->aux32;
        CUDA_TRY(cudaMemsetAsync(h->s32_max, 0, 2 * sizeof(unsigned), st));
        CUDA_TRY(launch_build_hot32(Hp, h->s32_max, st));
        CUDA_TRY(launch_pad_hot(4, h->hot32, h->N, npad, h->nch32, h->dl32, st));
        count_launches(2);
        h->s32_dirty = false;
    }
    const int64_t ngroups = npad / GROUP;
    const int tg = h->exact32 ? h->tile_groups : 1;
    const int64_t gx = ceil_div(nq, (int64_t)SCAN_THREADS * h->kinfo32.rows);
    const int64_t gx2 = ceil_div(nq, (int64_t)screen64_threads());
    if (gx > 0x7fffffff || gx2 > 0x7fffffff) return fail(LIP_ERR_ARG, "nq = %lld is too large", (long long)nq);
    int nsplit = 0, nsplit2 = 0;
    int64_t gps = 0, gps2 = 0;
    if (ngroups > 0) {
        const int64_t unit = h->exact32 ? tg : TILE_GROUPS_MAX;
        const int s = choose_splits(h, gx, ngroups / unit);
        gps = round_up(ceil_div(ngroups, s), unit);
        nsplit = (int)ceil_div(ngroups, gps);
        // the candidate pass reads groups straight from global memory, so its splits can be
        // as small as 8 groups (32 points): small query counts still fill the GPU
        const int s2 = choose_splits(h, gx2, ngroups / 8);
        gps2 = round_up(ceil_div(ngroups, s2), 8);
        nsplit2 = (int)ceil_div(ngroups, gps2);
    }
    h->last_splits = nsplit;
    const size_t q_b = round_up(nq * h->d * 4, 256), p1_b = round_up((int64_t)std::max(nsplit, 1) * nq * 16, 256);
    LIP_TRY(h->s64.ensure(q_b + p1_b, "FP64 screen scratch"));
    LIP_TRY(h->partial.ensure(std::max<size_t>(1, (size_t)nsplit2 * nq * sizeof(PartialRec<double>)), "scan scratch"));
    float* q32 = static_cast<float*>(h->s64.p);
    PartialRec<float>* p1 = reinterpret_cast<PartialRec<float>*>(static_cast<char*>(h->s64.p) + q_b);
    if (h->ev_scan0) CUDA_TRY(cudaEventRecord(h->ev_scan0, st));
    if (nsplit > 0) {
        CUDA_TRY(launch_to_float(static_cast<const double*>(Q), nq * h->d, q32, st));
        ScanParams P;
        fill_scan_params(h, P);
        P.dl = h->dl32;
        P.nch = h->nch32;
        P.hot = h->hot32;
        P.Q = q32;
        P.nq = nq;
        P.ngroups = ngroups;
        P.groups_per_split = gps;
        P.tile_groups = tg;
        P.partial = p1;
        CUDA_TRY(h->kinfo32.launch(P, (int)gx, nsplit, st));
        Screen64Params S{};
        S.Q = static_cast<const double*>(Q);
        S.nq = nq;
        S.C = h->C;
        S.dl = h->dl32;
        S.nch = h->nch32;
        for (int j = 0; j < D_MAX; ++j) {
            S.perm[j] = h->perm[j];
            S.scale[j] = h->M * h->sgnw[j];
        }
        S.hot32 = h->hot32;
        S.ngroups = ngroups;
        S.groups_per_split = gps2;
        S.nsplit1 = nsplit;
        S.partial1 = p1;
        S.maxbits = h->s32_max;
        S.M.d = h->d;
        S.M.M = h->M;
        S.M.norm = h->norm;
        for (int i = 0; i < D_MAX; ++i) {
            S.M.mon[i] = h->mon[i];
            S.M.w[i] = h->w[i];
        }
        S.M.X0 = h->X0;
        S.M.y0 = h->y0;
        S.partial2 = static_cast<PartialRec<double>*>(h->partial.p);
        CUDA_TRY(launch_screen64(h->norm, S, (int)gx2, nsplit2, st));
        count_launches(3);
    }
    if (h->ev_scan1) CUDA_TRY(cudaEventRecord(h->ev_scan1, st));
    MergeParams Mp;
    Mp.Q = Q;
    Mp.nq = nq;
    Mp.d = h->d;
    Mp.nsplit = nsplit > 0 ? nsplit2 : 0;
    Mp.M = h->M;
    Mp.norm = h->norm;
    for (int i = 0; i < D_MAX; ++i) {
        Mp.mon[i] = h->mon[i];
        Mp.w[i] = h->w[i];
    }
    Mp.X0 = h->X0;
    Mp.y0 = h->y0;
    Mp.partial = h->partial.p;
    Mp.g = g;
    Mp.lo = lo;
    Mp.hi = hi;
    Mp.idx_up = iu;
    Mp.idx_lo = il;
    CUDA_TRY(launch_merge(8, Mp, st));
    count_launches(1);
    return LIP_OK;
}

// The estimate over the tile pairs of block-cyclic part `part` of nparts (all pairs for
// 0 of 1): res = {M_est, i, j, M_est again as the key that orders parts (-1 without a
// pair)}, the FP64 definition's maximum over those pairs and its lowest (i, j).
// Synchronises the stream.
// lip_estimate_M on one GPU, FP32 handles with d <= 8 (estimate_pruned.cu): the estimate
// layout in spatial order with chunk and tile records, then the three pruned passes (the
// FP32 maximum, the FP64 maximum over the pairs near it, the lowest pair attaining it);
// the FP64 definition's result exactly.
lip_status estimate_pruned(lip_model* h, double* res, cudaStream_t st, bool wait) {
    const int tile = estimate_tile_points();
    const int64_t N = h->N, nb = ceil_div(N, tile), pts = nb * tile, nchunks = pts / 16;   // 16-point chunks
    const int64_t npairs = nb * (nb + 1) / 2;
    const int d = h->d, nch = d + 1;
    const size_t rec = (size_t)pruned_box_f4(d) * 16;
    const size_t lay_b = round_up(pts * nch * 4, 256), perm_b = round_up(N * 4, 256),
                 cbox_b = round_up((int64_t)(nchunks * rec), 256), tbox_b = round_up((int64_t)(nb * rec), 256),
                 bnd_b = round_up(D_MAX * 8, 256), pair_b = round_up(npairs * 4, 256), small_b = 256;
    LIP_TRY(h->est.ensure(lay_b + perm_b + cbox_b + tbox_b + bnd_b + 2 * pair_b + small_b + spatial_order_scratch(N),
                          "estimate scratch"));
    char* base = static_cast<char*>(h->est.p);
    char* at = base;
    auto take = [&](size_t bytes) { char* p = at; at += bytes; return p; };
    void* lay = take(lay_b);
    int* perm = reinterpret_cast<int*>(take(perm_b));
    void* cbox = take(cbox_b);
    void* tbox = take(tbox_b);
    float2* bounds = reinterpret_cast<float2*>(take(bnd_b));
    float* bq = reinterpret_cast<float*>(take(pair_b));
    unsigned* list = reinterpret_cast<unsigned*>(take(pair_b));
    // small: gbest at 0, the selection's words at 64, out (4 doubles) at 128, work (2) at 160
    char* small = take(small_b);
    int* gbest = reinterpret_cast<int*>(small);
    EstExactState* state = reinterpret_cast<EstExactState*>(small + 64);
    double* out = reinterpret_cast<double*>(small + 128);
    unsigned long long* work = reinterpret_cast<unsigned long long*>(small + 160);
    void* oscratch = at;
    // The pruned scan's position order of the same data (built by the same deterministic
    // spatial_order, so identical) is reused while the data are unchanged.
    const bool reuse = h->sp_data.p && !h->sp_dirty;
    if (reuse) perm = static_cast<int*>(h->sp_data.p);
    else CUDA_TRY(spatial_order(static_cast<const float*>(h->X0), N, d, perm, bounds, oscratch, st));
    HotParams Hp;
    Hp.X0 = h->X0;
    Hp.y0 = h->y0;
    Hp.k0 = 0;
    Hp.k1 = N;
    Hp.d = d;
    Hp.C = 0;
    Hp.dl = d;
    Hp.nch = nch;
    Hp.aux = 0;
    const bool weighted = est_weighted(h->w, d);
    for (int j = 0; j < D_MAX; ++j) {
        Hp.perm[j] = j;
        Hp.scale[j] = est_layout_scale(h->w, j, weighted);
    }
    Hp.hot = lay;
    Hp.err = h->status + 3;
    Hp.gather = perm;
    CUDA_TRY(launch_estimate_layout(4, Hp, st));
    CUDA_TRY(launch_pad_hot(4, lay, N, pts, nch, d, st));
    CUDA_TRY(launch_chunk_records(lay, N, nchunks, d, nch, false, cbox, st, 16));
    CUDA_TRY(launch_record_union(cbox, nb, tile / 16, d, tbox, st));
    CUDA_TRY(cudaMemsetAsync(small, 0, small_b, st));          // the selection's words, out, work
    CUDA_TRY(cudaMemsetAsync(gbest, 0xff, 4, st));             // no value yet
    EstPrunedParams P;
    P.lay = static_cast<const float4*>(lay);
    P.N = N;
    P.nb = (int)nb;
    P.cbox = static_cast<const float4*>(cbox);
    P.tbox = static_cast<const float4*>(tbox);
    P.gbest = gbest;
    P.bq = bq;
    P.weighted = weighted;
    for (int j = 0; j < d; ++j) P.w[j] = (float)h->w[j];
    P.work = work;
    CUDA_TRY(launch_estimate_pruned(h->norm, d, P, st));
    EstFinalParams F;
    F.cand = nullptr;
    F.nb = (int)nb;
    F.X0 = h->X0;
    F.y0 = h->y0;
    F.d = d;
    F.norm = h->norm;
    F.elem_bytes = h->esize;
    for (int j = 0; j < D_MAX; ++j) F.w[j] = h->w[j];
    F.out = out;
    F.write_key = 1;
    F.lay = P.lay;
    F.N = N;
    F.weighted = weighted;
    F.perm = perm;
    F.list = list;
    F.state = state;
    CUDA_TRY(launch_estimate_pruned_select(P, F, st));
    CUDA_TRY(launch_estimate_exact(F, st));
    count_launches(6 + ESTIMATE_EXACT_LAUNCHES + (reuse ? 0 : spatial_order_launches()));
    const int64_t total = npairs * (tile / 32) * (tile / 16);    // 32-point rows x 16-point chunks
    if (!wait) {                                                  // lip_estimate_M_async
        CUDA_TRY(cudaMemcpyAsync(h->est_back, out, 48, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaEventRecord(h->est_done, st));
        h->est_pending = 1;
        h->est_pending_total = total;
        return LIP_OK;
    }
    // the result (4 doubles) and the work counters in one read
    unsigned char back[48];
    CUDA_TRY(cudaMemcpyAsync(back, out, sizeof back, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    memcpy(res, back, 4 * sizeof(double));
    unsigned long long wk[2];
    memcpy(wk, back + 32, sizeof wk);
    h->est_work[0] = (int64_t)wk[0];
    h->est_work[1] = (int64_t)wk[1];
    h->est_work[2] = total;
    return LIP_OK;
}

// With wait = false (lip_estimate_M_async, part 0 of 1) the result is left to
// estimate_collect: est_pending becomes 1 when device work was queued, and stays 0 when
// res already holds the result (fewer than two points).
lip_status estimate_part(lip_model* h, int part, int nparts, double* res, cudaStream_t st, bool wait) {
    DeviceGuard gd(h->device);
    for (int k = 0; k < 3; ++k) h->est_work[k] = -1;
    res[0] = 0.0;
    res[1] = res[2] = -1.0;
    res[3] = -1.0;
    if (h->N < 2) return LIP_OK;
    const int tile = estimate_tile_points();
    const int64_t nb = ceil_div(h->N, tile);
    if (nb > 65535) return fail(LIP_ERR_UNSUPPORTED, "N = %lld is too large for lip_estimate_M", (long long)h->N);
    // Below 32,768 points the full screen's N^2 work is a few tens of microseconds and the
    // pruned form's spatial order and records (a dozen launches) cost more than they save.
    const bool pruned = h->est_form == 2 || (h->est_form == 0 && h->N >= 32768);
    if (nparts == 1 && h->esize == 4 && estimate_pruned_available(h->d) && pruned)
        return estimate_pruned(h, res, st, wait);
    const int64_t pts = nb * tile;
    const int nch = h->d + 1;
    const size_t lay_b = round_up(pts * nch * 4, 256), cand_b = round_up(nb * nb * 16, 256),
                 list_b = round_up(nb * nb * 4, 256);
    LIP_TRY(h->est.ensure(lay_b + cand_b + 256 + list_b, "estimate scratch"));
    char* base = static_cast<char*>(h->est.p);
    // FP32 layout in the caller's order: coordinates times est_layout_scale
    const bool weighted = est_weighted(h->w, h->d);
    HotParams Hp;
    Hp.X0 = h->X0;
    Hp.y0 = h->y0;
    Hp.k0 = 0;
    Hp.k1 = h->N;
    Hp.d = h->d;
    Hp.C = 0;
    Hp.dl = h->d;
    Hp.nch = nch;
    Hp.aux = 0;
    for (int j = 0; j < D_MAX; ++j) {
        Hp.perm[j] = j;
        Hp.scale[j] = est_layout_scale(h->w, j, weighted);
    }
    Hp.hot = base;
    Hp.err = h->status + 1;
    CUDA_TRY(launch_estimate_layout(h->esize, Hp, st));
    CUDA_TRY(launch_pad_hot(4, base, h->N, pts, nch, h->d, st));
    EstParams P;
    P.lay = reinterpret_cast<const float4*>(base);
    P.N = h->N;
    P.nb = (int)nb;
    P.cand = reinterpret_cast<float4*>(base + lay_b);
    P.part = part;
    P.nparts = nparts;
    P.weighted = weighted;
    for (int j = 0; j < h->d; ++j) P.w[j] = (float)h->w[j];
    CUDA_TRY(launch_estimate(h->norm, h->d, P, st));
    EstFinalParams F;
    F.cand = P.cand;
    F.nb = (int)nb;
    F.X0 = h->X0;
    F.y0 = h->y0;
    F.d = h->d;
    F.norm = h->norm;
    F.elem_bytes = h->esize;
    for (int j = 0; j < D_MAX; ++j) F.w[j] = h->w[j];
    F.out = reinterpret_cast<double*>(base + lay_b + cand_b);
    F.part = part;
    F.nparts = nparts;
    F.write_key = 1;
    F.lay = P.lay;
    F.N = h->N;
    F.weighted = weighted;
    F.state = reinterpret_cast<EstExactState*>(base + lay_b + cand_b + 64);
    F.list = reinterpret_cast<unsigned*>(base + lay_b + cand_b + 256);
    CUDA_TRY(launch_estimate_final(F, st));
    count_launches(3 + ESTIMATE_FINAL_LAUNCHES);
    if (!wait) {
        CUDA_TRY(cudaMemcpyAsync(h->est_back, F.out, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaEventRecord(h->est_done, st));
        h->est_pending = 1;
        h->est_pending_total = -1;
        return LIP_OK;
    }
    CUDA_TRY(cudaMemcpyAsync(res, F.out, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return LIP_OK;
}

// The result of the estimate lip_estimate_M_async queued: waits for its copy.
lip_status estimate_collect(lip_model* h, double* res) {
    if (h->est_pending == 0) return fail(LIP_ERR_STATE, "no estimate queued on this handle");
    if (h->est_pending == 2) {
        memcpy(res, h->est_host_res, 4 * sizeof(double));
    } else {
        const cudaError_t e = cudaEventSynchronize(h->est_done);
        if (e != cudaSuccess) {
            h->est_pending = 0;
            return cuda_fail(e, "cudaEventSynchronize (estimate)");
        }
        memcpy(res, h->est_back, 4 * sizeof(double));
        if (h->est_pending_total >= 0) {
            unsigned long long wk[2];
            memcpy(wk, h->est_back + 32, sizeof wk);
            h->est_work[0] = (int64_t)wk[0];
            h->est_work[1] = (int64_t)wk[1];
            h->est_work[2] = h->est_pending_total;
        }
    }
    h->est_pending = 0;
    return LIP_OK;
}

lip_status eval_device(lip_model* h, const void* Q, int64_t nq, void* g, void* lo, void* hi, int32_t* iu, int32_t* il,
                       cudaStream_t st) {
    if (h->tc) return eval_tc(h, Q, nq, g, lo, hi, iu, il, st);
    if (h->esize == 8 && h->fp64_mode == 0) return eval_screen64(h, Q, nq, g, lo, hi, iu, il, st);
    return eval_plain(h, Q, nq, g, lo, hi, iu, il, st);
}

}  // namespace lip

extern "C" {

lip_status lip_fit(const void* X, const void* y, int64_t N, int32_t d, double M, const lip_params* p, void* stream,
                   lip_handle* out) {
    return fit_common(X, y, N, d, M, p, stream, out, cudaMemcpyDeviceToDevice);
}

lip_status lip_fit_host(const void* X, const void* y, int64_t N, int32_t d, double M, const lip_params* p, void* stream,
                        lip_handle* out) {
    return fit_common(X, y, N, d, M, p, stream, out, cudaMemcpyHostToDevice);
}

lip_status lip_reserve(int64_t capacity, int32_t d, double M, const lip_params* p, lip_handle* out) {
    if (!out) return fail(LIP_ERR_ARG, "out is NULL");
    *out = nullptr;
    lip_model* h = nullptr;
    LIP_TRY(create_model(capacity, d, M, p, nullptr, &h));
    cudaError_t e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) {
        free_model(h);
        return cuda_fail(e, "lip_reserve");
    }
    *out = h;
    return LIP_OK;
}

lip_status lip_add(lip_handle h, const void* X, const void* y, int64_t n, void* stream) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    DeviceGuard g(h->device);
    return add_points(h, X, y, n, static_cast<cudaStream_t>(stream), cudaMemcpyDeviceToDevice);
}

lip_status lip_add_host(lip_handle h, const void* X, const void* y, int64_t n, void* stream) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    DeviceGuard g(h->device);
    return add_points(h, X, y, n, static_cast<cudaStream_t>(stream), cudaMemcpyHostToDevice);
}

lip_status lip_add_async(lip_handle h, const void* X, const void* y, int64_t n, void* stream) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    DeviceGuard g(h->device);
    return add_points(h, X, y, n, static_cast<cudaStream_t>(stream), cudaMemcpyDeviceToDevice, true);
}

lip_status lip_add_host_async(lip_handle h, const void* X, const void* y, int64_t n, void* stream) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    DeviceGuard g(h->device);
    return add_points(h, X, y, n, static_cast<cudaStream_t>(stream), cudaMemcpyHostToDevice, true);
}

lip_status lip_clear(lip_handle h, void* stream) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    DeviceGuard g(h->device);
    CUDA_TRY(launch_pad_hot(h->esize, h->hot, 0, round_up(h->N, PAD_POINTS), h->nch, h->dl, static_cast<cudaStream_t>(stream)));
    count_launches(1);
    h->N = 0;
    h->tc_dirty = true;
    h->s32_dirty = true;
    h->sp_dirty = true;
    h->loc_valid = false;
    return LIP_OK;
}

int64_t lip_size(lip_handle h) { return h ? h->N : -1; }

lip_status lip_set_M(lip_handle h, double M, void* stream) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (!(M >= 0.0) || !std::isfinite(M)) return fail(LIP_ERR_ARG, "M = %g must be finite and >= 0", M);
    DeviceGuard g(h->device);
    h->M = M;
    h->tc_dirty = true;
    h->s32_dirty = true;
    h->sp_dirty = true;
    HotParams P;
    fill_hot_params(h, P, 0, h->N);
    CUDA_TRY(launch_build_hot(h->esize, P, static_cast<cudaStream_t>(stream)));
    count_launches(1);
    return LIP_OK;
}

lip_status lip_eval(lip_handle h, const void* Q, int64_t nq, void* g, void* lo, void* hi, int32_t* idx_up,
                    int32_t* idx_lo, void* stream) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (nq < 0) return fail(LIP_ERR_ARG, "nq = %lld < 0", (long long)nq);
    if (nq == 0) return LIP_OK;
    if (!Q) return fail(LIP_ERR_ARG, "Q is NULL");
    DeviceGuard gd(h->device);
    return eval_device(h, Q, nq, g, lo, hi, idx_up, idx_lo, static_cast<cudaStream_t>(stream));
}

lip_status lip_eval_k(lip_handle h, const void* Q, int64_t nq, int32_t k, const double* wk, void* g, void* lo,
                      void* hi, int32_t* idx_up, int32_t* idx_lo, void* stream) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (nq < 0) return fail(LIP_ERR_ARG, "nq = %lld < 0", (long long)nq);
    if (k < 1 || k > 8) return fail(LIP_ERR_ARG, "k = %d is outside [1, 8]", k);
    if (!wk) return fail(LIP_ERR_ARG, "wk is NULL");
    for (int e = 0; e < k; ++e)
        if (!(wk[e] >= 0.0) || !std::isfinite(wk[e])) return fail(LIP_ERR_ARG, "wk[%d] = %g must be finite and >= 0", e, wk[e]);
    if (nq == 0) return LIP_OK;
    if (!Q) return fail(LIP_ERR_ARG, "Q is NULL");
    DeviceGuard gd(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int K = k <= 2 ? 2 : (k <= 4 ? 4 : 8);
    const int64_t ngroups = round_up(h->N, PAD_POINTS) / GROUP;
    const int64_t gx = ceil_div(nq, (int64_t)topk_threads());
    if (gx > 0x7fffffff) return fail(LIP_ERR_ARG, "nq = %lld is too large", (long long)nq);
    int nsplit = 0;
    int64_t gps = 0;
    if (ngroups > 0) {
        const int64_t want = std::max<int64_t>(1, ceil_div((int64_t)4 * h->sms * 4, gx));
        const int64_t s = std::min<int64_t>(std::min<int64_t>(want, 64), std::max<int64_t>(1, ngroups / 16));
        gps = ceil_div(ngroups, s);
        nsplit = (int)ceil_div(ngroups, gps);
    }
    LIP_TRY(h->partial.ensure(std::max<size_t>(1, (size_t)nsplit * nq * 2 * K * (h->esize + 4)), "k-neighbour scratch"));
    TopkParams P{};
    P.Q = Q;
    P.nq = nq;
    P.d = h->d;
    P.C = h->C;
    P.dl = h->dl;
    P.nch = h->nch;
    for (int j = 0; j < D_MAX; ++j) {
        P.perm[j] = h->perm[j];
        P.scale[j] = h->M * h->sgnw[j];
    }
    P.hot = h->hot;
    P.ngroups = ngroups;
    P.groups_per_split = gps;
    P.partial = h->partial.p;
    TopkMergeParams Mp{};
    Mp.Q = Q;
    Mp.nq = nq;
    Mp.d = h->d;
    Mp.k = k;
    Mp.K = K;
    Mp.nsplit = nsplit;
    Mp.norm = h->norm;
    Mp.M = h->M;
    for (int i = 0; i < D_MAX; ++i) {
        Mp.mon[i] = h->mon[i];
        Mp.w[i] = h->w[i];
    }
    for (int e = 0; e < 8; ++e) Mp.wk[e] = e < k ? wk[e] : 0.0;
    Mp.X0 = h->X0;
    Mp.y0 = h->y0;
    Mp.partial = h->partial.p;
    Mp.g = g;
    Mp.lo = lo;
    Mp.hi = hi;
    Mp.idx_up = idx_up;
    Mp.idx_lo = idx_lo;
    CUDA_TRY(launch_topk(h->esize, h->norm, K, P, (int)gx, nsplit, Mp, st));
    count_launches(nsplit > 0 ? 2 : 1);
    return LIP_OK;
}

// The host path.  With wait, both streams are synchronised before returning.  Without,
// the call returns once everything is queued: the kernels on the caller's stream, the
// copies on the handle's copy stream, which needs no wait on the caller's stream (the
// staging buffers are reused only by this path, whose copies are ordered on that stream
// and whose kernels wait for their inputs' copies); lip_check waits for the copies.
static lip_status eval_host(lip_handle h, const void* Q, int64_t nq, void* g, void* lo, void* hi, int32_t* idx_up,
                            int32_t* idx_lo, void* stream, bool wait) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (nq < 0) return fail(LIP_ERR_ARG, "nq = %lld < 0", (long long)nq);
    if (nq == 0) return LIP_OK;
    if (!Q) return fail(LIP_ERR_ARG, "Q is NULL");
    DeviceGuard gd(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!h->copy_stream) {
        CUDA_TRY(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
        for (int b = 0; b < 2; ++b) {
            CUDA_TRY(cudaEventCreateWithFlags(&h->ev_in[b], cudaEventDisableTiming));
            CUDA_TRY(cudaEventCreateWithFlags(&h->ev_out[b], cudaEventDisableTiming));
        }
    }
    const size_t es = h->esize;
    // Chunks of 2^19 queries overlap the copies with the kernels.  The pruned scan orders
    // its queries in space and prunes per row of 32 neighbours, so it loses far more on a
    // chunk (sparser queries, looser rows) than the overlap gains: it takes up to 2^23 at once.
    const int64_t chunk = std::min<int64_t>(nq, (int64_t)1 << (h->pruned && !h->tc ? 23 : 19));
    // per buffer: Q chunk, g, lo, hi, idx_up, idx_lo
    const size_t qb = round_up((int64_t)(chunk * h->d * es), 256), vb = round_up((int64_t)(chunk * es), 256),
                 ib = round_up((int64_t)(chunk * 4), 256);
    const size_t per = qb + 3 * vb + 2 * ib;
    LIP_TRY(h->io.ensure(2 * per, "host-path staging"));
    char* base = static_cast<char*>(h->io.p);
    auto dQ = [&](int b) { return base + b * per; };
    auto dV = [&](int b, int k) { return base + b * per + qb + k * vb; };
    auto dI = [&](int b, int k) { return base + b * per + qb + 3 * vb + k * ib; };
    const int64_t nchunks = ceil_div(nq, chunk);
    cudaStream_t cs = h->copy_stream;
    if (wait) {
        // the copy stream starts after everything already queued on the caller's stream
        CUDA_TRY(cudaEventRecord(h->ev_out[0], st));
        CUDA_TRY(cudaStreamWaitEvent(cs, h->ev_out[0], 0));
    }
    auto h2d = [&](int64_t c) -> lip_status {
        const int b = (int)(c & 1);
        const int64_t q0 = c * chunk, n = std::min(chunk, nq - q0);
        CUDA_TRY(cudaMemcpyAsync(dQ(b), static_cast<const char*>(Q) + (size_t)q0 * h->d * es, (size_t)n * h->d * es,
                                 cudaMemcpyHostToDevice, cs));
        CUDA_TRY(cudaEventRecord(h->ev_in[b], cs));
        return LIP_OK;
    };
    LIP_TRY(h2d(0));
    if (nchunks > 1) LIP_TRY(h2d(1));
    for (int64_t c = 0; c < nchunks; ++c) {
        const int b = (int)(c & 1);
        const int64_t q0 = c * chunk, n = std::min(chunk, nq - q0);
        CUDA_TRY(cudaStreamWaitEvent(st, h->ev_in[b], 0));
        LIP_TRY(eval_device(h, dQ(b), n, g ? dV(b, 0) : nullptr, lo ? dV(b, 1) : nullptr, hi ? dV(b, 2) : nullptr,
                            idx_up ? reinterpret_cast<int32_t*>(dI(b, 0)) : nullptr,
                            idx_lo ? reinterpret_cast<int32_t*>(dI(b, 1)) : nullptr, st));
        CUDA_TRY(cudaEventRecord(h->ev_out[b], st));
        CUDA_TRY(cudaStreamWaitEvent(cs, h->ev_out[b], 0));
        void* outs[3] = {g, lo, hi};
        for (int k = 0; k < 3; ++k)
            if (outs[k])
                CUDA_TRY(cudaMemcpyAsync(static_cast<char*>(outs[k]) + (size_t)q0 * es, dV(b, k), (size_t)n * es,
                                         cudaMemcpyDeviceToHost, cs));
        int32_t* idx[2] = {idx_up, idx_lo};
        for (int k = 0; k < 2; ++k)
            if (idx[k]) CUDA_TRY(cudaMemcpyAsync(idx[k] + q0, dI(b, k), (size_t)n * 4, cudaMemcpyDeviceToHost, cs));
        if (c + 2 < nchunks) LIP_TRY(h2d(c + 2));
    }
    if (wait) {
        CUDA_TRY(cudaStreamSynchronize(cs));
        CUDA_TRY(cudaStreamSynchronize(st));
    }
    return LIP_OK;
}

lip_status lip_eval_host(lip_handle h, const void* Q, int64_t nq, void* g, void* lo, void* hi, int32_t* idx_up,
                         int32_t* idx_lo, void* stream) {
    return eval_host(h, Q, nq, g, lo, hi, idx_up, idx_lo, stream, true);
}

lip_status lip_eval_host_async(lip_handle h, const void* Q, int64_t nq, void* g, void* lo, void* hi,
                               int32_t* idx_up, int32_t* idx_lo, void* stream) {
    return eval_host(h, Q, nq, g, lo, hi, idx_up, idx_lo, stream, false);
}

lip_status lip_estimate_M(lip_handle h, double* M_out, int64_t* i_out, int64_t* j_out, void* stream) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (!M_out || !i_out || !j_out) return fail(LIP_ERR_ARG, "an output pointer is NULL");
    double res[4];
    h->est_pending = 0;                  // a queued estimate's result is dropped
    LIP_TRY(estimate_part(h, 0, 1, res, static_cast<cudaStream_t>(stream), true));
    *M_out = res[0];
    *i_out = (int64_t)res[1];
    *j_out = (int64_t)res[2];
    return LIP_OK;
}

lip_status lip_estimate_M_async(lip_handle h, void* stream) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    DeviceGuard gd(h->device);
    if (h->est_pending == 1) CUDA_TRY(cudaEventSynchronize(h->est_done));   // est_back is reused
    h->est_pending = 0;
    if (!h->est_back) {
        void* p = nullptr;
        if (cudaMallocHost(&p, 64) != cudaSuccess) {
            cudaGetLastError();
            return fail(LIP_ERR_OOM, "pinned estimate result (64 bytes)");
        }
        h->est_back = static_cast<unsigned char*>(p);
    }
    if (!h->est_done) CUDA_TRY(cudaEventCreateWithFlags(&h->est_done, cudaEventDisableTiming));
    double res[4];
    LIP_TRY(estimate_part(h, 0, 1, res, static_cast<cudaStream_t>(stream), false));
    if (h->est_pending == 0) {           // known on the host (fewer than two points)
        memcpy(h->est_host_res, res, sizeof res);
        h->est_pending = 2;
    }
    return LIP_OK;
}

lip_status lip_estimate_M_result(lip_handle h, double* M_out, int64_t* i_out, int64_t* j_out) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (!M_out || !i_out || !j_out) return fail(LIP_ERR_ARG, "an output pointer is NULL");
    DeviceGuard gd(h->device);
    double res[4];
    LIP_TRY(estimate_collect(h, res));
    *M_out = res[0];
    *i_out = (int64_t)res[1];
    *j_out = (int64_t)res[2];
    return LIP_OK;
}

lip_status lip_estimate_M_part(lip_handle h, int32_t part, int32_t nparts, double* out, void* stream) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (!out) return fail(LIP_ERR_ARG, "out is NULL");
    if (nparts < 1 || part < 0 || part >= nparts) return fail(LIP_ERR_ARG, "part %d of %d is not valid", part, nparts);
    return estimate_part(h, part, nparts, out, static_cast<cudaStream_t>(stream), true);
}

lip_status lip_shard_scan(lip_handle h, const void* Q, int64_t nq, int64_t index_base, int64_t* key_up,
                          int64_t* key_lo, void* stream) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (nq < 0) return fail(LIP_ERR_ARG, "nq = %lld < 0", (long long)nq);
    if (index_base < 0 || index_base + h->cap > ((int64_t)1 << 31))
        return fail(LIP_ERR_ARG, "index_base %lld + capacity %lld exceeds 2^31", (long long)index_base,
                    (long long)h->cap);
    if (h->esize == 8) return fail(LIP_ERR_UNSUPPORTED, "data-sharded evaluation needs an FP32 or tensor-core handle");
    if (nq == 0) return LIP_OK;
    if (!Q || !key_up || !key_lo) return fail(LIP_ERR_ARG, "Q or a key array is NULL");
    DeviceGuard gd(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int nsplit = 0;
    LIP_TRY(scan_partials(h, Q, nq, st, &nsplit));
    CUDA_TRY(launch_shard_keys(h->esize, h->partial.p, nsplit, nq, Q, h->d, index_base, key_up, key_lo, st));
    count_launches(1);
    return LIP_OK;
}

lip_status lip_shard_reeval(lip_handle h, const void* Q, int64_t nq, int64_t index_base, const int64_t* key_up,
                            const int64_t* key_lo, double* hi64, double* lo64, void* stream) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (nq < 0) return fail(LIP_ERR_ARG, "nq = %lld < 0", (long long)nq);
    if (index_base < 0) return fail(LIP_ERR_ARG, "index_base = %lld < 0", (long long)index_base);
    if (nq == 0) return LIP_OK;
    if (!Q || !key_up || !key_lo || !hi64 || !lo64) return fail(LIP_ERR_ARG, "a pointer is NULL");
    DeviceGuard gd(h->device);
    MergeParams Mp;
    fill_merge_params(h, Q, nq, Mp);
    CUDA_TRY(launch_shard_reeval(h->esize, Mp, index_base, h->N, key_up, key_lo, hi64, lo64,
                                 static_cast<cudaStream_t>(stream)));
    count_launches(1);
    return LIP_OK;
}

lip_status lip_shard_finish(lip_handle h, int64_t nq, const int64_t* key_up, const int64_t* key_lo,
                            const double* hi64, const double* lo64, void* g, void* lo, void* hi, int32_t* idx_up,
                            int32_t* idx_lo, void* stream) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (nq < 0) return fail(LIP_ERR_ARG, "nq = %lld < 0", (long long)nq);
    if (nq == 0) return LIP_OK;
    if (!key_up || !key_lo || !hi64 || !lo64) return fail(LIP_ERR_ARG, "a key or value array is NULL");
    DeviceGuard gd(h->device);
    CUDA_TRY(launch_shard_finish(h->esize, nq, key_up, key_lo, hi64, lo64, g, lo, hi, idx_up, idx_lo,
                                 static_cast<cudaStream_t>(stream)));
    count_launches(1);
    return LIP_OK;
}

lip_status lip_backward(lip_handle h, const void* Q, int64_t nq, const int32_t* idx_up, const int32_t* idx_lo,
                        const void* grad_g, void* grad_Q, void* grad_y, double* grad_M, int32_t deterministic,
                        void* stream) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (nq < 0) return fail(LIP_ERR_ARG, "nq = %lld < 0", (long long)nq);
    if (nq > 0 && (!Q || !idx_up || !idx_lo || !grad_g)) return fail(LIP_ERR_ARG, "Q, indices or grad_g is NULL");
    DeviceGuard gd(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nb = backward_blocks(nq);
    const size_t part_b = round_up((int64_t)std::max(nb, 1) * 8, 256);
    const bool det = deterministic != 0 && grad_y && h->N > 0;
    const size_t fix_b = det ? round_up(h->N * 8, 256) : 0;
    LIP_TRY(h->bwd.ensure(part_b + 256 + fix_b, "backward scratch"));
    char* base = static_cast<char*>(h->bwd.p);
    BwdParams P;
    P.Q = Q;
    P.nq = nq;
    P.d = h->d;
    P.norm = h->norm;
    P.M = h->M;
    for (int i = 0; i < D_MAX; ++i) {
        P.mon[i] = h->mon[i];
        P.w[i] = h->w[i];
        P.sqf[i] = (float)((h->mon[i] < 0 ? -1.0 : 1.0) * h->w[i]);
    }
    P.X0 = h->X0;
    P.iu = idx_up;
    P.il = idx_lo;
    P.gbar = grad_g;
    P.grad_Q = grad_Q;
    P.gm_part = reinterpret_cast<double*>(base);
    P.arrived = reinterpret_cast<unsigned*>(base + part_b);
    P.grad_y = grad_y;
    P.grad_M = grad_M;
    P.gy_fix = det ? reinterpret_cast<unsigned long long*>(base + part_b + 256) : nullptr;
    P.gb_maxbits = P.arrived + 1;
    if (nq == 0) {
        if (grad_M) CUDA_TRY(cudaMemsetAsync(grad_M, 0, sizeof(double), st));
        return LIP_OK;
    }
    CUDA_TRY(cudaMemsetAsync(P.arrived, 0, 2 * sizeof(unsigned), st));
    if (det) {
        CUDA_TRY(cudaMemsetAsync(P.gy_fix, 0, (size_t)h->N * 8, st));
        CUDA_TRY(launch_grad_max(h->esize, grad_g, nq, P.arrived + 1, st));
    }
    CUDA_TRY(launch_backward(h->esize, P, st));
    if (det) CUDA_TRY(launch_grad_y_fix(h->esize, P.gy_fix, P.gb_maxbits, nq, h->N, grad_y, st));
    count_launches(det ? 3 : 1);
    return LIP_OK;
}

lip_status lip_check(lip_handle h, void* stream) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    DeviceGuard gd(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned bits = 0;
    CUDA_TRY(cudaMemcpyAsync(&bits, h->status, sizeof bits, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (h->copy_stream) CUDA_TRY(cudaStreamSynchronize(h->copy_stream));   // lip_eval_host_async's copies
    if (bits) {
        CUDA_TRY(cudaMemsetAsync(h->status, 0, sizeof bits, st));
        CUDA_TRY(cudaStreamSynchronize(st));
    }
    if (bits & ERRBIT_TIMEOUT) return fail(LIP_ERR_TIMEOUT, "a bounded wait in a kernel gave up");
    if (bits & ERRBIT_NONFINITE)
        return fail(LIP_ERR_NONFINITE, "a deferred add held NaN or Inf (those points were replaced)");
    return LIP_OK;
}

lip_status lip_set_tuning(lip_handle h, int32_t tile_groups, int32_t splits, int32_t variant) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (tile_groups != 0 && tile_groups != 8 && tile_groups != 16 && tile_groups != 32 && tile_groups != 64)
        return fail(LIP_ERR_ARG, "tile_groups = %d is not 0, 8, 16, 32 or 64", tile_groups);
    if (splits < 0 || splits > 4096) return fail(LIP_ERR_ARG, "splits = %d is outside [0, 4096]", splits);
    if (variant < -1 || variant >= SCAN_VARIANTS_ALL)
        return fail(LIP_ERR_ARG, "variant = %d is outside [-1, %d]", variant, SCAN_VARIANTS_ALL - 1);
    if (h->tc && variant > 5) return fail(LIP_ERR_ARG, "variant = %d: tensor-core handles take 0 to 5", variant);
    if (h->esize == 8 && variant > 1) return fail(LIP_ERR_ARG, "variant = %d: FP64 handles take 0 or 1", variant);
    DeviceGuard gd(h->device);
    if (tile_groups) h->tile_groups = tile_groups;
    h->splits = splits;
    if (variant >= 0 && h->tc) h->tc_variant = variant;
    if (variant >= 0 && h->esize == 8) h->fp64_mode = variant;
    if (h->esize == 8 && h->exact32) {
        const size_t smem32 = (size_t)SCAN_STAGES * h->tile_groups * h->nch32 * 16;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&h->occ32, h->kinfo32.kernel, SCAN_THREADS, smem32) !=
                cudaSuccess || h->occ32 < 1) {
            cudaGetLastError();
            h->occ32 = 1;
        }
    }
    if (variant >= 0 && h->exact) {
        // variants 6 / 7 (the pruned scan) keep the exact kernel of 0 / 1 for the shapes
        // and precisions without a pruned instantiation
        const ScanKernelInfo k = scan_exact_info(h->norm, h->C, h->d - h->C, variant < SCAN_VARIANTS ? variant : variant & 1);
        if (k.launch) {
            h->kinfo = k;
            h->variant = variant;
            h->pruned = false;
            if (variant >= SCAN_VARIANTS && h->esize == 4) {
                const PrunedKernelInfo pk = scan_pruned_info(h->norm, h->C, h->d - h->C, variant);
                if (pk.launch) {
                    h->pinfo = pk;
                    h->pruned = true;
                }
            }
        }
    }
    if (h->exact) {
        const size_t smem = (size_t)SCAN_STAGES * h->tile_groups * h->nch * 16;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&h->occ_blocks, h->kinfo.kernel, SCAN_THREADS, smem) !=
                cudaSuccess || h->occ_blocks < 1) {
            cudaGetLastError();
            h->occ_blocks = 1;
        }
    }
    return LIP_OK;
}

lip_status lip_autotune(lip_handle h, const void* Q, int64_t nq, int32_t reps, int32_t* tile_groups_out,
                        int32_t* splits_out, int32_t* variant_out, double* ms_out, void* stream) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (nq < 1 || !Q) return fail(LIP_ERR_ARG, "autotuning needs queries (nq = %lld)", (long long)nq);
    if (reps < 1 || reps > 100) return fail(LIP_ERR_ARG, "reps = %d is outside [1, 100]", reps);
    DeviceGuard gd(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void* out = nullptr;
    CUDA_TRY(dev_malloc(&out, (size_t)nq * (3 * h->esize + 8)));
    char* o = static_cast<char*>(out);
    void* g = o;
    int32_t* iu = reinterpret_cast<int32_t*>(o + (size_t)nq * 3 * h->esize);
    int32_t* il = iu + nq;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEvent_t u0 = h->ev_scan0, u1 = h->ev_scan1;
    h->ev_scan0 = h->ev_scan1 = nullptr;
    const int32_t keep_tg = h->tile_groups, keep_sp = h->splits;
    const int32_t keep_v = h->tc ? h->tc_variant : (h->esize == 8 ? h->fp64_mode : h->variant);
    lip_status s = LIP_OK;
    double best = 1e300;
    int32_t btg = keep_tg, bsp = keep_sp, bv = keep_v;
    const int tiles[] = {8, 16, 32, 64}, splits[] = {0, 1, 2, 3, 4, 6, 8, 12, 16};
    const int nv = h->tc ? 6 : (h->esize == 8 ? 2 : (h->exact ? SCAN_VARIANTS_ALL : 1));
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        s = fail(LIP_ERR_CUDA, "cudaEventCreate failed");
    } else {
        for (int v = 0; v < nv && s == LIP_OK; ++v)
            for (int ti = 0; ti < (h->tc ? 1 : 4) && s == LIP_OK; ++ti)
                for (int sp : splits) {
                    const int tg = h->tc ? keep_tg : tiles[ti];
                    if ((s = lip_set_tuning(h, tg, sp, v)) != LIP_OK) break;
                    std::vector<float> ms;
                    for (int r = 0; r <= reps && s == LIP_OK; ++r) {      // the first run warms up
                        cudaEventRecord(e0, st);
                        s = eval_device(h, Q, nq, g, nullptr, nullptr, iu, il, st);
                        cudaEventRecord(e1, st);
                        if (cudaEventSynchronize(e1) != cudaSuccess) s = fail(LIP_ERR_CUDA, "autotune timing failed");
                        float t = 0.f;
                        cudaEventElapsedTime(&t, e0, e1);
                        if (r > 0) ms.push_back(t);
                    }
                    if (s != LIP_OK) break;
                    std::sort(ms.begin(), ms.end());
                    const double med = ms[ms.size() / 2];
                    if (med < best) { best = med; btg = tg; bsp = sp; bv = v; }
                    if (h->tc || h->pruned) break;     // the tensor-core form ignores tiles and splits,
                                                       // the pruned scan the splits
                }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    h->ev_scan0 = u0;
    h->ev_scan1 = u1;
    if (s != LIP_OK) {
        lip_set_tuning(h, keep_tg, keep_sp, keep_v);
        return s;
    }
    LIP_TRY(lip_set_tuning(h, btg, bsp, bv));
    if (tile_groups_out) *tile_groups_out = btg;
    if (splits_out) *splits_out = bsp;
    if (variant_out) *variant_out = bv;
    if (ms_out) *ms_out = best;
    return LIP_OK;
}

lip_status lip_get_tuning(lip_handle h, int32_t* tile_groups, int32_t* splits, int32_t* last_splits,
                          int32_t* queries_per_thread, int32_t* variant) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (variant) *variant = h->tc ? h->tc_variant : (h->esize == 8 ? h->fp64_mode : h->variant);
    if (tile_groups) *tile_groups = h->tile_groups;
    if (splits) *splits = h->splits;
    if (last_splits) *last_splits = h->last_splits;
    if (queries_per_thread)
        *queries_per_thread = h->pruned ? h->pinfo.rows
                                        : ((h->esize == 8 && h->fp64_mode == 0) ? h->kinfo32.rows : h->kinfo.rows);
    return LIP_OK;
}

lip_status lip_set_timing_events(lip_handle h, void* ev_before_scan, void* ev_after_scan) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if ((ev_before_scan == nullptr) != (ev_after_scan == nullptr)) return fail(LIP_ERR_ARG, "give both events or neither");
    h->ev_scan0 = static_cast<cudaEvent_t>(ev_before_scan);
    h->ev_scan1 = static_cast<cudaEvent_t>(ev_after_scan);
    return LIP_OK;
}

uint64_t lip_kernel_launches(void) { return launches_total(); }

lip_status lip_last_estimate_work(lip_handle h, int64_t* out) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (!out) return fail(LIP_ERR_ARG, "out is NULL");
    for (int k = 0; k < 3; ++k) out[k] = h->est_work[k];
    return LIP_OK;
}

lip_status lip_last_scan_stats(lip_handle h, int64_t* out) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (!out) return fail(LIP_ERR_ARG, "out is NULL");
    out[0] = out[2] = out[4] = -1;
    out[1] = h->sp_total;
    out[3] = h->sp_total < 0 ? -1 : h->sp_tiles;
    if (h->sp_total < 0 || !h->sp_data.p) return LIP_OK;
    const int64_t N = h->N, npad = round_up(N, PAD_POINTS), ngroups = npad / GROUP;
    const size_t off = round_up(N * 4, 256) + round_up(ngroups * h->pinfo.nch * 16, 256) +
                       round_up(ngroups / PRUNED_CG * pruned_box_f4(h->dl) * 16, 256) + round_up(D_MAX * 8, 256);
    unsigned long long w[3] = {0, 0, 0};
    DeviceGuard gd(h->device);
    CUDA_TRY(cudaDeviceSynchronize());
    CUDA_TRY(cudaMemcpy(w, static_cast<char*>(h->sp_data.p) + off, sizeof w, cudaMemcpyDeviceToHost));
    out[0] = (int64_t)w[0];
    out[2] = (int64_t)w[1];
    out[4] = (int64_t)w[2];
    return LIP_OK;
}

lip_status lip_last_scan_work(lip_handle h, int64_t* evaluated, int64_t* total) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (!evaluated || !total) return fail(LIP_ERR_ARG, "an output pointer is NULL");
    int64_t s[5];
    LIP_TRY(lip_last_scan_stats(h, s));
    *evaluated = s[0];
    *total = s[1];
    return LIP_OK;
}

lip_status lip_set_estimate_full(lip_handle h, int32_t full) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (full < 0 || full > 2) return fail(LIP_ERR_ARG, "estimate form %d is not 0, 1 or 2", (int)full);
    h->est_form = full;
    return LIP_OK;
}

lip_status lip_set_tc_window(lip_handle h, int64_t bytes) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (bytes < 0) return fail(LIP_ERR_ARG, "window = %lld < 0", (long long)bytes);
    h->tc_window = bytes;
    return LIP_OK;
}

int64_t lip_last_fallback(lip_handle h) {
    if (!h) return -1;
    if (!h->tc_fb_count) return 0;
    int n = 0;
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(&n, h->tc_fb_count, sizeof n, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return n;
}

void lip_free(lip_handle h) { free_model(h); }

const char* lip_status_string(lip_status s) {
    switch (s) {
        case LIP_OK: return "ok";
        case LIP_ERR_ARG: return "invalid argument";
        case LIP_ERR_NONFINITE: return "non-finite data";
        case LIP_ERR_OOM: return "out of memory";
        case LIP_ERR_CUDA: return "CUDA error";
        case LIP_ERR_CAPACITY: return "capacity exceeded";
        case LIP_ERR_TIMEOUT: return "device wait timed out";
        case LIP_ERR_UNSUPPORTED: return "unsupported";
        case LIP_ERR_NO_DEVICE: return "no CUDA device";
        case LIP_ERR_STATE: return "call out of order";
    }
    return "unknown status";
}

size_t lip_last_error(char* buf, size_t len) {
    if (buf && len > 0) {
        const std::string& e = last_error_text();
        const size_t n = std::min(len - 1, e.size());
        std::memcpy(buf, e.data(), n);
        buf[n] = 0;
    }
    return last_error_text().size();
}

size_t lip_last_error_detail(char* buf, size_t len) { return lip_last_error(buf, len); }

lip_status lip_eval_batched(lip_batch b, void* stream) { return lip_batch_eval(b, stream); }

const char* lip_version(void) { return "0.1.0 sm_103a"; }

lip_status lip_debug_fail_alloc(int64_t n) {
    if (n < 0) return fail(LIP_ERR_ARG, "n = %lld < 0", (long long)n);
    g_fail_alloc_countdown.store(n, std::memory_order_relaxed);
    return LIP_OK;
}

lip_status lip_debug_sqrt_fma(const float* s, float* out, int64_t n, void* stream) {
    if (n < 0) return fail(LIP_ERR_ARG, "n = %lld < 0", (long long)n);
    if (n > 0 && (!s || !out)) return fail(LIP_ERR_ARG, "s or out is NULL");
    CUDA_TRY(launch_sqrt_fma(s, out, n, static_cast<cudaStream_t>(stream)));
    count_launches(n > 0 ? 1 : 0);
    return LIP_OK;
}

lip_status lip_debug_scan_fault(lip_handle h, uint64_t wait_limit_ns, int32_t skip_tile) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (skip_tile < -1) return fail(LIP_ERR_ARG, "skip_tile = %d < -1", skip_tile);
    if (wait_limit_ns > WAIT_LIMIT_NS) return fail(LIP_ERR_ARG, "wait limit above the default %llu ns", WAIT_LIMIT_NS);
    h->dbg_wait_ns = wait_limit_ns;
    h->dbg_skip_tile = skip_tile;
    return LIP_OK;
}

}  // extern "C"
