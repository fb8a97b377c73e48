// C ABI, local Lipschitz constants (Sec. 4.3): fitting the per-datum step functions, the
// knots and table, and the evaluation with the local constants (k = 1 and k > 1).
#include "model.h"

// ------------------------------------------------ local Lipschitz constants (Sec. 4.3)

namespace {

constexpr size_t LOC_SMALL_BYTES = LOC_BUCKETS * sizeof(unsigned) + 2 * LOC_KNOTS * sizeof(double) +
                                   3 * LOC_KNOTS * sizeof(float) + sizeof(LocMeta);

lip_status local_supported(const lip_model* h) {
    if (h->N < 1) return fail(LIP_ERR_ARG, "the handle holds no data");
    return LIP_OK;
}

// Carves the per-datum buffers and fills P's pointers (sizes for the current N).
lip_status local_buffers(lip_model* h, int64_t S, LocalParams& P) {
    const int64_t N = h->N, npad = local_pad(N);
    const int pr = local_record_floats(h->d);
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t b_rec = al((size_t)npad * pr * 4), b_mt = al((size_t)npad * LOC_KNOTS * 4);
    const size_t b_mt64 = al((size_t)N * LOC_KNOTS * 8), b_vec = al((size_t)N * 8);
    LIP_TRY(h->loc_buf.ensure(b_rec + b_mt + b_mt64 + 2 * b_vec, "local Lipschitz tables"));
    // the samples and their two counts, then the screen's per-datum buffers
    const size_t b_s = al((size_t)std::max<int64_t>(S, 1) * 8) + al((size_t)std::max<int64_t>(S, 1) * 2 * 4);
    const size_t b_n = al((size_t)N * 4), b_c = al((size_t)N * local_candidates() * 4);
    LIP_TRY(h->loc_tmp.ensure(b_s + 3 * b_n + b_c, "local Lipschitz scratch"));
    if (!h->loc_small) {
        cudaError_t e = dev_malloc(reinterpret_cast<void**>(&h->loc_small), LOC_SMALL_BYTES);
        if (e != cudaSuccess) {
            h->loc_small = nullptr;
            return cuda_fail(e, "local Lipschitz knots");
        }
    }
    char* b = static_cast<char*>(h->loc_buf.p);
    P = LocalParams{};
    P.X0 = h->X0;
    P.y0 = h->y0;
    P.es = h->esize;
    P.N = N;
    P.npad = npad;
    P.d = h->d;
    P.dp = local_dim_pad(h->d);
    P.pr = pr;
    P.norm = h->norm;
    for (int i = 0; i < D_MAX; ++i) P.w[i] = i < h->d ? h->w[i] : 1.0;
    P.mono = h->C > 0 ? 1 : 0;
    P.cmask = 0;
    for (int i = 0; i < D_MAX; ++i) {
        P.mon[i] = i < h->d ? h->mon[i] : 0;
        if (P.mon[i] != 0) P.cmask |= 1u << i;
    }
    P.rec = reinterpret_cast<float*>(b);
    P.mt = reinterpret_cast<float*>(b + b_rec);
    P.mt64 = reinterpret_cast<double*>(b + b_rec + b_mt);
    P.d1 = reinterpret_cast<double*>(b + b_rec + b_mt + b_mt64);
    P.F = reinterpret_cast<double*>(b + b_rec + b_mt + b_mt64 + b_vec);
    P.bpack = reinterpret_cast<unsigned*>(h->loc_small);
    P.T64 = reinterpret_cast<double*>(P.bpack + LOC_BUCKETS);
    P.raw = P.T64 + LOC_KNOTS;
    P.Tf = reinterpret_cast<float*>(P.raw + LOC_KNOTS);
    P.meta = reinterpret_cast<LocMeta*>(P.Tf + 3 * LOC_KNOTS);
    P.sample = static_cast<double*>(h->loc_tmp.p);
    char* t = static_cast<char*>(h->loc_tmp.p);
    P.counts = reinterpret_cast<int*>(t + al((size_t)std::max<int64_t>(S, 1) * 8));
    P.ubound = reinterpret_cast<float*>(t + b_s);
    P.over = reinterpret_cast<int*>(t + b_s + b_n);
    P.ncand = reinterpret_cast<int*>(t + b_s + 2 * b_n);
    P.cand = reinterpret_cast<int*>(t + b_s + 3 * b_n);
    P.S = S;
    return LIP_OK;
}

// Layout, knots (sampled, or the m given ones), both table passes; synchronises to read
// the knots back.
lip_status local_run(lip_model* h, bool sampled, int m, int64_t S, uint64_t seed, const double* knots,
                     cudaStream_t st) {
    h->loc_valid = false;
    LocalParams P;
    LIP_TRY(local_buffers(h, sampled ? S : 0, P));
    P.m = m;
    P.seed = seed;
    CUDA_TRY(cudaMemsetAsync(P.meta, 0, sizeof(LocMeta), st));
    if (!sampled && m > 0) CUDA_TRY(cudaMemcpyAsync(P.raw, knots, (size_t)m * sizeof(double), cudaMemcpyHostToDevice, st));
    CUDA_TRY(launch_local_layout(P, st));
    CUDA_TRY(launch_local_knots(P, sampled, st));
    // the table kernels' lookup depends on whether a bucket holds two knots
    LocMeta meta{};
    CUDA_TRY(cudaMemcpyAsync(&meta, P.meta, sizeof meta, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    CUDA_TRY(launch_local_table(P, meta.bucket_ok != 0, meta.m, st));
    count_launches(5 + (sampled && S > 0 ? 3 : 0));   // layout, knots, screen, exact, pass 2; sample, rank, pick
    CUDA_TRY(cudaMemcpyAsync(&meta, P.meta, sizeof meta, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(h->loc_T, P.T64, sizeof h->loc_T, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    h->loc_m = meta.m;
    h->loc_bucket = meta.bucket_ok != 0;
    h->loc_scale = meta.scale;
    h->loc_over = meta.n_over;
    h->loc_max_cand = meta.max_cand;
    h->loc_valid = true;
    return LIP_OK;
}

}  // namespace

extern "C" {

lip_status lip_local_fit(lip_handle h, int32_t nknots, int64_t sample_pairs, uint64_t seed, void* stream) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (nknots < 0 || nknots > LIP_LOCAL_KNOTS_MAX)
        return fail(LIP_ERR_ARG, "nknots = %d is outside [0, %d]", nknots, LIP_LOCAL_KNOTS_MAX);
    if (sample_pairs < 0 || sample_pairs > LIP_LOCAL_SAMPLE_MAX)
        return fail(LIP_ERR_ARG, "sample_pairs = %lld is outside [0, %d]", (long long)sample_pairs, LIP_LOCAL_SAMPLE_MAX);
    LIP_TRY(local_supported(h));
    DeviceGuard g(h->device);
    return local_run(h, true, nknots, sample_pairs, seed, nullptr, static_cast<cudaStream_t>(stream));
}

lip_status lip_local_fit_knots(lip_handle h, const double* knots, int32_t nknots, void* stream) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (nknots < 0 || nknots > LIP_LOCAL_KNOTS_MAX)
        return fail(LIP_ERR_ARG, "nknots = %d is outside [0, %d]", nknots, LIP_LOCAL_KNOTS_MAX);
    if (nknots > 0 && !knots) return fail(LIP_ERR_ARG, "knots is NULL");
    for (int i = 0; i < nknots; ++i) {
        if (!(knots[i] > 0.0) || !std::isfinite(knots[i]))
            return fail(LIP_ERR_ARG, "knots[%d] = %g must be finite and > 0", i, knots[i]);
        if (i > 0 && !(knots[i] > knots[i - 1])) return fail(LIP_ERR_ARG, "knots must increase strictly (index %d)", i);
    }
    LIP_TRY(local_supported(h));
    DeviceGuard g(h->device);
    return local_run(h, false, nknots, 0, 0, knots, static_cast<cudaStream_t>(stream));
}

lip_status lip_local_knots(lip_handle h, double* knots, int32_t* nknots) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (!h->loc_valid) return fail(LIP_ERR_STATE, "no local Lipschitz table: call lip_local_fit after the last data change");
    if (nknots) *nknots = h->loc_m;
    if (knots)
        for (int i = 0; i < h->loc_m; ++i) knots[i] = h->loc_T[i];
    return LIP_OK;
}

lip_status lip_local_stats(lip_handle h, int32_t* overflow_rows, int32_t* max_candidates) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (!h->loc_valid) return fail(LIP_ERR_STATE, "no local Lipschitz table: call lip_local_fit after the last data change");
    if (overflow_rows) *overflow_rows = h->loc_over;
    if (max_candidates) *max_candidates = h->loc_max_cand;
    return LIP_OK;
}

lip_status lip_local_table(lip_handle h, double* d1, double* F, double* Mtab, void* stream) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (!h->loc_valid) return fail(LIP_ERR_STATE, "no local Lipschitz table: call lip_local_fit after the last data change");
    DeviceGuard g(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LocalParams P;
    LIP_TRY(local_buffers(h, 0, P));
    if (d1) CUDA_TRY(cudaMemcpyAsync(d1, P.d1, (size_t)h->N * 8, cudaMemcpyDeviceToDevice, st));
    if (F) CUDA_TRY(cudaMemcpyAsync(F, P.F, (size_t)h->N * 8, cudaMemcpyDeviceToDevice, st));
    if (Mtab)
        CUDA_TRY(cudaMemcpy2DAsync(Mtab, (size_t)(h->loc_m + 1) * 8, P.mt64, (size_t)LOC_KNOTS * 8,
                                   (size_t)(h->loc_m + 1) * 8, (size_t)h->N, cudaMemcpyDeviceToDevice, st));
    return LIP_OK;
}

lip_status lip_eval_local_k(lip_handle h, const void* Q, int64_t nq, int32_t k, const double* wk, void* g, void* lo,
                            void* hi, int32_t* idx_up, int32_t* idx_lo, void* stream) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (nq < 0) return fail(LIP_ERR_ARG, "nq = %lld < 0", (long long)nq);
    if (k < 1 || k > 8) return fail(LIP_ERR_ARG, "k = %d is outside [1, 8]", k);
    if (!wk) return fail(LIP_ERR_ARG, "wk is NULL");
    for (int e = 0; e < k; ++e)
        if (!(wk[e] >= 0.0) || !std::isfinite(wk[e])) return fail(LIP_ERR_ARG, "wk[%d] = %g must be finite and >= 0", e, wk[e]);
    if (!h->loc_valid) return fail(LIP_ERR_STATE, "no local Lipschitz table: call lip_local_fit after the last data change");
    if (nq == 0) return LIP_OK;
    if (!Q) return fail(LIP_ERR_ARG, "Q is NULL");
    DeviceGuard gd(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LocalParams P;
    LIP_TRY(local_buffers(h, 0, P));
    const int K = k <= 2 ? 2 : (k <= 4 ? 4 : 8);
    const int64_t gx = ceil_div(nq, (int64_t)local_topk_threads());
    if (gx > 0x7fffffff) return fail(LIP_ERR_ARG, "nq = %lld is too large", (long long)nq);
    const int64_t tile = local_scan_tile();
    const int64_t tiles = P.npad / tile;
    const int64_t want = std::max<int64_t>(1, ceil_div((int64_t)4 * h->sms * 4, gx));
    const int64_t s = std::min<int64_t>(std::min<int64_t>(want, 64), tiles);
    const int64_t pps = round_up(ceil_div(P.npad, s), tile);
    const int nsplit = (int)ceil_div(P.npad, pps);
    LIP_TRY(h->partial.ensure((size_t)nsplit * nq * 2 * K * 8, "k-neighbour scratch"));
    LocalScanParams S{};
    S.Q = Q;
    S.es = h->esize;
    S.nq = nq;
    S.d = h->d;
    S.dp = P.dp;
    // the query's scaling: mirrored where decreasing for monotone handles (as the records)
    for (int i = 0; i < D_MAX; ++i) S.w[i] = (P.mono && P.mon[i] < 0) ? -P.w[i] : P.w[i];
    S.mono = P.mono;
    S.cmask = P.cmask;
    S.rec = P.rec;
    S.mt = P.mt;
    S.Tf = P.Tf;
    S.bpack = P.bpack;
    S.scale = h->loc_scale;
    S.bucket_ok = h->loc_bucket ? 1 : 0;
    S.npad = P.npad;
    S.points_per_split = pps;
    S.partial = h->partial.p;
    LocalMergeParams Mp{};
    Mp.Q = S.Q;
    Mp.es = h->esize;
    Mp.nq = nq;
    Mp.d = h->d;
    Mp.norm = h->norm;
    Mp.m = h->loc_m;
    Mp.nsplit = nsplit;
    for (int i = 0; i < D_MAX; ++i) {
        Mp.w[i] = P.w[i];
        Mp.mon[i] = P.mon[i];
    }
    Mp.mono = P.mono;
    Mp.X0 = P.X0;
    Mp.y0 = P.y0;
    Mp.d1 = P.d1;
    Mp.F = P.F;
    Mp.mt64 = P.mt64;
    Mp.T64 = P.T64;
    Mp.partial = h->partial.p;
    Mp.g = g;
    Mp.lo = lo;
    Mp.hi = hi;
    Mp.idx_up = idx_up;
    Mp.idx_lo = idx_lo;
    LocalTopkWeights W{};
    for (int e = 0; e < 8; ++e) W.wk[e] = e < k ? wk[e] : 0.0;
    CUDA_TRY(launch_local_eval_k(h->norm, k, K, S, (int)gx, nsplit, Mp, W, st));
    count_launches(2);
    return LIP_OK;
}

lip_status lip_eval_local(lip_handle h, const void* Q, int64_t nq, void* g, void* lo, void* hi, int32_t* idx_up,
                          int32_t* idx_lo, void* stream) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (nq < 0) return fail(LIP_ERR_ARG, "nq = %lld < 0", (long long)nq);
    if (!h->loc_valid) return fail(LIP_ERR_STATE, "no local Lipschitz table: call lip_local_fit after the last data change");
    if (nq == 0) return LIP_OK;
    if (!Q) return fail(LIP_ERR_ARG, "Q is NULL");
    DeviceGuard gd(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LocalParams P;
    LIP_TRY(local_buffers(h, 0, P));
    const int64_t gx = ceil_div(nq, (int64_t)(P.mono ? local_queries_per_block_mono() : local_queries_per_block(h->d)));
    if (gx > 0x7fffffff) return fail(LIP_ERR_ARG, "nq = %lld is too large", (long long)nq);
    const int64_t tile = local_scan_tile();
    const int64_t tiles = P.npad / tile;
    const int s = choose_splits(h, gx, tiles);
    const int64_t pps = round_up(ceil_div(P.npad, s), tile);
    const int nsplit = (int)ceil_div(P.npad, pps);
    h->last_splits = nsplit;
    LIP_TRY(h->partial.ensure((size_t)nsplit * nq * sizeof(PartialRec<float>), "scan scratch"));
    LocalScanParams S{};
    S.Q = Q;
    S.es = h->esize;
    S.nq = nq;
    S.d = h->d;
    S.dp = P.dp;
    // the query's scaling: mirrored where decreasing for monotone handles (as the records)
    for (int i = 0; i < D_MAX; ++i) S.w[i] = (P.mono && P.mon[i] < 0) ? -P.w[i] : P.w[i];
    S.mono = P.mono;
    S.cmask = P.cmask;
    S.rec = P.rec;
    S.mt = P.mt;
    S.Tf = P.Tf;
    S.bpack = P.bpack;
    S.scale = h->loc_scale;
    S.bucket_ok = h->loc_bucket ? 1 : 0;
    S.npad = P.npad;
    S.points_per_split = pps;
    S.partial = h->partial.p;
    LocalMergeParams Mp{};
    Mp.Q = S.Q;
    Mp.es = h->esize;
    Mp.nq = nq;
    Mp.d = h->d;
    Mp.norm = h->norm;
    Mp.m = h->loc_m;
    Mp.nsplit = nsplit;
    for (int i = 0; i < D_MAX; ++i) {
        Mp.w[i] = P.w[i];
        Mp.mon[i] = P.mon[i];
    }
    Mp.mono = P.mono;
    Mp.X0 = P.X0;
    Mp.y0 = P.y0;
    Mp.d1 = P.d1;
    Mp.F = P.F;
    Mp.mt64 = P.mt64;
    Mp.T64 = P.T64;
    Mp.partial = h->partial.p;
    Mp.g = g;
    Mp.lo = lo;
    Mp.hi = hi;
    Mp.idx_up = idx_up;
    Mp.idx_lo = idx_lo;
    if (h->ev_scan0) CUDA_TRY(cudaEventRecord(h->ev_scan0, st));
    CUDA_TRY(launch_local_eval(h->norm, S, (int)gx, nsplit, h->loc_bucket, Mp, st));
    if (h->ev_scan1) CUDA_TRY(cudaEventRecord(h->ev_scan1, st));
    count_launches(2);
    return LIP_OK;
}

}  // extern "C"
