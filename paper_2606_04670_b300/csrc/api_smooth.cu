// C ABI, penalty smoothing (Sec. 4.4): the objective of Eq. (optim) with its gradient, and
// the L-BFGS minimisation that replaces y by y + eps.
#include "model.h"

namespace {

// ------------------------------------------------ penalty smoothing (Sec. 4.4)

struct SmoothRun {
    lip_model* h;
    SmoothParams P;
    int gx;
    cudaStream_t st;
    double* out;      // [2]: Phi, S1
    double* red;      // [1]: reduction result
    double* bsum;     // [2 * reduce blocks]
    double* rpart;    // [reduce blocks]
};

lip_status smooth_check(const lip_model* h, double M, double p) {
    if (!(M >= 0.0) || !std::isfinite(M)) return fail(LIP_ERR_ARG, "M = %g must be finite and >= 0", M);
    if (!(p > 0.0) || !std::isfinite(p)) return fail(LIP_ERR_ARG, "p = %g must be finite and > 0", p);
    if (h->N < 1) return fail(LIP_ERR_ARG, "the handle holds no data");
    return LIP_OK;
}

lip_status smooth_setup(lip_model* h, double M, double p, cudaStream_t st, SmoothRun& r) {
    r = SmoothRun{};
    r.h = h;
    r.st = st;
    SmoothParams& P = r.P;
    P.X0 = h->X0;
    P.y0 = h->y0;
    P.es = h->esize;
    P.N = h->N;
    const int64_t tile = smooth_tile();
    P.npad = round_up(h->N, tile);
    P.d = h->d;
    P.dp = h->d <= 16 ? (h->d + 3) / 4 * 4 : 32;     // one wide shape for d above 16
    P.C = h->C;
    P.norm = h->norm;
    for (int j = 0; j < D_MAX; ++j) {
        P.perm[j] = h->perm[j];
        P.scale[j] = M * h->sgnw[j];
    }
    P.p = p;
    r.gx = (int)ceil_div(h->N, (int64_t)smooth_rows_per_block(h->esize));
    const int64_t tiles = P.npad / tile;
    // the pass is triangular (row i takes k > i), so many blocks are short or empty: fine
    // splits (up to 64) keep the last wave short
    const int64_t want = std::max<int64_t>(1, ceil_div((int64_t)h->sms * 256, r.gx));
    const int64_t s = std::min<int64_t>(std::min<int64_t>(want, 64), tiles);
    P.points_per_split = round_up(ceil_div(P.npad, s), tile);
    P.nsplit = (int)ceil_div(P.npad, P.points_per_split);
    if (h->esize == 8) {               // FP64 pair terms: the double layout
        LIP_TRY(h->sm_rec.ensure((size_t)P.npad * (P.dp + 2) * sizeof(double), "smoothing layout"));
        P.rec64 = static_cast<double*>(h->sm_rec.p);
    } else {
        LIP_TRY(h->sm_rec.ensure((size_t)P.npad * (P.dp + 4) * sizeof(float), "smoothing layout"));
    }
    const size_t part_b = (size_t)P.nsplit * h->N * 2 * sizeof(double), col_b = (size_t)h->N * 8;
    LIP_TRY(h->sm_part.ensure(part_b + col_b + 16, "smoothing partials"));
    const int rb = smooth_reduce_blocks();
    LIP_TRY(h->sm_small.ensure((size_t)(4 + 3 * rb) * sizeof(double), "smoothing scalars"));
    if (h->esize != 8) P.rec = static_cast<float*>(h->sm_rec.p);
    P.partial = static_cast<double*>(h->sm_part.p);
    P.colfix = reinterpret_cast<unsigned long long*>(static_cast<char*>(h->sm_part.p) + part_b);
    P.zbits = reinterpret_cast<unsigned*>(static_cast<char*>(h->sm_part.p) + part_b + col_b);
    r.out = static_cast<double*>(h->sm_small.p);
    r.red = r.out + 2;
    r.bsum = r.out + 4;
    r.rpart = r.bsum + 2 * rb;
    return LIP_OK;
}

lip_status smooth_eval(SmoothRun& r, const double* eps, double* grad, double* f) {
    CUDA_TRY(launch_smooth_objective(r.P, eps, grad, r.bsum, r.out, r.gx, r.st));
    count_launches(4);
    CUDA_TRY(cudaMemcpyAsync(f, r.out, sizeof(double), cudaMemcpyDeviceToHost, r.st));
    CUDA_TRY(cudaStreamSynchronize(r.st));
    return LIP_OK;
}

// op 0: a'b; op 1: max |a|
lip_status smooth_reduce(SmoothRun& r, const double* a, const double* b, int op, double* out) {
    CUDA_TRY(launch_vec_reduce(a, b, r.h->N, op, r.rpart, r.red, r.st));
    count_launches(2);
    CUDA_TRY(cudaMemcpyAsync(out, r.red, sizeof(double), cudaMemcpyDeviceToHost, r.st));
    CUDA_TRY(cudaStreamSynchronize(r.st));
    return LIP_OK;
}

lip_status smooth_axpy(SmoothRun& r, double* out, const double* a, double alpha, const double* b) {
    CUDA_TRY(launch_vec_axpy(out, a, alpha, b, r.h->N, r.st));
    count_launches(1);
    return LIP_OK;
}

lip_status smooth_scale(SmoothRun& r, double* out, const double* a, double alpha) {
    CUDA_TRY(launch_vec_scale(out, a, alpha, r.h->N, r.st));
    count_launches(1);
    return LIP_OK;
}

// L-BFGS from eps = 0 (Nocedal and Wright, Algorithms 7.4 and 7.5): the two-loop
// recursion with gamma = s'y / y'y of the newest pair, backtracking from step 1 (halving)
// to the Armijo condition with c1 = 1e-4, pairs kept when s'y > 1e-12 |s| |y|, a restart
// from steepest descent if the direction is not a descent one; stops at max |g| <= gtol.
lip_status smooth_lbfgs(SmoothRun& r, int max_iter, int hist, double gtol, double* f_out, int* iters_out,
                        int* evals_out, double** x_out) {
    const int64_t N = r.h->N;
    LIP_TRY(r.h->sm_vec.ensure((size_t)(6 + 2 * hist) * N * sizeof(double), "smoothing vectors"));
    double* base = static_cast<double*>(r.h->sm_vec.p);
    double *x = base, *g = base + N, *dir = base + 2 * N, *xn = base + 3 * N, *gn = base + 4 * N, *q = base + 5 * N;
    double* S = base + 6 * N;
    double* Y = S + (size_t)hist * N;
    std::vector<double> rho(hist), alpha(hist);
    int nstore = 0, head = 0;
    CUDA_TRY(cudaMemsetAsync(x, 0, N * sizeof(double), r.st));
    double f = 0.0;
    LIP_TRY(smooth_eval(r, x, g, &f));
    int it = 0, evals = 1;
    for (; it < max_iter; ++it) {
        double gmax = 0.0;
        LIP_TRY(smooth_reduce(r, g, g, 1, &gmax));
        if (gmax <= gtol) break;
        LIP_TRY(smooth_scale(r, q, g, 1.0));
        for (int j = nstore - 1; j >= 0; --j) {
            const int sl = (head + j) % hist;
            double t = 0.0;
            LIP_TRY(smooth_reduce(r, S + (size_t)sl * N, q, 0, &t));
            alpha[sl] = rho[sl] * t;
            LIP_TRY(smooth_axpy(r, q, q, -alpha[sl], Y + (size_t)sl * N));
        }
        double gamma = 1.0;
        if (nstore > 0) {
            const int sl = (head + nstore - 1) % hist;
            double sy = 0.0, yy = 0.0;
            LIP_TRY(smooth_reduce(r, S + (size_t)sl * N, Y + (size_t)sl * N, 0, &sy));
            LIP_TRY(smooth_reduce(r, Y + (size_t)sl * N, Y + (size_t)sl * N, 0, &yy));
            gamma = sy / yy;
        }
        LIP_TRY(smooth_scale(r, q, q, gamma));
        for (int j = 0; j < nstore; ++j) {
            const int sl = (head + j) % hist;
            double t = 0.0;
            LIP_TRY(smooth_reduce(r, Y + (size_t)sl * N, q, 0, &t));
            const double beta = rho[sl] * t;
            LIP_TRY(smooth_axpy(r, q, q, alpha[sl] - beta, S + (size_t)sl * N));
        }
        LIP_TRY(smooth_scale(r, dir, q, -1.0));
        double gd = 0.0;
        LIP_TRY(smooth_reduce(r, g, dir, 0, &gd));
        if (!(gd < 0.0)) {
            LIP_TRY(smooth_scale(r, dir, g, -1.0));
            LIP_TRY(smooth_reduce(r, g, dir, 0, &gd));
            nstore = 0;
        }
        double a = 1.0, fn = f;
        bool ok = false;
        for (int ls = 0; ls < 60; ++ls) {
            LIP_TRY(smooth_axpy(r, xn, x, a, dir));
            LIP_TRY(smooth_eval(r, xn, gn, &fn));
            ++evals;
            if (fn <= f + 1e-4 * a * gd) { ok = true; break; }
            a *= 0.5;
        }
        if (!ok) break;
        LIP_TRY(smooth_axpy(r, q, xn, -1.0, x));        // s
        LIP_TRY(smooth_axpy(r, dir, gn, -1.0, g));      // y
        double sy = 0.0, ss = 0.0, yy = 0.0;
        LIP_TRY(smooth_reduce(r, q, dir, 0, &sy));
        LIP_TRY(smooth_reduce(r, q, q, 0, &ss));
        LIP_TRY(smooth_reduce(r, dir, dir, 0, &yy));
        if (sy > 1e-12 * std::sqrt(ss * yy)) {
            const int sl = nstore < hist ? (head + nstore) % hist : head;
            CUDA_TRY(cudaMemcpyAsync(S + (size_t)sl * N, q, N * sizeof(double), cudaMemcpyDeviceToDevice, r.st));
            CUDA_TRY(cudaMemcpyAsync(Y + (size_t)sl * N, dir, N * sizeof(double), cudaMemcpyDeviceToDevice, r.st));
            rho[sl] = 1.0 / sy;
            if (nstore < hist) ++nstore;
            else head = (head + 1) % hist;
        }
        std::swap(x, xn);
        std::swap(g, gn);
        f = fn;
    }
    *f_out = f;
    *iters_out = it;
    *evals_out = evals;
    *x_out = x;
    return LIP_OK;
}

}  // namespace

extern "C" {

lip_status lip_smooth_objective(lip_handle h, double M, double p, const double* eps, double* f_out, double* grad,
                                void* stream) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (!eps || !f_out) return fail(LIP_ERR_ARG, "eps or f_out is NULL");
    LIP_TRY(smooth_check(h, M, p));
    DeviceGuard g(h->device);
    SmoothRun r;
    LIP_TRY(smooth_setup(h, M, p, static_cast<cudaStream_t>(stream), r));
    return smooth_eval(r, eps, grad, f_out);
}

lip_status lip_smooth(lip_handle h, double M, double p, int32_t max_iter, int32_t history, double gtol,
                      double* eps_out, double* f_out, int32_t* iters_out, int32_t* evals_out, void* stream) {
    if (!h) return fail(LIP_ERR_ARG, "handle is NULL");
    if (max_iter < 0) return fail(LIP_ERR_ARG, "max_iter = %d < 0", max_iter);
    if (history < 1 || history > 64) return fail(LIP_ERR_ARG, "history = %d is outside [1, 64]", history);
    if (!(gtol >= 0.0)) return fail(LIP_ERR_ARG, "gtol = %g must be >= 0", gtol);
    LIP_TRY(smooth_check(h, M, p));
    DeviceGuard g(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SmoothRun r;
    LIP_TRY(smooth_setup(h, M, p, st, r));
    double f = 0.0;
    int iters = 0, evals = 0;
    double* x = nullptr;
    LIP_TRY(smooth_lbfgs(r, max_iter, history, gtol, &f, &iters, &evals, &x));
    if (eps_out) CUDA_TRY(cudaMemcpyAsync(eps_out, x, (size_t)h->N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    // y <- y + eps, M <- the smoothing constant, and the scan layout rebuilt for both
    CUDA_TRY(launch_apply_eps(h->y0, h->esize, x, h->N, st));
    h->s32_dirty = true;
    h->sp_dirty = true;
    h->M = M;
    HotParams hp;
    fill_hot_params(h, hp, 0, h->N);
    CUDA_TRY(launch_build_hot(h->esize, hp, st));
    count_launches(2);
    CUDA_TRY(cudaStreamSynchronize(st));
    h->tc_dirty = true;
    h->loc_valid = false;
    if (f_out) *f_out = f;
    if (iters_out) *iters_out = iters;
    if (evals_out) *evals_out = evals;
    return LIP_OK;
}

}  // extern "C"
