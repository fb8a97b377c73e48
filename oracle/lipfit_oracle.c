/*
 * FP64 brute-force oracle for optimal Lipschitz interpolation.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker that the CUDA library is
 * compared against; only the tests, the package smoke check and the benchmark's
 * CPU-baseline leg may load it.  It shares no code, header, table or constant
 * with the CUDA path and never calls it.
 *
 * Everything is computed in IEEE double with default rounding, by the plain
 * definitions, one (query, datum) pair at a time in increasing datum order:
 *
 *   H_up(x) = min_k ( y^k + M dist_up(x, x^k) )          Sec. 3, Eq. (upperlower)
 *   H_lo(x) = max_k ( y^k - M dist_lo(x, x^k) )          Sec. 3, Eq. (upperlower)
 *   g(x)    = (H_up(x) + H_lo(x)) / 2                    Sec. 3, Eq. (eq:g)
 *
 * Distances (Sec. 3 after Eq. (upperlower); Sec. 4.1 Eq. (distmon)).  For
 * coordinate i let t_i = x_i - x^k_i, negated when the function is decreasing in
 * coordinate i (Sec. 4.1 treats increasing w.l.o.g.; decreasing is the mirror
 * image), then multiplied by the norm weight w_i > 0.  Unconstrained coordinates
 * use t_i in both bounds.  Constrained coordinates use the positive part
 * (t_i)_+ in the upper bound, which makes g(x) <= y^k whenever x precedes x^k,
 * and (-t_i)_+ (that is, |min(t_i,0)|) in the lower bound, which makes
 * g(x) >= y^k whenever x^k precedes x (both stated in Sec. 4.1).
 * dist = L1 / L2 / Linf norm of that vector.
 *
 * Ties: the first strict improvement wins, so the lowest datum index is kept.
 *
 * Lipschitz constant estimate (Sec. 5): M_est = max over i<j of
 * |y^i - y^j| / dist(x^i, x^j) with the symmetric weighted norm (monotonicity
 * plays no role in it).  A pair with dist = 0 and equal y is skipped; dist = 0
 * with unequal y gives +inf.
 *
 * k > 1 neighbours (Sec. 5, extra features): the weighted sums of the k smallest upper
 * bounds and of the k largest lower bounds replace the minimum and the maximum.
 *
 * Gradient of g (piecewise linear, differentiable almost everywhere, Table 1):
 *   dg/dq  = M/2 ( grad_q dist_up(q, x^u) - grad_q dist_lo(q, x^l) )
 *   dg/dy^k = 1/2 sum_q gbar_q ([u_q = k] + [l_q = k])
 *   dg/dM  = 1/2 sum_q gbar_q ( dist_up(q,x^u) - dist_lo(q,x^l) )
 * with u_q, l_q the argmin / argmax of the two envelopes, subgradient 0 at a
 * zero distance, and the lowest coordinate at an Linf argmax tie.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_L1 1
#define OR_L2 2
#define OR_LINF 3

typedef struct {
    const double* X; const double* y; int64_t N; int d; double M; int norm;
    const int8_t* mon; const double* w;
    const double* Q; int64_t q0, q1;
    double *hi, *lo, *g, *gap_up, *gap_lo; int64_t *iu, *il;
} eval_job;

/* The signed, weighted coordinate difference t_i of Eq. (distmon). */
static double coord_diff(const double* q, const double* x, int i, const int8_t* mon, const double* w) {
    double t = q[i] - x[i];
    if (mon && mon[i] < 0) t = -t;
    if (w) t *= w[i];
    return t;
}

/* dist_up (which = +1) or dist_lo (which = -1) between query q and datum x. */
static double oracle_dist(const double* q, const double* x, int d, int norm,
                          const int8_t* mon, const double* w, int which) {
    double acc = 0.0;
    for (int i = 0; i < d; i++) {
        double t = coord_diff(q, x, i, mon, w);
        double v;
        if (mon && mon[i] != 0) v = (which > 0) ? (t > 0 ? t : 0.0) : (t < 0 ? -t : 0.0);
        else v = fabs(t);
        if (norm == OR_L1) acc += v;
        else if (norm == OR_L2) acc += v * v;
        else if (v > acc) acc = v;
    }
    return norm == OR_L2 ? sqrt(acc) : acc;
}

static void* eval_worker(void* arg) {
    eval_job* J = (eval_job*)arg;
    for (int64_t qi = J->q0; qi < J->q1; qi++) {
        const double* q = J->Q + qi * J->d;
        double bu = INFINITY, su = INFINITY, bl = -INFINITY, sl = -INFINITY;
        int64_t ku = -1, kl = -1;
        int bad = 0;
        for (int i = 0; i < J->d; i++) if (!isfinite(q[i])) bad = 1;
        if (!bad) {
            for (int64_t k = 0; k < J->N; k++) {
                const double* x = J->X + k * J->d;
                double vu = J->y[k] + J->M * oracle_dist(q, x, J->d, J->norm, J->mon, J->w, +1);
                double vl = J->y[k] - J->M * oracle_dist(q, x, J->d, J->norm, J->mon, J->w, -1);
                if (vu < bu) { su = bu; bu = vu; ku = k; } else if (vu < su) su = vu;
                if (vl > bl) { sl = bl; bl = vl; kl = k; } else if (vl > sl) sl = vl;
            }
        }
        double hi = bad ? NAN : bu, lo = bad ? NAN : bl;
        if (J->hi) J->hi[qi] = hi;
        if (J->lo) J->lo[qi] = lo;
        if (J->g) J->g[qi] = 0.5 * (hi + lo);
        if (J->iu) J->iu[qi] = ku;
        if (J->il) J->il[qi] = kl;
        if (J->gap_up) J->gap_up[qi] = bad ? NAN : su - bu;
        if (J->gap_lo) J->gap_lo[qi] = bad ? NAN : bl - sl;
    }
    return NULL;
}

static int clamp_threads(int nthreads, int64_t work) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (work < nthreads) nthreads = work > 0 ? (int)work : 1;
    return nthreads;
}

/* Envelopes, midpoint, argmin/argmax and the gap between best and second best. */
int oracle_eval(const double* X, const double* y, int64_t N, int d, double M, int norm,
                const int8_t* mon, const double* w, const double* Q, int64_t nq,
                double* hi, double* lo, double* g, int64_t* iu, int64_t* il,
                double* gap_up, double* gap_lo, int nthreads) {
    if (N < 1 || d < 1 || nq < 0 || norm < 1 || norm > 3) return 1;
    if (nq == 0) return 0;
    nthreads = clamp_threads(nthreads, nq);
    pthread_t th[256];
    eval_job jobs[256];
    for (int t = 0; t < nthreads; t++) {
        eval_job j = {X, y, N, d, M, norm, mon, w, Q, nq * t / nthreads, nq * (t + 1) / nthreads,
                      hi, lo, g, gap_up, gap_lo, iu, il};
        jobs[t] = j;
        pthread_create(&th[t], NULL, eval_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    return 0;
}

/* ------------------------------------------------------------------ M_est (Sec. 5) */

typedef struct {
    const double* X; const double* y; int64_t N; int d; int norm; const double* w;
    int64_t i0, i1;
    double best; int64_t bi, bj;
} est_job;

static double sym_dist(const double* a, const double* b, int d, int norm, const double* w) {
    double acc = 0.0;
    for (int i = 0; i < d; i++) {
        double v = fabs(a[i] - b[i]);
        if (w) v *= w[i];
        if (norm == OR_L1) acc += v;
        else if (norm == OR_L2) acc += v * v;
        else if (v > acc) acc = v;
    }
    return norm == OR_L2 ? sqrt(acc) : acc;
}

static void* est_worker(void* arg) {
    est_job* J = (est_job*)arg;
    double best = -1.0; int64_t bi = -1, bj = -1;
    for (int64_t i = J->i0; i < J->i1; i++) {
        for (int64_t j = i + 1; j < J->N; j++) {
            double dy = fabs(J->y[i] - J->y[j]);
            double dd = sym_dist(J->X + i * J->d, J->X + j * J->d, J->d, J->norm, J->w);
            double r;
            if (dd == 0.0) { if (dy == 0.0) continue; r = INFINITY; }
            else r = dy / dd;
            if (r > best) { best = r; bi = i; bj = j; }
        }
    }
    J->best = best; J->bi = bi; J->bj = bj;
    return NULL;
}

/* Rows are interleaved over threads (row i goes to thread i mod T) to balance the
 * triangle; the per-thread maxima are merged keeping the lowest (i, j) on ties. */
typedef struct { est_job base; int stride, phase; } est_job2;

static void* est_worker2(void* arg) {
    est_job2* J2 = (est_job2*)arg;
    est_job* J = &J2->base;
    double best = -1.0; int64_t bi = -1, bj = -1;
    for (int64_t i = J2->phase; i < J->N; i += J2->stride) {
        for (int64_t j = i + 1; j < J->N; j++) {
            double dy = fabs(J->y[i] - J->y[j]);
            double dd = sym_dist(J->X + i * J->d, J->X + j * J->d, J->d, J->norm, J->w);
            double r;
            if (dd == 0.0) { if (dy == 0.0) continue; r = INFINITY; }
            else r = dy / dd;
            if (r > best) { best = r; bi = i; bj = j; }
        }
    }
    J->best = best; J->bi = bi; J->bj = bj;
    return NULL;
}

int oracle_estimate_M(const double* X, const double* y, int64_t N, int d, int norm,
                      const double* w, double* M_out, int64_t* i_out, int64_t* j_out, int nthreads) {
    if (N < 1 || d < 1 || norm < 1 || norm > 3) return 1;
    nthreads = clamp_threads(nthreads, N);
    pthread_t th[256];
    est_job2 jobs[256];
    for (int t = 0; t < nthreads; t++) {
        est_job2 j = {{X, y, N, d, norm, w, 0, 0, -1.0, -1, -1}, nthreads, t};
        jobs[t] = j;
        pthread_create(&th[t], NULL, est_worker2, &jobs[t]);
    }
    double best = -1.0; int64_t bi = -1, bj = -1;
    for (int t = 0; t < nthreads; t++) {
        pthread_join(th[t], NULL);
        est_job* J = &jobs[t].base;
        if (J->bi < 0) continue;
        if (J->best > best || (J->best == best && (J->bi < bi || (J->bi == bi && J->bj < bj)))) {
            best = J->best; bi = J->bi; bj = J->bj;
        }
    }
    /* No pair with a positive distance or a change in y: the data are constant. */
    *M_out = best < 0 ? 0.0 : best;
    *i_out = bi; *j_out = bj;
    return 0;
}

/* Single-threaded M_est over an explicit row range [i0, i1): the same loop, used for
 * timing a bounded sample of the triangle. */
int oracle_estimate_M_rows(const double* X, const double* y, int64_t N, int d, int norm,
                           const double* w, int64_t i0, int64_t i1,
                           double* M_out, int64_t* i_out, int64_t* j_out) {
    est_job j = {X, y, N, d, norm, w, i0, i1, -1.0, -1, -1};
    est_worker(&j);
    *M_out = j.best; *i_out = j.bi; *j_out = j.bj;
    return 0;
}

/* ------------------------------------------------------------ gradient (Table 1) */

/* d dist / d q_i for the chosen side; out[] gets d entries. */
static void dist_grad(const double* q, const double* x, int d, int norm, const int8_t* mon,
                      const double* w, int which, double* out) {
    double v[64], s[64];
    double acc = 0.0;
    int imax = -1;
    for (int i = 0; i < d; i++) {
        double t = coord_diff(q, x, i, mon, w);
        double sgn_q = ((mon && mon[i] < 0) ? -1.0 : 1.0) * (w ? w[i] : 1.0); /* dt/dq_i */
        double vi, dvi;                                                    /* v_i, dv_i/dt */
        if (mon && mon[i] != 0) {
            if (which > 0) { vi = t > 0 ? t : 0.0; dvi = t > 0 ? 1.0 : 0.0; }
            else           { vi = t < 0 ? -t : 0.0; dvi = t < 0 ? -1.0 : 0.0; }
        } else {
            vi = fabs(t); dvi = t > 0 ? 1.0 : (t < 0 ? -1.0 : 0.0);
        }
        v[i] = vi; s[i] = dvi * sgn_q;
        if (norm == OR_L1) acc += vi;
        else if (norm == OR_L2) acc += vi * vi;
        else if (vi > acc) { acc = vi; imax = i; }
    }
    for (int i = 0; i < d; i++) out[i] = 0.0;
    if (norm == OR_L1) {
        for (int i = 0; i < d; i++) out[i] = s[i];
    } else if (norm == OR_L2) {
        double nrm = sqrt(acc);
        if (nrm > 0) for (int i = 0; i < d; i++) out[i] = s[i] * v[i] / nrm;
    } else {
        if (acc > 0 && imax >= 0) out[imax] = s[imax];
    }
}

int oracle_grad(const double* X, const double* y, int64_t N, int d, double M, int norm,
                const int8_t* mon, const double* w, const double* Q, int64_t nq,
                const int64_t* iu, const int64_t* il, const double* gbar,
                double* grad_Q, double* grad_y, double* grad_M) {
    if (N < 1 || d < 1 || d > 64 || norm < 1 || norm > 3) return 1;
    double gu[64], gl[64];
    double gm = 0.0;
    (void)y;
    for (int64_t qi = 0; qi < nq; qi++) {
        const double* q = Q + qi * d;
        double gb = gbar ? gbar[qi] : 1.0;
        if (iu[qi] < 0 || il[qi] < 0) { if (grad_Q) for (int i = 0; i < d; i++) grad_Q[qi * d + i] = 0; continue; }
        const double* xu = X + iu[qi] * d;
        const double* xl = X + il[qi] * d;
        dist_grad(q, xu, d, norm, mon, w, +1, gu);
        dist_grad(q, xl, d, norm, mon, w, -1, gl);
        if (grad_Q) for (int i = 0; i < d; i++) grad_Q[qi * d + i] = gb * 0.5 * M * (gu[i] - gl[i]);
        if (grad_y) { grad_y[iu[qi]] += 0.5 * gb; grad_y[il[qi]] += 0.5 * gb; }
        gm += 0.5 * gb * (oracle_dist(q, xu, d, norm, mon, w, +1) - oracle_dist(q, xl, d, norm, mon, w, -1));
    }
    if (grad_M) *grad_M = gm;
    return 0;
}

/* ---------------------------------------------- k > 1 neighbours (Sec. 5, extra features) */
/* H_up^k(x) = sum_j wk_j v_(j), v_(1) <= v_(2) <= ... the k smallest of y^i + M dist_up(x, x^i);
 * H_lo^k(x) = sum_j wk_j v_[j], v_[1] >= v_[2] >= ... the k largest of y^i - M dist_lo(x, x^i);
 * g = (H_up^k + H_lo^k) / 2.  The order among equal values is by increasing data index.
 * Selection keeps a sorted list of the best k seen so far, scanning the data in order. */
typedef struct {
    const double* X; const double* y; int64_t N; int d; double M; int norm;
    const int8_t* mon; const double* w; const double* Q; int64_t q0, q1; int k; const double* wk;
    double *hi, *lo, *g; int64_t *iu, *il;
} evalk_job;

static void* evalk_worker(void* arg) {
    evalk_job* J = (evalk_job*)arg;
    double bu[64], bl[64];
    int64_t ku[64], kl[64];
    for (int64_t qi = J->q0; qi < J->q1; qi++) {
        const double* q = J->Q + qi * J->d;
        int nu = 0, nl = 0;
        for (int64_t k = 0; k < J->N; k++) {
            const double* x = J->X + k * J->d;
            double vu = J->y[k] + J->M * oracle_dist(q, x, J->d, J->norm, J->mon, J->w, +1);
            double vl = J->y[k] - J->M * oracle_dist(q, x, J->d, J->norm, J->mon, J->w, -1);
            /* insert vu into the ascending list (after equal values: lower index first) */
            if (nu < J->k || vu < bu[nu - 1]) {
                int p = nu < J->k ? nu++ : J->k - 1;
                while (p > 0 && bu[p - 1] > vu) { bu[p] = bu[p - 1]; ku[p] = ku[p - 1]; p--; }
                bu[p] = vu; ku[p] = k;
            }
            if (nl < J->k || vl > bl[nl - 1]) {
                int p = nl < J->k ? nl++ : J->k - 1;
                while (p > 0 && bl[p - 1] < vl) { bl[p] = bl[p - 1]; kl[p] = kl[p - 1]; p--; }
                bl[p] = vl; kl[p] = k;
            }
        }
        double hu = 0.0, hl = 0.0;
        for (int j = 0; j < J->k; j++) {
            hu += J->wk[j] * (j < nu ? bu[j] : NAN);
            hl += J->wk[j] * (j < nl ? bl[j] : NAN);
            if (J->iu) J->iu[qi * J->k + j] = j < nu ? ku[j] : -1;
            if (J->il) J->il[qi * J->k + j] = j < nl ? kl[j] : -1;
        }
        if (J->hi) J->hi[qi] = hu;
        if (J->lo) J->lo[qi] = hl;
        if (J->g) J->g[qi] = 0.5 * (hu + hl);
    }
    return NULL;
}

int oracle_eval_k(const double* X, const double* y, int64_t N, int d, double M, int norm,
                  const int8_t* mon, const double* w, const double* Q, int64_t nq, int k, const double* wk,
                  double* hi, double* lo, double* g, int64_t* iu, int64_t* il, int nthreads) {
    if (N < 1 || d < 1 || nq < 0 || norm < 1 || norm > 3 || k < 1 || k > 64) return 1;
    if (nq == 0) return 0;
    nthreads = clamp_threads(nthreads, nq);
    pthread_t th[256];
    evalk_job jobs[256];
    for (int t = 0; t < nthreads; t++) {
        evalk_job j = {X, y, N, d, M, norm, mon, w, Q, nq * t / nthreads, nq * (t + 1) / nthreads, k, wk,
                       hi, lo, g, iu, il};
        jobs[t] = j;
        pthread_create(&th[t], NULL, evalk_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    return 0;
}

/* ------------------------------------------------ local Lipschitz constants (Sec. 4.3) */
/*
 * For every datum x^k a non-decreasing step function M_k(t) of the distance t from x^k
 * replaces the global M in Eq. (upperlower):
 *
 *   H_up(x) = min_k ( y^k + M_k(t_k) t_k ),  H_lo(x) = max_k ( y^k - M_k(t_k) t_k ),
 *   t_k = dist(x, x^k) (the symmetric weighted norm).
 *
 * First segment, t in [0, d1_k] with d1_k the distance to the nearest other datum:
 * M_k = F_k = |y^k - y^(1)| / d1_k (the largest such ratio when several data share the
 * nearest distance).  Beyond it, with knots T_1 < ... < T_m common to all data (empirical
 * quantiles of a sample of interpoint distances) and T_{m+1} = +inf: for t in
 * (T_s, T_{s+1}], t > d1_k,
 *
 *   M_k(t) = max { |y^k - y^j| / d_kj : 0 < d_kj <= max(T_{s+1}, d1_k) }.
 *
 * That is the paper's rule (the ratio over the data no farther than the next knot) with
 * the per-datum first knot d1_k in front of the common ones.  Pairs at distance 0
 * (duplicated points) are skipped.  The table holds Mtab_k[s], s = 0..m, the value on
 * segment s (s = the number of knots below t); it is also the value for every t
 * <= T_{s+1} beyond d1_k, so M_k(t) = (t <= d1_k) ? F_k : Mtab_k[#{i : T_i < t}].
 *
 * Knots: S pairs (a_s, b_s) are drawn with SplitMix64 (Steele, Lea and Flood 2014; output
 * c of a generator seeded with `seed` is mix(seed + (c + 1) * 0x9E3779B97F4A7C15)), a_s =
 * out(2s) mod N and b_s = out(2s + 1) mod N.  Their positive distances, sorted, D_(1) <=
 * ... <= D_(S'), give T_i = D_(ceil(i S' / m)), i = 1..m (the inverted-CDF quantile at
 * i/m), with repeated values dropped.
 *
 * Distances here are the symmetric weighted norm of Sec. 5's estimate: |a_i - b_i|
 * times w_i, then summed (L1), squared and summed then square-rooted (L2) or maxed (Linf),
 * in increasing coordinate order.
 */

uint64_t oracle_splitmix64(uint64_t seed, uint64_t c) {
    uint64_t z = seed + (c + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static int cmp_double(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* Monotone coordinates (Sec. 5: values_local(query, model, k) follows the same
 * convention as to monotonicity types as values()): mon, or NULL when no coordinate is
 * constrained, in which case every local function takes the symmetric distance. */
static const int8_t* mono_or_null(const int8_t* mon, int d) {
    if (!mon) return NULL;
    for (int i = 0; i < d; i++) if (mon[i] != 0) return mon;
    return NULL;
}

/* The distance of the local constants between point a and datum b for the bound on side
 * `which`: with monotone coordinates the one-sided distances of Eq. (distmon), dist_up
 * (which = +1, (a - b)_+ on constrained coordinates) or dist_lo (which = -1, (b - a)_+);
 * without them the symmetric distance. */
static double local_dist(const double* a, const double* b, int d, int norm, const int8_t* mon,
                         const double* w, int which) {
    return mon ? oracle_dist(a, b, d, norm, mon, w, which) : sym_dist(a, b, d, norm, w);
}

/* Knots from S sampled pairs; returns the number of distinct knots (<= m), -1 on bad
 * arguments.  pairs_out (2S) and dist_out (S) receive the sample when not NULL. */
int oracle_local_knots(const double* X, int64_t N, int d, int norm, const double* w, const int8_t* mon,
                       uint64_t seed, int64_t S, int m, double* knots_out, int64_t* pairs_out, double* dist_out) {
    if (N < 1 || d < 1 || norm < 1 || norm > 3 || S < 0 || m < 0) return -1;
    mon = mono_or_null(mon, d);
    double* D = (double*)malloc((size_t)(S > 0 ? S : 1) * sizeof(double));
    if (!D) return -1;
    int64_t kept = 0;
    for (int64_t s = 0; s < S; s++) {
        int64_t a = (int64_t)(oracle_splitmix64(seed, 2 * (uint64_t)s) % (uint64_t)N);
        int64_t b = (int64_t)(oracle_splitmix64(seed, 2 * (uint64_t)s + 1) % (uint64_t)N);
        /* with monotone coordinates: the upper-side distance of datum b's pair with a */
        double dd = local_dist(X + a * d, X + b * d, d, norm, mon, w, +1);
        if (pairs_out) { pairs_out[2 * s] = a; pairs_out[2 * s + 1] = b; }
        if (dist_out) dist_out[s] = dd;
        if (dd > 0.0) D[kept++] = dd;
    }
    qsort(D, (size_t)kept, sizeof(double), cmp_double);
    int n = 0;
    if (kept > 0) {
        for (int i = 1; i <= m; i++) {
            int64_t pos = ((int64_t)i * kept + m - 1) / m;      /* ceil(i S' / m), 1-based */
            double v = D[pos - 1];
            if (n == 0 || v > knots_out[n - 1]) knots_out[n++] = v;
        }
    }
    free(D);
    return n;
}

typedef struct {
    const double* X; const double* y; int64_t N; int d; int norm; const double* w; const int8_t* mon;
    const double* T; int m; int64_t k0, k1; const int64_t* rows;
    double *d1, *F, *Mtab;
} ltab_job;

/* Event e of the pair (k, j) for datum k's table: its distance *dd and ratio *r; returns 0
 * when the event does not exist (distance 0).  Without monotone coordinates one event,
 * the symmetric distance with |y^k - y^j| / d.  With them two: the upper bound of datum k
 * at x^j needs M_k(u) u >= y^j - y^k at u = dist_up(x^j, x^k) (event 0, ratio
 * (y^j - y^k)_+ / u), the lower bound needs M_k(l) l >= y^k - y^j at l = dist_lo(x^j, x^k)
 * (event 1, ratio (y^k - y^j)_+ / l). */
static int local_event(const ltab_job* J, int64_t k, int64_t j, int e, double* dd, double* r) {
    const double* xk = J->X + k * J->d;
    const double* xj = J->X + j * J->d;
    if (!J->mon) {
        *dd = sym_dist(xk, xj, J->d, J->norm, J->w);
        if (*dd == 0.0) return 0;
        *r = fabs(J->y[k] - J->y[j]) / *dd;
        return 1;
    }
    *dd = oracle_dist(xj, xk, J->d, J->norm, J->mon, J->w, e == 0 ? +1 : -1);
    if (*dd == 0.0) return 0;
    double dy = e == 0 ? J->y[j] - J->y[k] : J->y[k] - J->y[j];
    *r = (dy > 0.0 ? dy : 0.0) / *dd;
    return 1;
}

static void* ltab_worker(void* arg) {
    ltab_job* J = (ltab_job*)arg;
    const int nev = J->mon ? 2 : 1;
    for (int64_t o = J->k0; o < J->k1; o++) {
        const int64_t k = J->rows ? J->rows[o] : o;       /* datum of output row o */
        double d1 = INFINITY, F = 0.0;
        for (int64_t j = 0; j < J->N; j++)                   /* nearest distance and its ratio */
            for (int e = 0; e < nev; e++) {
                double dd, r;
                if (!local_event(J, k, j, e, &dd, &r)) continue;
                if (dd < d1) { d1 = dd; F = r; }
                else if (dd == d1 && r > F) F = r;
            }
        double* row = J->Mtab + o * (J->m + 1);
        for (int s = 0; s <= J->m; s++) row[s] = F;
        for (int64_t j = 0; j < J->N; j++)                   /* every segment whose knot covers d_kj */
            for (int e = 0; e < nev; e++) {
                double dd, r;
                if (!local_event(J, k, j, e, &dd, &r)) continue;
                for (int s = 0; s <= J->m; s++) {
                    double knot = s < J->m ? J->T[s] : INFINITY;
                    if (dd <= knot && r > row[s]) row[s] = r;
                }
            }
        J->d1[o] = d1;
        J->F[o] = F;
    }
    return NULL;
}

/* d1, F and Mtab [.][m + 1] for knots T [m] (strictly increasing): for every datum
 * (rows = NULL, nrows = N) or for the data rows[0..nrows) only. */
int oracle_local_table_rows(const double* X, const double* y, int64_t N, int d, int norm, const double* w,
                            const int8_t* mon, const double* T, int m, const int64_t* rows, int64_t nrows,
                            double* d1, double* F, double* Mtab, int nthreads) {
    if (N < 1 || d < 1 || norm < 1 || norm > 3 || m < 0 || nrows < 0) return 1;
    mon = mono_or_null(mon, d);
    if (rows)
        for (int64_t o = 0; o < nrows; o++) if (rows[o] < 0 || rows[o] >= N) return 1;
    if (nrows == 0) return 0;
    nthreads = clamp_threads(nthreads, nrows);
    pthread_t th[256];
    ltab_job jobs[256];
    for (int t = 0; t < nthreads; t++) {
        ltab_job j = {X, y, N, d, norm, w, mon, T, m, nrows * t / nthreads, nrows * (t + 1) / nthreads, rows,
                      d1, F, Mtab};
        jobs[t] = j;
        pthread_create(&th[t], NULL, ltab_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    return 0;
}

int oracle_local_table(const double* X, const double* y, int64_t N, int d, int norm, const double* w,
                       const int8_t* mon, const double* T, int m, double* d1, double* F, double* Mtab, int nthreads) {
    return oracle_local_table_rows(X, y, N, d, norm, w, mon, T, m, NULL, N, d1, F, Mtab, nthreads);
}

/* M_k(t) from datum k's table row. */
static double local_M(const double* T, int m, double d1, double F, const double* row, double t) {
    if (t <= d1) return F;
    int s = 0;
    while (s < m && T[s] < t) s++;
    return row[s];
}

typedef struct {
    const double* X; const double* y; int64_t N; int d; int norm; const double* w; const int8_t* mon;
    const double* T; int m; const double *d1, *F, *Mtab;
    const double* Q; int64_t q0, q1; double eta, tau;
    double *hi, *lo, *g; int64_t *iu, *il; int8_t *amb_up, *amb_lo; double *hi_plus, *lo_minus;
} leval_job;

static void* leval_worker(void* arg) {
    leval_job* J = (leval_job*)arg;
    const int d = J->d;
    for (int64_t qi = J->q0; qi < J->q1; qi++) {
        const double* q = J->Q + qi * d;
        int bad = 0;
        for (int i = 0; i < d; i++) if (!isfinite(q[i])) bad = 1;
        double bu = INFINITY, bl = -INFINITY;
        int64_t ku = -1, kl = -1;
        int au = 0, al = 0;
        if (!bad) {
            for (int64_t k = 0; k < J->N; k++) {
                const double* row = J->Mtab + k * (J->m + 1);
                double tu = local_dist(q, J->X + k * d, d, J->norm, J->mon, J->w, +1);
                double tl = J->mon ? local_dist(q, J->X + k * d, d, J->norm, J->mon, J->w, -1) : tu;
                double vu = J->y[k] + local_M(J->T, J->m, J->d1[k], J->F[k], row, tu) * tu;
                double vl = J->y[k] - local_M(J->T, J->m, J->d1[k], J->F[k], row, tl) * tl;
                if (vu < bu) { bu = vu; ku = k; }
                if (vl > bl) { bl = vl; kl = k; }
            }
            /* An evaluation whose distances are off by up to eta, and whose bound values
             * are off by up to tau / 2, may decide a segment differently and pick another
             * datum.  With every constant taken as high as such an error allows,
             * M_k(t + eta), the envelopes are hi_plus and lo_minus.  Datum k can be
             * picked only if its value with its lowest possible constant M_k(t - eta)
             * comes within tau of them (every other datum's value is then at least as
             * unfavourable).  The query is flagged when such a datum's exact value is
             * more than tau from the exact envelope. */
            if (J->eta > 0.0) {
                double hp = INFINITY, lm = -INFINITY;
                for (int64_t k = 0; k < J->N; k++) {
                    const double* row = J->Mtab + k * (J->m + 1);
                    double tu = local_dist(q, J->X + k * d, d, J->norm, J->mon, J->w, +1);
                    double tl = J->mon ? local_dist(q, J->X + k * d, d, J->norm, J->mon, J->w, -1) : tu;
                    double mbu = local_M(J->T, J->m, J->d1[k], J->F[k], row, tu + J->eta);
                    double mbl = local_M(J->T, J->m, J->d1[k], J->F[k], row, tl + J->eta);
                    if (J->y[k] + mbu * tu < hp) hp = J->y[k] + mbu * tu;
                    if (J->y[k] - mbl * tl > lm) lm = J->y[k] - mbl * tl;
                }
                for (int64_t k = 0; k < J->N; k++) {
                    const double* row = J->Mtab + k * (J->m + 1);
                    double tu = local_dist(q, J->X + k * d, d, J->norm, J->mon, J->w, +1);
                    double tl = J->mon ? local_dist(q, J->X + k * d, d, J->norm, J->mon, J->w, -1) : tu;
                    double mtu = local_M(J->T, J->m, J->d1[k], J->F[k], row, tu);
                    double mau = local_M(J->T, J->m, J->d1[k], J->F[k], row, tu - J->eta);
                    double mtl = local_M(J->T, J->m, J->d1[k], J->F[k], row, tl);
                    double mal = local_M(J->T, J->m, J->d1[k], J->F[k], row, tl - J->eta);
                    if (J->y[k] + mau * tu <= hp + J->tau && J->y[k] + mtu * tu > bu + J->tau) au = 1;
                    if (J->y[k] - mal * tl >= lm - J->tau && J->y[k] - mtl * tl < bl - J->tau) al = 1;
                }
                if (J->hi_plus) J->hi_plus[qi] = hp;
                if (J->lo_minus) J->lo_minus[qi] = lm;
            }
        }
        if (J->eta > 0.0 && bad) {
            if (J->hi_plus) J->hi_plus[qi] = NAN;
            if (J->lo_minus) J->lo_minus[qi] = NAN;
        }
        double hi = bad ? NAN : bu, lo = bad ? NAN : bl;
        if (J->hi) J->hi[qi] = hi;
        if (J->lo) J->lo[qi] = lo;
        if (J->g) J->g[qi] = 0.5 * (hi + lo);
        if (J->iu) J->iu[qi] = ku;
        if (J->il) J->il[qi] = kl;
        if (J->amb_up) J->amb_up[qi] = (int8_t)au;
        if (J->amb_lo) J->amb_lo[qi] = (int8_t)al;
    }
    return NULL;
}

/* Envelopes with the local constants; eta > 0 also fills the ambiguity flags and the
 * envelopes with every constant at its highest within eta (hi_plus, lo_minus). */
int oracle_eval_local(const double* X, const double* y, int64_t N, int d, int norm, const double* w,
                      const int8_t* mon, const double* T, int m, const double* d1, const double* F, const double* Mtab,
                      const double* Q, int64_t nq, double eta, double tau, double* hi, double* lo, double* g,
                      int64_t* iu, int64_t* il, int8_t* amb_up, int8_t* amb_lo, double* hi_plus,
                      double* lo_minus, int nthreads) {
    if (N < 1 || d < 1 || nq < 0 || norm < 1 || norm > 3 || m < 0) return 1;
    if (nq == 0) return 0;
    mon = mono_or_null(mon, d);
    nthreads = clamp_threads(nthreads, nq);
    pthread_t th[256];
    leval_job jobs[256];
    for (int t = 0; t < nthreads; t++) {
        leval_job j = {X, y, N, d, norm, w, mon, T, m, d1, F, Mtab, Q, nq * t / nthreads, nq * (t + 1) / nthreads,
                       eta, tau, hi, lo, g, iu, il, amb_up, amb_lo, hi_plus, lo_minus};
        jobs[t] = j;
        pthread_create(&th[t], NULL, leval_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    return 0;
}

/* k > 1 neighbours with the local constants (Sec. 5, values_local(query, model, k)): the
 * weighted sums of the k smallest y^i + M_i(t_i) t_i and of the k largest y^i - M_i(t_i) t_i,
 * equal values in increasing data index, as in oracle_eval_k. */
typedef struct {
    const double* X; const double* y; int64_t N; int d; int norm; const double* w; const int8_t* mon;
    const double* T; int m; const double *d1, *F, *Mtab;
    const double* Q; int64_t q0, q1; int k; const double* wk;
    double *hi, *lo, *g; int64_t *iu, *il;
} levalk_job;

static void* levalk_worker(void* arg) {
    levalk_job* J = (levalk_job*)arg;
    double bu[64], bl[64];
    int64_t ku[64], kl[64];
    for (int64_t qi = J->q0; qi < J->q1; qi++) {
        const double* q = J->Q + qi * J->d;
        int nu = 0, nl = 0, bad = 0;
        for (int i = 0; i < J->d; i++) if (!isfinite(q[i])) bad = 1;
        for (int64_t k = 0; k < J->N && !bad; k++) {
            const double* row = J->Mtab + k * (J->m + 1);
            double tu = local_dist(q, J->X + k * J->d, J->d, J->norm, J->mon, J->w, +1);
            double tl = J->mon ? local_dist(q, J->X + k * J->d, J->d, J->norm, J->mon, J->w, -1) : tu;
            double vu = J->y[k] + local_M(J->T, J->m, J->d1[k], J->F[k], row, tu) * tu;
            double vl = J->y[k] - local_M(J->T, J->m, J->d1[k], J->F[k], row, tl) * tl;
            if (nu < J->k || vu < bu[nu - 1]) {
                int p = nu < J->k ? nu++ : J->k - 1;
                while (p > 0 && bu[p - 1] > vu) { bu[p] = bu[p - 1]; ku[p] = ku[p - 1]; p--; }
                bu[p] = vu; ku[p] = k;
            }
            if (nl < J->k || vl > bl[nl - 1]) {
                int p = nl < J->k ? nl++ : J->k - 1;
                while (p > 0 && bl[p - 1] < vl) { bl[p] = bl[p - 1]; kl[p] = kl[p - 1]; p--; }
                bl[p] = vl; kl[p] = k;
            }
        }
        double hu = 0.0, hl = 0.0;
        for (int j = 0; j < J->k; j++) {
            hu += J->wk[j] * (j < nu ? bu[j] : NAN);
            hl += J->wk[j] * (j < nl ? bl[j] : NAN);
            if (J->iu) J->iu[qi * J->k + j] = j < nu ? ku[j] : -1;
            if (J->il) J->il[qi * J->k + j] = j < nl ? kl[j] : -1;
        }
        if (J->hi) J->hi[qi] = hu;
        if (J->lo) J->lo[qi] = hl;
        if (J->g) J->g[qi] = 0.5 * (hu + hl);
    }
    return NULL;
}

int oracle_eval_local_k(const double* X, const double* y, int64_t N, int d, int norm, const double* w,
                        const int8_t* mon, const double* T, int m, const double* d1, const double* F, const double* Mtab,
                        const double* Q, int64_t nq, int k, const double* wk,
                        double* hi, double* lo, double* g, int64_t* iu, int64_t* il, int nthreads) {
    if (N < 1 || d < 1 || nq < 0 || norm < 1 || norm > 3 || m < 0 || k < 1 || k > 64) return 1;
    if (nq == 0) return 0;
    mon = mono_or_null(mon, d);
    nthreads = clamp_threads(nthreads, nq);
    pthread_t th[256];
    levalk_job jobs[256];
    for (int t = 0; t < nthreads; t++) {
        levalk_job j = {X, y, N, d, norm, w, mon, T, m, d1, F, Mtab, Q, nq * t / nthreads, nq * (t + 1) / nthreads, k, wk,
                        hi, lo, g, iu, il};
        jobs[t] = j;
        pthread_create(&th[t], NULL, levalk_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    return 0;
}

/* The value datum idx[q] gives query q: y + M_k(t + shift) t (side > 0) or
 * y - M_k(t + shift) t, t = dist(q, x^k): shift = 0 is the exact value, shift = -eta or
 * +eta the value with the constant an evaluation off by eta in distance may take. */
int oracle_local_terms(const double* X, const double* y, int64_t N, int d, int norm, const double* w,
                       const int8_t* mon, const double* T, int m, const double* d1, const double* F,
                       const double* Mtab, const double* Q, int64_t nq, const int64_t* idx, int side, double shift,
                       double* out) {
    if (N < 1 || d < 1 || nq < 0 || norm < 1 || norm > 3 || m < 0) return 1;
    mon = mono_or_null(mon, d);
    for (int64_t qi = 0; qi < nq; qi++) {
        int64_t k = idx[qi];
        if (k < 0 || k >= N) { out[qi] = NAN; continue; }
        double t = local_dist(Q + qi * d, X + k * d, d, norm, mon, w, side > 0 ? +1 : -1);
        double Mk = local_M(T, m, d1[k], F[k], Mtab + k * (m + 1), t + shift);
        out[qi] = side > 0 ? y[k] + Mk * t : y[k] - Mk * t;
    }
    return 0;
}

/* ------------------------------------------------ penalty smoothing (Sec. 4.4, Eq. (optim)) */
/*
 * Changes eps to the data values are chosen to minimise
 *
 *   Phi(eps) = (1/p) ||eps||^2
 *            + sum_{i != k} ( (y_i - y_k - M d+_ik - (eps_k - eps_i))_+ )^2        [Eq. (const1)]
 *            + sum_{i != k} ( (y_k - y_i - M d-_ik + eps_k - eps_i)_+ )^2          [Eq. (const2)]
 *
 * Eq. (const1) asks y_i + eps_i <= y_k + eps_k + M d_ik, the condition for the upper bound
 * at x^i to be at least the smoothed value there, so its distance is dist_up(x^i, x^k);
 * Eq. (const2) asks y_i + eps_i >= y_k + eps_k - M d_ik, the lower-bound condition, with
 * dist_lo(x^i, x^k).  Without monotone coordinates both are the symmetric distance.
 * The gradient differentiates each term: a positive part v of const1 adds 2v to
 * dPhi/deps_i and -2v to dPhi/deps_k; one of const2 adds 2v to dPhi/deps_k and -2v to
 * dPhi/deps_i; the first term adds (2/p) eps.
 *
 * The minimiser is found with L-BFGS (Nocedal and Wright, Numerical Optimization, 2nd ed.,
 * Algorithms 7.4 and 7.5): the two-loop recursion with the initial scaling
 * gamma = s'y / y'y of the newest pair, a backtracking line search from step 1 halving the
 * step until the Armijo condition Phi(eps + a d) <= Phi(eps) + 1e-4 a g'd holds, and a pair
 * kept only when s'y > 1e-12 ||s|| ||y||.  It stops when max |g| <= gtol or after max_iter
 * iterations.
 */

int oracle_smooth_objective(const double* X, const double* y, int64_t N, int d, double M, int norm,
                            const int8_t* mon, const double* w, double p, const double* eps,
                            double* f_out, double* grad, double* s1_out, double* s2_out) {
    if (N < 1 || d < 1 || norm < 1 || norm > 3 || !(p > 0)) return 1;
    double s1 = 0.0, s2 = 0.0, e2 = 0.0;
    for (int64_t i = 0; i < N; i++) {
        if (grad) grad[i] = 2.0 / p * eps[i];
        e2 += eps[i] * eps[i];
    }
    for (int64_t i = 0; i < N; i++) {
        const double* xi = X + i * d;
        for (int64_t k = 0; k < N; k++) {
            if (k == i) continue;
            const double* xk = X + k * d;
            double dup = oracle_dist(xi, xk, d, norm, mon, w, +1);
            double dlo = oracle_dist(xi, xk, d, norm, mon, w, -1);
            double v1 = y[i] - y[k] - M * dup - (eps[k] - eps[i]);
            double v2 = y[k] - y[i] - M * dlo + eps[k] - eps[i];
            if (v1 > 0) {
                s1 += v1 * v1;
                if (grad) { grad[i] += 2.0 * v1; grad[k] -= 2.0 * v1; }
            }
            if (v2 > 0) {
                s2 += v2 * v2;
                if (grad) { grad[k] += 2.0 * v2; grad[i] -= 2.0 * v2; }
            }
        }
    }
    if (f_out) *f_out = e2 / p + s1 + s2;
    if (s1_out) *s1_out = s1;
    if (s2_out) *s2_out = s2;
    return 0;
}

/* dPhi/deps_j for the data rows[0..nrows) only: the terms of both sums in which j is the
 * first or the second index, O(N) per row. */
int oracle_smooth_grad_rows(const double* X, const double* y, int64_t N, int d, double M, int norm,
                            const int8_t* mon, const double* w, double p, const double* eps,
                            const int64_t* rows, int64_t nrows, double* out) {
    if (N < 1 || d < 1 || norm < 1 || norm > 3 || !(p > 0)) return 1;
    for (int64_t o = 0; o < nrows; o++) {
        const int64_t j = rows[o];
        if (j < 0 || j >= N) return 1;
        double g = 2.0 / p * eps[j];
        for (int64_t k = 0; k < N; k++) {
            if (k == j) continue;
            const double *xj = X + j * d, *xk = X + k * d;
            /* pair (i = j, k) */
            double v1 = y[j] - y[k] - M * oracle_dist(xj, xk, d, norm, mon, w, +1) - (eps[k] - eps[j]);
            double v2 = y[k] - y[j] - M * oracle_dist(xj, xk, d, norm, mon, w, -1) + eps[k] - eps[j];
            if (v1 > 0) g += 2.0 * v1;
            if (v2 > 0) g -= 2.0 * v2;
            /* pair (i = k, k = j) */
            v1 = y[k] - y[j] - M * oracle_dist(xk, xj, d, norm, mon, w, +1) - (eps[j] - eps[k]);
            v2 = y[j] - y[k] - M * oracle_dist(xk, xj, d, norm, mon, w, -1) + eps[j] - eps[k];
            if (v1 > 0) g -= 2.0 * v1;
            if (v2 > 0) g += 2.0 * v2;
        }
        out[o] = g;
    }
    return 0;
}

static double dotv(const double* a, const double* b, int64_t n) {
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

/* L-BFGS from eps = 0; eps_out [N] receives the minimiser, *f_out Phi there, *iters_out the
 * iterations taken.  hist (1..64) is the number of stored pairs. */
int oracle_smooth(const double* X, const double* y, int64_t N, int d, double M, int norm,
                  const int8_t* mon, const double* w, double p, int max_iter, int hist, double gtol,
                  double* eps_out, double* f_out, int* iters_out) {
    if (N < 1 || d < 1 || norm < 1 || norm > 3 || !(p > 0) || hist < 1 || hist > 64 || max_iter < 0) return 1;
    double* buf = (double*)calloc((size_t)N * (5 + 2 * hist), sizeof(double));
    if (!buf) return 2;
    double *x = eps_out, *g = buf, *dir = buf + N, *xn = buf + 2 * N, *gn = buf + 3 * N, *q = buf + 4 * N;
    double* S = buf + 5 * N;
    double* Y = S + (size_t)hist * N;
    double rho[64], alpha[64];
    int nstore = 0, head = 0;       /* pairs in the ring, index of the oldest */
    for (int64_t i = 0; i < N; i++) x[i] = 0.0;
    double f;
    oracle_smooth_objective(X, y, N, d, M, norm, mon, w, p, x, &f, g, NULL, NULL);
    int it = 0;
    for (; it < max_iter; it++) {
        double gmax = 0.0;
        for (int64_t i = 0; i < N; i++) if (fabs(g[i]) > gmax) gmax = fabs(g[i]);
        if (gmax <= gtol) break;
        /* two-loop recursion: q = H g */
        for (int64_t i = 0; i < N; i++) q[i] = g[i];
        for (int j = nstore - 1; j >= 0; j--) {
            int s = (head + j) % hist;
            alpha[s] = rho[s] * dotv(S + (size_t)s * N, q, N);
            for (int64_t i = 0; i < N; i++) q[i] -= alpha[s] * Y[(size_t)s * N + i];
        }
        double gamma = 1.0;
        if (nstore > 0) {
            int s = (head + nstore - 1) % hist;
            gamma = dotv(S + (size_t)s * N, Y + (size_t)s * N, N) / dotv(Y + (size_t)s * N, Y + (size_t)s * N, N);
        }
        for (int64_t i = 0; i < N; i++) q[i] *= gamma;
        for (int j = 0; j < nstore; j++) {
            int s = (head + j) % hist;
            double beta = rho[s] * dotv(Y + (size_t)s * N, q, N);
            for (int64_t i = 0; i < N; i++) q[i] += S[(size_t)s * N + i] * (alpha[s] - beta);
        }
        for (int64_t i = 0; i < N; i++) dir[i] = -q[i];
        double gd = dotv(g, dir, N);
        if (!(gd < 0)) {            /* not a descent direction: restart from steepest descent */
            for (int64_t i = 0; i < N; i++) dir[i] = -g[i];
            gd = dotv(g, dir, N);
            nstore = 0;
        }
        /* backtracking Armijo line search */
        double a = 1.0, fn = f;
        int ok = 0;
        for (int ls = 0; ls < 60; ls++) {
            for (int64_t i = 0; i < N; i++) xn[i] = x[i] + a * dir[i];
            oracle_smooth_objective(X, y, N, d, M, norm, mon, w, p, xn, &fn, gn, NULL, NULL);
            if (fn <= f + 1e-4 * a * gd) { ok = 1; break; }
            a *= 0.5;
        }
        if (!ok) break;
        /* curvature pair s = xn - x, y = gn - g (in q and dir, free now); stored in the
         * ring, replacing the oldest when full, only if s'y is clearly positive */
        for (int64_t i = 0; i < N; i++) { q[i] = xn[i] - x[i]; dir[i] = gn[i] - g[i]; }
        double sy = dotv(q, dir, N);
        if (sy > 1e-12 * sqrt(dotv(q, q, N) * dotv(dir, dir, N))) {
            int slot = nstore < hist ? (head + nstore) % hist : head;
            for (int64_t i = 0; i < N; i++) { S[(size_t)slot * N + i] = q[i]; Y[(size_t)slot * N + i] = dir[i]; }
            rho[slot] = 1.0 / sy;
            if (nstore < hist) nstore++;
            else head = (head + 1) % hist;
        }
        for (int64_t i = 0; i < N; i++) { x[i] = xn[i]; g[i] = gn[i]; }
        f = fn;
    }
    if (f_out) *f_out = f;
    if (iters_out) *iters_out = it;
    free(buf);
    return 0;
}
