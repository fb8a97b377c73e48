// Local Lipschitz constants (Sec. 4.3): per-datum step functions M_k(t) and the
// evaluation of Eq. (upperlower) with M replaced by M_k(dist(x, x^k)).
//
//   M_k(t) = F_k                   for t <= d1_k (nearest other datum at d1_k, F_k the
//                                  largest |y^k - y^j| / d1_k among those at d1_k)
//   M_k(t) = Mtab_k[#{i : T_i < t}] beyond it, Mtab_k[s] = max(F_k, max |y^k - y^j| / d_kj
//                                  over the data with 0 < d_kj <= T_{s+1}), T_{m+1} = +inf
//
// with the knots T_1 < ... < T_m the inverted-CDF quantiles at i/m of the positive
// distances of S pairs drawn by SplitMix64 (output c of the generator seeded with
// `seed` is mix(seed + (c + 1) * golden gamma); pair s is (out(2s) mod N, out(2s+1) mod N)).
// Distances are the symmetric weighted norm (|x_i - x'_i| * w_i, then L1 / L2 / Linf).
//
// The decisions that pick a table entry (which segment a distance falls in, which
// datum is nearest) are integer outcomes of floating-point comparisons, so the table
// is computed with the exact FP64 distance and ratio of every pair that can matter:
//  * loc_dist64 takes |a_i - b_i|, multiplies by w_i, and sums (L1), sums squares and
//    takes the correctly rounded square root (L2) or maxes (Linf), in coordinate order,
//    every operation a separately rounded IEEE double operation; the ratio is a correctly
//    rounded division.  Any FP64 implementation of those definitions gives the same bits.
//  * The N^2 screen runs in FP32 with a bound |d32 - d64| <= e_rel d32 + e_abs, e_rel =
//    2^-22 (d + 2), e_abs = e_rel * R (R the largest scaled coordinate): the coordinates
//    are scaled and rounded once (2^-24 |w x|), differenced (2^-24 of the difference) and
//    accumulated ((d + 1) roundings), which the factor 4 over 2^-24 covers with room.
//    Segment counts are bounded from the bucket table (seg_up, seg_dn).  The screen keeps,
//    per datum, an upper bound U_k >= d1_k and cumulative lower bounds Lb_k[s] <=
//    Mtab_k[s]; a pair may decide row k only if its distance may be within U_k (a
//    nearest-neighbour candidate) or its ratio may exceed Lb_k at the lowest segment its
//    distance may fall in.  Every other pair is ruled out, and those that are not are
//    recomputed in FP64, so the table is the exact FP64 one.  One scan does both: a pair
//    that passes the test against the running bounds is listed (loc_screen_kernel), and
//    the list is tested again against the final bounds (loc_exact_kernel).
// The evaluation scan runs in FP32 from the same layout; the winners are re-evaluated in
// FP64 with the exact table.
#include "launch.h"

namespace lip {

namespace {

constexpr int LOC_THREADS = 128;
constexpr int LOC_TILE = 128;       // data points per shared-memory tile (table passes)
constexpr int LOC_SCAN_TILE = 64;   // data points per shared-memory tile (evaluation)
constexpr int LOC_RANK_TILE = 1024;
constexpr int LOC_RANK_SLICES = 8;  // slices of the samples per rank count (grid y)
constexpr int LOC_CAND = 64;        // table candidates listed per datum (more: the second scan)
constexpr int LOC_PILOT = 1024;     // strided data that warm the screen's bounds

// Query pairs per thread of the evaluation scan for DP padded coordinates.
constexpr int local_scan_groups(int dp) { return dp <= 4 ? 2 : 1; }

__device__ __forceinline__ int64_t lmin(int64_t a, int64_t b) { return a < b ? a : b; }

__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t c) {
    uint64_t z = seed + (c + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Element i of a float (es = 4) or double (es = 8) array, as a double.
__device__ __forceinline__ double ldv(const void* p, int es, int64_t i) {
    return es == 8 ? static_cast<const double*>(p)[i] : (double)static_cast<const float*>(p)[i];
}

__device__ __forceinline__ void stv(void* p, int es, int64_t i, double v) {
    if (es == 8) static_cast<double*>(p)[i] = v;
    else static_cast<float*>(p)[i] = (float)v;
}

// Exact symmetric distance between rows starting at elements a0 of A and b0 of B: every
// step one IEEE double operation, in coordinate order.
__device__ __forceinline__ double loc_dist64(const void* A, int64_t a0, const void* B, int64_t b0, int es, int d,
                                             int norm, const double* w) {
    double acc = 0.0;
    for (int i = 0; i < d; ++i) {
        const double v = __dmul_rn(fabs(__dsub_rn(ldv(A, es, a0 + i), ldv(B, es, b0 + i))), w[i]);
        if (norm == LIP_L1) acc = __dadd_rn(acc, v);
        else if (norm == LIP_L2) acc = __dadd_rn(acc, __dmul_rn(v, v));
        else if (v > acc) acc = v;
    }
    return norm == LIP_L2 ? __dsqrt_rn(acc) : acc;
}

// Exact one-sided distance (monotone coordinates, Sec. 4.1 Eq. (distmon)) between rows a0
// of A and b0 of B in FP64, every step one IEEE double operation in coordinate order:
// t = a_i - b_i, negated where decreasing, times w_i; then on constrained coordinates the
// side's part (side > 0: max(t, 0) for dist_up; side < 0: max(-t, 0) for dist_lo) and |t|
// elsewhere; summed (L1), squared and summed then square-rooted (L2) or maxed (Linf).
__device__ __forceinline__ double loc_mdist64(const void* A, int64_t a0, const void* B, int64_t b0, int es, int d,
                                              int norm, const double* w, const int8_t* mon, int side) {
    double acc = 0.0;
    for (int i = 0; i < d; ++i) {
        double t = __dsub_rn(ldv(A, es, a0 + i), ldv(B, es, b0 + i));
        if (mon[i] < 0) t = -t;
        t = __dmul_rn(t, w[i]);
        double v;
        if (mon[i] != 0) v = side > 0 ? (t > 0.0 ? t : 0.0) : (t < 0.0 ? -t : 0.0);
        else v = fabs(t);
        if (norm == LIP_L1) acc = __dadd_rn(acc, v);
        else if (norm == LIP_L2) acc = __dadd_rn(acc, __dmul_rn(v, v));
        else if (v > acc) acc = v;
    }
    return norm == LIP_L2 ? __dsqrt_rn(acc) : acc;
}

// FP32 one-sided distances from record a to record b (both mirrored and scaled): with
// t = a_i - b_i, du takes max(t, 0) and dl max(-t, 0) on the constrained coordinates (bits
// of cmask), |t| elsewhere.  The error bound of the symmetric distance holds for both.
template <int NORM, int DP>
__device__ __forceinline__ void mdist32(const float* a, const float* b, unsigned cmask, float& du, float& dl) {
    float au = 0.f, al = 0.f;
#pragma unroll
    for (int i = 0; i < DP; ++i) {
        const float t = a[i] - b[i];
        const bool c = (cmask >> i) & 1u;
        const float u = c ? fmaxf(t, 0.f) : fabsf(t);
        const float l = c ? fmaxf(-t, 0.f) : fabsf(t);
        if (NORM == LIP_L1) { au += u; al += l; }
        else if (NORM == LIP_L2) { au = fmaf(u, u, au); al = fmaf(l, l, al); }
        else { au = fmaxf(au, u); al = fmaxf(al, l); }
    }
    du = NORM == LIP_L2 ? sqrt_approx(au) : au;
    dl = NORM == LIP_L2 ? sqrt_approx(al) : al;
}

// #{i : T[i] < v} for a sorted 32-entry table whose unused tail is +inf.
__device__ __forceinline__ int knot_count(const float* T, float v) {
    int c = 0;
    c += T[c + 15] < v ? 16 : 0;
    c += T[c + 7] < v ? 8 : 0;
    c += T[c + 3] < v ? 4 : 0;
    c += T[c + 1] < v ? 2 : 0;
    c += T[c] < v ? 1 : 0;
    return c;
}

template <int NORM, int DP>
__device__ __forceinline__ float dist32(const float* xk, const float* xj) {
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < DP; ++i) {
        const float t = xk[i] - xj[i];
        if (NORM == LIP_L1) acc += fabsf(t);
        else if (NORM == LIP_L2) acc = fmaf(t, t, acc);
        else acc = fmaxf(acc, fabsf(t));
    }
    return acc;
}

// A bucket entry in 4 bytes: the bits of the knot inside the bucket with the low 5 bits
// replaced by the number of knots below (at most 31).  Read as a float it is the knot moved
// by less than 32 ulp (2^-18 relative, below the FP32 distance error bound the evaluation's
// FP64 merge allows for); with no knot inside (+inf) it is a NaN, so the comparison is
// false.
__device__ __forceinline__ unsigned pack_bucket(int below, float knot) {
    return (__float_as_uint(knot) & ~31u) | (unsigned)below;
}

// #{knots < t} for t in the entry's bucket, from a packed entry.
__device__ __forceinline__ int packed_count(unsigned e, float t) {
    return (int)(e & 31u) + (__uint_as_float(e) < t ? 1 : 0);
}

// Bucket of a non-negative distance for the knot lookup: floor(min(t * scale, NB - 1)),
// monotone in t (the rounding-toward-zero add to 2^23 is the floor for 0 <= u < 2^23).
// A NaN t lands in the last bucket.
__device__ __forceinline__ int knot_bucket(float t, float scale) {
    const float u = fminf(t * scale, (float)(LOC_BUCKETS - 1));
    return __float_as_int(__fadd_rz(u, 8388608.0f)) - 0x4B000000;
}

// ------------------------------------------------------------------ layout

__global__ void loc_layout_kernel(const LocalParams P) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P.npad) return;
    float* r = P.rec + k * P.pr;
    float amax = 0.f;
    if (k < P.N) {
        for (int i = 0; i < P.dp; ++i) {
            // monotone coordinates: mirrored where decreasing (sign * w * x, the product in FP64)
            const double sw = (P.mono && i < P.d && P.mon[i] < 0) ? -P.w[i] : P.w[i];
            const float v = i < P.d ? (float)(sw * ldv(P.X0, P.es, k * P.d + i)) : 0.f;
            r[i] = v;
            amax = fmaxf(amax, fabsf(v));
        }
        r[P.dp] = (float)ldv(P.y0, P.es, k);
    } else {
        for (int i = 0; i < P.dp; ++i) r[i] = 0.f;
        r[P.dp] = __int_as_float(0x7fc00000);         // padding: y = NaN is never selected
    }
    r[P.dp + 1] = INFINITY;
    r[P.dp + 2] = 0.f;
    r[P.dp + 3] = 0.f;
    const unsigned act = __activemask();
    const unsigned m = __reduce_max_sync(act, __float_as_uint(amax));   // |v| orders as its bits
    if ((int)(threadIdx.x & 31) == __ffs(act) - 1) atomicMax(&P.meta->rbits, m);
}

// ------------------------------------------------------------------ knots

__global__ void loc_sample_kernel(const LocalParams P) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= P.S) return;
    const uint64_t a = splitmix64(P.seed, 2 * (uint64_t)s) % (uint64_t)P.N;
    const uint64_t b = splitmix64(P.seed, 2 * (uint64_t)s + 1) % (uint64_t)P.N;
    // with monotone coordinates: the upper-side distance dist_up(x^a, x^b)
    const double dd = P.mono ? loc_mdist64(P.X0, (int64_t)a * P.d, P.X0, (int64_t)b * P.d, P.es, P.d, P.norm, P.w,
                                           P.mon, +1)
                             : loc_dist64(P.X0, (int64_t)a * P.d, P.X0, (int64_t)b * P.d, P.es, P.d, P.norm, P.w);
    P.sample[s] = dd;
    if (dd > 0.0) atomicAdd(&P.meta->npos, 1);
}

// For every sample v, #{u < v} and #{u <= v} over the samples (zeros included), counted over
// LOC_RANK_SLICES slices of the samples (grid y) and added atomically.  Positive doubles
// order as their bit patterns.
__global__ void __launch_bounds__(LOC_THREADS) loc_rank_kernel(const LocalParams P) {
    __shared__ unsigned long long tile[LOC_RANK_TILE];
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long v = s < P.S ? (unsigned long long)__double_as_longlong(P.sample[s]) : 0ull;
    const int64_t span = (P.S + gridDim.y - 1) / gridDim.y;
    const int64_t t_begin = (int64_t)blockIdx.y * span, t_end = lmin(t_begin + span, P.S);
    int lt = 0, le = 0;
    for (int64_t t0 = t_begin; t0 < t_end; t0 += LOC_RANK_TILE) {
        const int n = (int)lmin(LOC_RANK_TILE, t_end - t0);
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x)
            tile[i] = (unsigned long long)__double_as_longlong(P.sample[t0 + i]);
        __syncthreads();
        for (int i = 0; i < n; ++i) {
            const unsigned long long u = tile[i];
            lt += u < v ? 1 : 0;
            le += u <= v ? 1 : 0;
        }
    }
    if (s >= P.S || v == 0ull) return;
    atomicAdd(&P.counts[s], lt);
    atomicAdd(&P.counts[P.S + s], le);
}

// The samples at the quantile positions ceil(i S' / m), i = 1..m, of the positive samples
// (S' of them) into raw[i - 1].  The sample at 0-based position p is any v with
// #{0 < u < v} <= p < #{0 < u <= v}: all such samples are equal, so whichever writes, the
// bits are the same.
__global__ void loc_pick_kernel(const LocalParams P) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= P.S) return;
    const double v = P.sample[s];
    if (!(v > 0.0)) return;
    const int64_t npos = P.meta->npos, nzero = P.S - npos;
    const int64_t lt = P.counts[s] - nzero, le = P.counts[P.S + s] - nzero;
    for (int i = 1; i <= P.m; ++i) {
        const int64_t p = ((int64_t)i * npos + P.m - 1) / P.m - 1;
        if (lt <= p && p < le) P.raw[i - 1] = v;
    }
}

// Distinct knots (raw is non-decreasing) into T64, padded with +inf, and their float
// roundings: to nearest (evaluation), down and up (the screen's bounds).  Then the bucket
// table: bucket b holds the number of knots in lower buckets and the knot inside it (+inf
// if none), packed in 4 bytes (pack_bucket: random per-lane shared loads of 4-byte entries
// conflict about half as often as of 8-byte ones); bucket_ok is cleared if a bucket holds
// two knots.
__global__ void loc_knots_kernel(const LocalParams P, int sampled) {
    if (blockIdx.x != 0) return;
    if (threadIdx.x == 0) {
        int n = 0;
        const int m = (sampled && P.meta->npos == 0) ? 0 : P.m;
        for (int i = 0; i < m; ++i) {
            const double v = P.raw[i];
            if (n == 0 || v > P.T64[n - 1]) P.T64[n++] = v;
        }
        P.meta->m = n;
        for (int i = 0; i < LOC_KNOTS; ++i) {
            const double v = i < n ? P.T64[i] : INFINITY;
            if (i >= n) P.T64[i] = INFINITY;
            P.Tf[i] = __double2float_rn(v);
            P.Tf[LOC_KNOTS + i] = __double2float_rd(v);
            P.Tf[2 * LOC_KNOTS + i] = __double2float_ru(v);
        }
        P.meta->scale = n > 0 ? fminf((float)LOC_BUCKETS / P.Tf[n - 1], 1e30f) : 0.f;
        P.meta->bucket_ok = 1;
    }
    __syncthreads();
    const int n = P.meta->m;
    const float scale = P.meta->scale;
    for (int b = threadIdx.x; b < LOC_BUCKETS; b += blockDim.x) {
        int below = 0, inside = 0;
        float first = INFINITY;
        for (int i = 0; i < n; ++i) {
            const int bi = knot_bucket(P.Tf[i], scale);
            if (bi < b) ++below;
            else if (bi == b) {
                if (inside == 0) first = P.Tf[i];
                ++inside;
            }
        }
        if (inside > 1) atomicExch(&P.meta->bucket_ok, 0);
        P.bpack[b] = pack_bucket(below, first);
    }
}

// ------------------------------------------------------------------ table

// Bounds on the segment index #{i : T_i < v} of an FP64 distance known only to lie in
// [lo, hi], from float data.  With the packed bucket table (no bucket holds two knots):
//  * up(hi) counts the packed table at v = hi (1 + 2^-22).  Each knot T < hi has its
//    nearest float Tn <= T (1 + 2^-24) < v, so it lies in a lower bucket (counted) or in
//    v's bucket, where the packed knot K' <= Tn < v is counted too: up(hi) >= #{T < hi}.
//  * dn(lo) counts it at v = lo (1 - 2^-17).  A knot counted from a lower bucket has
//    Tn < v; the knot inside v's bucket is counted when K' < v, and K' >= Tn (1 - 31 2^-23).
//    Either way T <= Tn (1 + 2^-24) < lo, so dn(lo) <= #{T < lo}.
// Without it (two knots share a bucket), the binary search over the knots rounded down
// (for up) and up (for dn) gives the same bounds.
template <bool BK>
__device__ __forceinline__ int seg_up(const unsigned* bk, const float* Tdn, float scale, float hi) {
    if (BK) {
        const float v = hi * (1.f + 0x1p-22f);
        return packed_count(bk[knot_bucket(v, scale)], v);
    }
    return knot_count(Tdn, hi);
}

template <bool BK>
__device__ __forceinline__ int seg_dn(const unsigned* bk, const float* Tup, float scale, float lo) {
    if (BK) {
        const float v = fmaxf(lo, 0.f) * (1.f - 0x1p-17f);
        return packed_count(bk[knot_bucket(v, scale)], v);
    }
    return knot_count(Tup, lo);
}

// The screen's constants: |d32 - d64| <= e_rel d32 + e_abs, and with FP64 data the float y
// carries 2^-24 |y|, so |dy32 - dy64| <= 2^-22 (|y_k| + |y_j|).
struct ScreenConsts {
    float e_rel, e_abs, up_margin, lo_margin, ey;
};

__device__ __forceinline__ ScreenConsts screen_consts(const LocalParams& P) {
    ScreenConsts c;
    c.e_rel = ldexpf((float)(P.d + 2), -22);
    c.e_abs = c.e_rel * __uint_as_float(P.meta->rbits);
    c.up_margin = 1.f + ldexpf(1.f, -20);
    c.lo_margin = 1.f - ldexpf(1.f, -20);
    c.ey = ldexpf(1.f, -22);
    return c;
}

// Whether the pair (k, j) may decide row k's table given U >= d1_k and the cumulative lower
// bounds Lb[s] <= Mtab_k[s] (stride LOC_THREADS): it may be a (tied) nearest neighbour, or
// its ratio may exceed Lb at the lowest segment its distance may fall in.
template <int NORM, int DP, bool Y64, bool BK>
__device__ __forceinline__ bool table_candidate(const float* xk, float yk, const float* xj, float U, const float* Lb,
                                                const unsigned* bk, const float* Tup, float scale,
                                                const ScreenConsts& c) {
    float d32 = dist32<NORM, DP>(xk, xj);
    if (NORM == LIP_L2) d32 = sqrt_approx(d32);
    const float del = fmaf(c.e_rel, d32, c.e_abs);
    const float lo = d32 - 2.f * del;
    if (lo <= U) return true;
    const int s = seg_dn<BK>(bk, Tup, scale, lo);
    float dy = fabsf(yk - xj[DP]);
    if (Y64) dy += c.ey * (fabsf(yk) + fabsf(xj[DP]));
    return dy * c.up_margin > Lb[s * LOC_THREADS] * lo * c.lo_margin;
}

// Exact FP64 contribution of the pair (k, jj) to row k: nearest distance d1, its ratio F
// (largest among ties) and the per-segment maxima E.
struct ExactRow {
    double d1, F;
    double E[LOC_KNOTS];
};

__device__ __forceinline__ void exact_pair(const LocalParams& P, int64_t k, int64_t jj, double yk64, const double* T64,
                                           int m, ExactRow& r) {
    const double d64 = loc_dist64(P.X0, k * P.d, P.X0, jj * P.d, P.es, P.d, P.norm, P.w);
    if (!(d64 > 0.0)) return;
    const double q = __ddiv_rn(fabs(__dsub_rn(yk64, ldv(P.y0, P.es, jj))), d64);
    if (d64 < r.d1) { r.d1 = d64; r.F = q; }
    else if (d64 == r.d1 && q > r.F) r.F = q;
    int s = 0;
    while (s < m && T64[s] < d64) ++s;
    r.E[s] = fmax(r.E[s], q);
}

template <int PR>
__device__ __forceinline__ void write_row(const LocalParams& P, int64_t k, int m, const ExactRow& r) {
    constexpr int DP = PR - 4;
    P.d1[k] = r.d1;
    P.F[k] = r.F;
    P.rec[k * PR + DP + 1] = (float)r.d1;
    P.rec[k * PR + DP + 2] = (float)r.F;
    double run = r.F;
    for (int s = 0; s < LOC_KNOTS; ++s) {
        if (s <= m) run = fmax(run, r.E[s]);
        P.mt64[k * LOC_KNOTS + s] = run;
        P.mt[k * LOC_KNOTS + s] = (float)run;
    }
}

// Shared memory of the table kernels: the data tile (LOC_TILE points of pr floats), the
// per-thread cumulative lower bounds (nseg segments), the packed bucket table (BK) and the
// knots rounded down and up.  The screen's pair records (pr - 2 float2 per two points) fit
// in the same tile size.
size_t table_smem(int pr, int nseg, bool bk) {
    return ((size_t)LOC_TILE * pr + (size_t)nseg * LOC_THREADS + (bk ? LOC_BUCKETS : 0) + 2 * LOC_KNOTS) *
           sizeof(float);
}

// Running bounds of one datum in the screen: U >= d1_k, and cumulative lower bounds
// Lb_k[s] <= Mtab_k[s], s <= m, in shared memory (stride LOC_THREADS), with copies of
// Lb_k at four coarse segments 0 <= c1 <= c2 <= c3 (about m/4, m/2, 3m/4) in registers.
// coarse() bounds Lb_k at the lowest segment of a distance >= lo from below without a
// lookup: lo above the c-th knot rounded up puts at least c knots below the distance,
// and Lb is non-decreasing.  raise() adds a pair known to be at a positive distance in
// [lo, hi]: U falls to hi, and its ratio lower bound is entered from segment up(hi) on
// (the loop stops at the first entry already at least as large).
struct ScreenRow {
    float U;
    float L0, L1, L2, L3;            // Lb_k[0], Lb_k[c1], Lb_k[c2], Lb_k[c3]
};

struct CoarseKnots {
    int c1, c2, c3;
    float t1, t2, t3;                // knots c1, c2, c3 rounded up (+inf without knots)
};

__device__ __forceinline__ CoarseKnots coarse_knots(const float* Tup, int m) {
    CoarseKnots q;
    q.c1 = m >= 4 ? m / 4 : (m > 0 ? 1 : 0);
    q.c2 = m / 2 > q.c1 ? m / 2 : q.c1;
    q.c3 = 3 * m / 4 > q.c2 ? 3 * m / 4 : q.c2;
    q.t1 = q.c1 > 0 ? Tup[q.c1 - 1] : INFINITY;
    q.t2 = q.c2 > 0 ? Tup[q.c2 - 1] : INFINITY;
    q.t3 = q.c3 > 0 ? Tup[q.c3 - 1] : INFINITY;
    return q;
}

__device__ __forceinline__ float coarse_lb(const ScreenRow& w, const CoarseKnots& q, float lo) {
    float L = w.L0;
    L = lo > q.t1 ? w.L1 : L;
    L = lo > q.t2 ? w.L2 : L;
    L = lo > q.t3 ? w.L3 : L;
    return L;
}

template <bool Y64, bool BK>
__device__ __forceinline__ void screen_raise(float* Ak, int m, const CoarseKnots& q, ScreenRow& w, float hi, float dy,
                                             float yk, float yj, const unsigned* bk, const float* Tdn, float scale,
                                             const ScreenConsts& c) {
    w.U = fminf(w.U, hi);
    const float dyl = Y64 ? fmaxf(dy - c.ey * (fabsf(yk) + fabsf(yj)), 0.f) : dy;
    const float rlo = dyl * rcp_approx(hi) * c.lo_margin;
    if (rlo <= w.L0) return;                                  // Lb[up(hi)] >= Lb[0]
    const int su = seg_up<BK>(bk, Tdn, scale, hi);
    for (int s = su; s <= m; ++s) {
        if (Ak[s * LOC_THREADS] >= rlo) break;
        Ak[s * LOC_THREADS] = rlo;
    }
    w.L0 = Ak[0];
    w.L1 = Ak[q.c1 * LOC_THREADS];
    w.L2 = Ak[q.c2 * LOC_THREADS];
    w.L3 = Ak[q.c3 * LOC_THREADS];
}

// Two data points per shared-memory record, coordinate-interleaved: record p holds
// (x_2p[i], x_2p+1[i]) for i < DP, then (y_2p, y_2p+1) and a zero pad, so that a pair of
// points feeds packed f32x2 instructions.  Points idx(r), r < n; a missing partner (odd n)
// is NaN, which no test passes.
template <int DP>
constexpr int pair_rec() { return DP + 2; }          // float2 per record

template <int DP, typename Idx>
__device__ __forceinline__ void load_pairs(float2* t2, const float* rec, int n, Idx idx) {
    constexpr int PR = DP + 4, W = pair_rec<DP>();
    const float nan = __int_as_float(0x7fc00000);
    const int np = (n + 1) / 2;
    for (int i = threadIdx.x; i < np * W; i += LOC_THREADS) {
        const int p = i / W, c = i % W;
        float2 v = make_float2(0.f, 0.f);
        if (c <= DP) {
            const int r0 = 2 * p, r1 = 2 * p + 1;
            v.x = rec[idx(r0) * PR + c];
            v.y = r1 < n ? rec[idx(r1) * PR + c] : nan;
        }
        t2[i] = v;
    }
}

// Distances from datum k (coordinates duplicated in both halves) to the two points of a
// pair record.
template <int NORM, int DP>
__device__ __forceinline__ float2 dist32x2(const float2 (&xk2)[DP], const float2* x2) {
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < DP; ++i) {
        const float2 t = sub2(xk2[i], x2[i]);
        if (NORM == LIP_L2) acc = fma2(t, t, acc);
        else if (NORM == LIP_L1) acc = make_float2(acc.x + fabsf(t.x), acc.y + fabsf(t.y));
        else acc = make_float2(fmaxf(acc.x, fabsf(t.x)), fmaxf(acc.y, fabsf(t.y)));
    }
    if (NORM == LIP_L2) acc = make_float2(sqrt_approx(acc.x), sqrt_approx(acc.y));
    return acc;
}

// The table's N^2 screen.  A thread owns datum k and keeps the running bounds; a pair that
// passes the screen's test (table_candidate) against them is appended to k's candidate
// list.  The running bounds are never tighter than the final ones (U only falls, Lb only
// rises), so every pair that passes the test against the final bounds is on the list;
// loc_exact_kernel tests the list again against the final bounds and recomputes the
// survivors in FP64.  A pair that fails the test cannot raise the bounds (its ratio lower
// bound is below Lb at its lowest segment), so only candidates update them, and most far
// pairs are rejected against Lb_k at a coarse segment without a lookup.  The bounds are
// first warmed on a pilot of (up to) 1024 strided data, so that fewer pairs of the main scan
// pass against early, loose bounds.  Data points come two at a time (load_pairs): both are
// tested against the same snapshot of the bounds, which is valid since any earlier bounds
// are looser.  Outputs per datum: U, the cumulative Lb, the list length and the list; a
// list longer than LOC_CAND sends the datum to loc_pass2_kernel.
template <int NORM, int DP, bool Y64, bool BK>
__global__ void __launch_bounds__(LOC_THREADS) loc_screen_kernel(const LocalParams P) {
    constexpr int PR = DP + 4, W = pair_rec<DP>();
    const int m = P.meta->m;
    extern __shared__ float4 sm4[];
    float2* t2 = reinterpret_cast<float2*>(sm4);                                 // [LOC_TILE / 2][W]
    float* A = reinterpret_cast<float*>(t2 + LOC_TILE / 2 * W);                  // [m + 1][LOC_THREADS]
    unsigned* bk = reinterpret_cast<unsigned*>(A + (m + 1) * LOC_THREADS);       // [LOC_BUCKETS] if BK
    float* Tdn = reinterpret_cast<float*>(bk + (BK ? LOC_BUCKETS : 0));          // [LOC_KNOTS]
    float* Tup = Tdn + LOC_KNOTS;                                                // [LOC_KNOTS]
    const int tid = threadIdx.x;
    const int64_t k = (int64_t)blockIdx.x * LOC_THREADS + tid;
    const bool valid = k < P.N;
    float2 xk2[DP];
    float yk = 0.f;
#pragma unroll
    for (int i = 0; i < DP; ++i) {
        const float v = valid ? P.rec[k * PR + i] : 0.f;
        xk2[i] = make_float2(v, v);
    }
    if (valid) yk = P.rec[k * PR + DP];
    const float2 yk2 = make_float2(yk, yk);
    float* Ak = A + tid;
    for (int s = 0; s <= m; ++s) Ak[s * LOC_THREADS] = 0.f;
    if (BK)
        for (int b = tid; b < LOC_BUCKETS; b += LOC_THREADS) bk[b] = P.bpack[b];
    if (tid < LOC_KNOTS) {
        Tdn[tid] = P.Tf[LOC_KNOTS + tid];
        Tup[tid] = P.Tf[2 * LOC_KNOTS + tid];
    }
    __syncthreads();
    const float scale = P.meta->scale;
    const ScreenConsts c = screen_consts(P);
    const CoarseKnots q = coarse_knots(Tup, m);
    const float2 erel2 = make_float2(c.e_rel, c.e_rel), eabs2 = make_float2(c.e_abs, c.e_abs);
    const float2 m2 = make_float2(-2.f, -2.f), up2 = make_float2(c.up_margin, c.up_margin);
    const float2 lm2 = make_float2(c.lo_margin, c.lo_margin);
    ScreenRow w;
    w.U = INFINITY;
    w.L0 = w.L1 = w.L2 = w.L3 = 0.f;
    // pilot: bounds only
    const int64_t pn = P.N >= 8 * LOC_PILOT ? LOC_PILOT : P.N / 8;
    const int64_t stride = pn > 0 ? P.N / pn : 1;
    for (int64_t p0 = 0; p0 < pn; p0 += LOC_TILE) {
        const int n = (int)lmin(LOC_TILE, pn - p0);
        __syncthreads();
        load_pairs<DP>(t2, P.rec, n, [&](int row) { return (p0 + row) * stride; });
        __syncthreads();
        if (!valid) continue;
        for (int p = 0; p < (n + 1) / 2; ++p) {
            const float2* x2 = t2 + p * W;
            const float2 d = dist32x2<NORM, DP>(xk2, x2);
            const float2 del = fma2(erel2, d, eabs2), hi = fma2(make_float2(2.f, 2.f), del, d);
            const float2 y2 = x2[DP];
            if (d.x > del.x) screen_raise<Y64, BK>(Ak, m, q, w, hi.x, fabsf(yk - y2.x), yk, y2.x, bk, Tdn, scale, c);
            if (d.y > del.y) screen_raise<Y64, BK>(Ak, m, q, w, hi.y, fabsf(yk - y2.y), yk, y2.y, bk, Tdn, scale, c);
        }
    }
    int* list = P.cand + k * LOC_CAND;
    int cnt = 0;
    for (int64_t j0 = 0; j0 < P.N; j0 += LOC_TILE) {
        const int n = (int)lmin(LOC_TILE, P.N - j0);
        __syncthreads();
        load_pairs<DP>(t2, P.rec, n, [&](int row) { return j0 + row; });
        __syncthreads();
        if (!valid) continue;
#pragma unroll 4
        for (int p = 0; p < (n + 1) / 2; ++p) {
            const float2* x2 = t2 + p * W;
            const float2 d = dist32x2<NORM, DP>(xk2, x2);
            const float2 del = fma2(erel2, d, eabs2);
            const float2 lo = fma2(m2, del, d);
            const float2 y2 = x2[DP];
            float2 dy = sub2(yk2, y2);
            dy = make_float2(fabsf(dy.x), fabsf(dy.y));
            float2 dyu = dy;
            if (Y64) dyu = fma2(make_float2(c.ey, c.ey), make_float2(fabsf(yk) + fabsf(y2.x), fabsf(yk) + fabsf(y2.y)), dy);
            dyu = mul2(dyu, up2);
            const float2 lom = mul2(lo, lm2);
            const float2 Lc = mul2(make_float2(coarse_lb(w, q, lo.x), coarse_lb(w, q, lo.y)), lom);
            // per point: 1 = nearest candidate, 2 = needs the segment test, 0 = rejected
            const int f0 = lo.x <= w.U ? 1 : (dyu.x > Lc.x ? 2 : 0);
            const int f1 = lo.y <= w.U ? 1 : (dyu.y > Lc.y ? 2 : 0);
            if ((f0 | f1) == 0) continue;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int f = e == 0 ? f0 : f1;
                if (f == 0) continue;
                const float lo_e = e == 0 ? lo.x : lo.y;
                bool cand = f == 1;
                if (!cand) {
                    const int sd = seg_dn<BK>(bk, Tup, scale, lo_e);
                    cand = (e == 0 ? dyu.x : dyu.y) > Ak[sd * LOC_THREADS] * (e == 0 ? lom.x : lom.y);
                }
                if (!cand) continue;
                if (cnt < LOC_CAND) list[cnt] = (int)(j0 + 2 * p + e);
                ++cnt;
                const float d_e = e == 0 ? d.x : d.y, del_e = e == 0 ? del.x : del.y;
                const float yj = e == 0 ? y2.x : y2.y;
                if (d_e > del_e)
                    screen_raise<Y64, BK>(Ak, m, q, w, d_e + 2.f * del_e, e == 0 ? dy.x : dy.y, yk, yj, bk, Tdn,
                                          scale, c);
            }
        }
    }
    if (!valid) return;
    P.ubound[k] = w.U;
    P.ncand[k] = cnt;
    for (int s = 0; s < LOC_KNOTS; ++s) P.mt[k * LOC_KNOTS + s] = Ak[(s <= m ? s : m) * LOC_THREADS];
    if (cnt > LOC_CAND) P.over[atomicAdd(&P.meta->n_over, 1)] = (int)k;
    else atomicMax(&P.meta->max_cand, cnt);
}

// The exact table rows of the data whose lists did not overflow: each listed pair is
// tested against the final bounds and, if it passes, recomputed in FP64.
template <int NORM, int DP, bool Y64, bool BK>
__global__ void __launch_bounds__(LOC_THREADS) loc_exact_kernel(const LocalParams P) {
    constexpr int PR = DP + 4;
    __shared__ float Lb[LOC_KNOTS * LOC_THREADS];
    __shared__ double T64[LOC_KNOTS];
    __shared__ float Tup[LOC_KNOTS];
    const int tid = threadIdx.x;
    const int64_t k = (int64_t)blockIdx.x * LOC_THREADS + tid;
    if (tid < LOC_KNOTS) {
        T64[tid] = P.T64[tid];
        Tup[tid] = P.Tf[2 * LOC_KNOTS + tid];
    }
    const bool valid = k < P.N && P.ncand[k] <= LOC_CAND;
    if (valid)
        for (int s = 0; s < LOC_KNOTS; ++s) Lb[s * LOC_THREADS + tid] = P.mt[k * LOC_KNOTS + s];
    __syncthreads();
    if (!valid) return;
    float xk[DP];
#pragma unroll
    for (int i = 0; i < DP; ++i) xk[i] = P.rec[k * PR + i];
    const float yk = P.rec[k * PR + DP], U = P.ubound[k];
    const float scale = P.meta->scale;
    const int m = P.meta->m;
    const ScreenConsts c = screen_consts(P);
    const double yk64 = ldv(P.y0, P.es, k);
    const int cnt = P.ncand[k];
    const int* list = P.cand + k * LOC_CAND;
    ExactRow r;
    r.d1 = INFINITY;
    r.F = 0.0;
    for (int s = 0; s < LOC_KNOTS; ++s) r.E[s] = 0.0;
    for (int i = 0; i < cnt; ++i) {
        const int64_t jj = list[i];
        float xj[PR];
#pragma unroll
        for (int e = 0; e < PR; e += 4) {
            const float4 v = reinterpret_cast<const float4*>(P.rec + jj * PR)[e / 4];
            xj[e] = v.x; xj[e + 1] = v.y; xj[e + 2] = v.z; xj[e + 3] = v.w;
        }
        if (!table_candidate<NORM, DP, Y64, BK>(xk, yk, xj, U, Lb + tid, P.bpack, Tup, scale, c)) continue;
        exact_pair(P, k, jj, yk64, T64, m, r);
    }
    write_row<PR>(P, k, m, r);
}

// The exact table of the data whose candidate lists overflowed: a full N^2 scan per datum
// against its final bounds from loc_screen_kernel, FP64 for the pairs that pass.
template <int NORM, int DP, bool Y64, bool BK>
__global__ void __launch_bounds__(LOC_THREADS) loc_pass2_kernel(const LocalParams P) {
    constexpr int PR = DP + 4;
    if ((int64_t)blockIdx.x * LOC_THREADS >= P.meta->n_over) return;   // the whole block
    extern __shared__ float4 sm4[];
    float* tile = reinterpret_cast<float*>(sm4);
    float* Lb = tile + LOC_TILE * PR;
    unsigned* bk = reinterpret_cast<unsigned*>(Lb + LOC_KNOTS * LOC_THREADS);
    float* Tup = reinterpret_cast<float*>(bk + (BK ? LOC_BUCKETS : 0)) + LOC_KNOTS;
    __shared__ double T64[LOC_KNOTS];
    const int tid = threadIdx.x;
    const int64_t slot = (int64_t)blockIdx.x * LOC_THREADS + tid;
    const bool valid = slot < P.meta->n_over;
    const int64_t k = valid ? P.over[slot] : 0;
    float xk[DP];
    float yk = 0.f, U = 0.f;
#pragma unroll
    for (int i = 0; i < DP; ++i) xk[i] = valid ? P.rec[k * PR + i] : 0.f;
    if (valid) {
        yk = P.rec[k * PR + DP];
        U = P.ubound[k];
        for (int s = 0; s < LOC_KNOTS; ++s) Lb[s * LOC_THREADS + tid] = P.mt[k * LOC_KNOTS + s];
    }
    if (BK)
        for (int b = tid; b < LOC_BUCKETS; b += LOC_THREADS) bk[b] = P.bpack[b];
    if (tid < LOC_KNOTS) {
        Tup[tid] = P.Tf[2 * LOC_KNOTS + tid];
        T64[tid] = P.T64[tid];
    }
    const float scale = P.meta->scale;
    const int m = P.meta->m;
    const ScreenConsts c = screen_consts(P);
    const double yk64 = valid ? ldv(P.y0, P.es, k) : 0.0;
    ExactRow r;
    r.d1 = INFINITY;
    r.F = 0.0;
    for (int s = 0; s < LOC_KNOTS; ++s) r.E[s] = 0.0;
    for (int64_t j0 = 0; j0 < P.N; j0 += LOC_TILE) {
        const int n = (int)lmin(LOC_TILE, P.N - j0);
        __syncthreads();
        const float4* src = reinterpret_cast<const float4*>(P.rec + j0 * PR);
        for (int i = tid; i < n * PR / 4; i += LOC_THREADS) sm4[i] = src[i];
        __syncthreads();
        if (!valid) continue;
        for (int j = 0; j < n; ++j) {
            if (!table_candidate<NORM, DP, Y64, BK>(xk, yk, tile + j * PR, U, Lb + tid, bk, Tup, scale, c)) continue;
            exact_pair(P, k, j0 + j, yk64, T64, m, r);
        }
    }
    if (valid) write_row<PR>(P, k, m, r);
}

// ------------------------------------------------ table with monotone coordinates

// Datum k's two events with point j (Sec. 4.3 with the one-sided distances of Eq. (distmon)):
// its upper bound at x^j needs M_k(u) u >= y^j - y^k at u = dist_up(x^j, x^k), its lower
// bound needs M_k(l) l >= y^k - y^j at l = dist_lo(x^j, x^k).  Event e (0: upper, 1: lower)
// has that distance and the ratio (y^j - y^k)_+ / u or (y^k - y^j)_+ / l.

// Whether one event (FP32 distance d32, ratio numerator bound dy) may decide row k: the
// symmetric screen's test (table_candidate) for that event.
template <bool BK>
__device__ __forceinline__ bool event_candidate(float d32, float dy, float U, const float* Lb, const unsigned* bk,
                                                const float* Tup, float scale, const ScreenConsts& c) {
    const float del = fmaf(c.e_rel, d32, c.e_abs);
    const float lo = d32 - 2.f * del;
    if (lo <= U) return true;
    const int s = seg_dn<BK>(bk, Tup, scale, lo);
    return dy * c.up_margin > Lb[s * LOC_THREADS] * lo * c.lo_margin;
}

// The events' FP32 distances and ratio numerators (upper bounds of the exact ones for the
// candidate test; the raw float differences for raising the bounds).
template <int NORM, int DP, bool Y64>
__device__ __forceinline__ void mono_events(const float* xk, float yk, const float* xj, unsigned cmask,
                                            const ScreenConsts& c, float (&d)[2], float (&dy)[2], float (&dyb)[2]) {
    mdist32<NORM, DP>(xj, xk, cmask, d[0], d[1]);            // t = x^j - x^k
    const float yj = xj[DP];
    dy[0] = fmaxf(yj - yk, 0.f);
    dy[1] = fmaxf(yk - yj, 0.f);
    const float e = Y64 ? c.ey * (fabsf(yk) + fabsf(yj)) : 0.f;
    dyb[0] = dy[0] + e;
    dyb[1] = dy[1] + e;
}

template <int NORM, int DP, bool Y64, bool BK>
__device__ __forceinline__ bool mono_candidate(const float* xk, float yk, const float* xj, unsigned cmask, float U,
                                               const float* Lb, const unsigned* bk, const float* Tup, float scale,
                                               const ScreenConsts& c) {
    float d[2], dy[2], dyb[2];
    mono_events<NORM, DP, Y64>(xk, yk, xj, cmask, c, d, dy, dyb);
    return event_candidate<BK>(d[0], dyb[0], U, Lb, bk, Tup, scale, c) ||
           event_candidate<BK>(d[1], dyb[1], U, Lb, bk, Tup, scale, c);
}

// Both exact FP64 events of the pair (k, jj) into row k.
__device__ __forceinline__ void exact_pair_mono(const LocalParams& P, int64_t k, int64_t jj, double yk64,
                                                const double* T64, int m, ExactRow& r) {
    const double yj64 = ldv(P.y0, P.es, jj);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const double dd = loc_mdist64(P.X0, jj * P.d, P.X0, k * P.d, P.es, P.d, P.norm, P.w, P.mon, e == 0 ? +1 : -1);
        if (!(dd > 0.0)) continue;
        const double dy = e == 0 ? __dsub_rn(yj64, yk64) : __dsub_rn(yk64, yj64);
        const double q = __ddiv_rn(dy > 0.0 ? dy : 0.0, dd);
        if (dd < r.d1) { r.d1 = dd; r.F = q; }
        else if (dd == r.d1 && q > r.F) r.F = q;
        int s = 0;
        while (s < m && T64[s] < dd) ++s;
        r.E[s] = fmax(r.E[s], q);
    }
}

// The N^2 screen with monotone coordinates: as loc_screen_kernel (running bounds, a
// strided pilot, candidate lists), one point at a time, each pair tested and raised as its
// two events.
template <int NORM, int DP, bool Y64, bool BK>
__global__ void __launch_bounds__(LOC_THREADS) loc_screen_mono_kernel(const LocalParams P) {
    constexpr int PR = DP + 4;
    const int m = P.meta->m;
    extern __shared__ float4 sm4[];
    float* tile = reinterpret_cast<float*>(sm4);                                 // [LOC_TILE][PR]
    float* A = tile + LOC_TILE * PR;                                             // [m + 1][LOC_THREADS]
    unsigned* bk = reinterpret_cast<unsigned*>(A + (m + 1) * LOC_THREADS);       // [LOC_BUCKETS] if BK
    float* Tdn = reinterpret_cast<float*>(bk + (BK ? LOC_BUCKETS : 0));          // [LOC_KNOTS]
    float* Tup = Tdn + LOC_KNOTS;                                                // [LOC_KNOTS]
    const int tid = threadIdx.x;
    const int64_t k = (int64_t)blockIdx.x * LOC_THREADS + tid;
    const bool valid = k < P.N;
    float xk[DP];
    float yk = 0.f;
#pragma unroll
    for (int i = 0; i < DP; ++i) xk[i] = valid ? P.rec[k * PR + i] : 0.f;
    if (valid) yk = P.rec[k * PR + DP];
    float* Ak = A + tid;
    for (int s = 0; s <= m; ++s) Ak[s * LOC_THREADS] = 0.f;
    if (BK)
        for (int b = tid; b < LOC_BUCKETS; b += LOC_THREADS) bk[b] = P.bpack[b];
    if (tid < LOC_KNOTS) {
        Tdn[tid] = P.Tf[LOC_KNOTS + tid];
        Tup[tid] = P.Tf[2 * LOC_KNOTS + tid];
    }
    __syncthreads();
    const float scale = P.meta->scale;
    const ScreenConsts c = screen_consts(P);
    const CoarseKnots q = coarse_knots(Tup, m);
    ScreenRow w;
    w.U = INFINITY;
    w.L0 = w.L1 = w.L2 = w.L3 = 0.f;
    // pilot: bounds only
    const int64_t pn = P.N >= 8 * LOC_PILOT ? LOC_PILOT : P.N / 8;
    const int64_t stride = pn > 0 ? P.N / pn : 1;
    for (int64_t p0 = 0; p0 < pn; p0 += LOC_TILE) {
        const int n = (int)lmin(LOC_TILE, pn - p0);
        __syncthreads();
        for (int i = tid; i < n * PR; i += LOC_THREADS) tile[i] = P.rec[((p0 + i / PR) * stride) * PR + i % PR];
        __syncthreads();
        if (!valid) continue;
        for (int j = 0; j < n; ++j) {
            float d[2], dy[2], dyb[2];
            mono_events<NORM, DP, Y64>(xk, yk, tile + j * PR, P.cmask, c, d, dy, dyb);
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float del = fmaf(c.e_rel, d[e], c.e_abs);
                if (d[e] > del)
                    screen_raise<Y64, BK>(Ak, m, q, w, d[e] + 2.f * del, dy[e], yk, tile[j * PR + DP], bk, Tdn, scale,
                                          c);
            }
        }
    }
    int* list = P.cand + k * LOC_CAND;
    int cnt = 0;
    for (int64_t j0 = 0; j0 < P.N; j0 += LOC_TILE) {
        const int n = (int)lmin(LOC_TILE, P.N - j0);
        __syncthreads();
        const float4* src = reinterpret_cast<const float4*>(P.rec + j0 * PR);
        for (int i = tid; i < n * PR / 4; i += LOC_THREADS) sm4[i] = src[i];
        __syncthreads();
        if (!valid) continue;
        for (int j = 0; j < n; ++j) {
            const float* xj = tile + j * PR;
            float d[2], dy[2], dyb[2];
            mono_events<NORM, DP, Y64>(xk, yk, xj, P.cmask, c, d, dy, dyb);
            bool cand[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float del = fmaf(c.e_rel, d[e], c.e_abs);
                const float lo = d[e] - 2.f * del;
                const float lom = lo * c.lo_margin, dyu = dyb[e] * c.up_margin;
                cand[e] = lo <= w.U;
                if (!cand[e] && dyu > coarse_lb(w, q, lo) * lom) {
                    const int sd = seg_dn<BK>(bk, Tup, scale, lo);
                    cand[e] = dyu > Ak[sd * LOC_THREADS] * lom;
                }
            }
            if (!cand[0] && !cand[1]) continue;
            if (cnt < LOC_CAND) list[cnt] = (int)(j0 + j);
            ++cnt;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float del = fmaf(c.e_rel, d[e], c.e_abs);
                if (cand[e] && d[e] > del)
                    screen_raise<Y64, BK>(Ak, m, q, w, d[e] + 2.f * del, dy[e], yk, xj[DP], bk, Tdn, scale, c);
            }
        }
    }
    if (!valid) return;
    P.ubound[k] = w.U;
    P.ncand[k] = cnt;
    for (int s = 0; s < LOC_KNOTS; ++s) P.mt[k * LOC_KNOTS + s] = Ak[(s <= m ? s : m) * LOC_THREADS];
    if (cnt > LOC_CAND) P.over[atomicAdd(&P.meta->n_over, 1)] = (int)k;
    else atomicMax(&P.meta->max_cand, cnt);
}

// Exact rows of the data whose lists did not overflow (monotone coordinates).
template <int NORM, int DP, bool Y64, bool BK>
__global__ void __launch_bounds__(LOC_THREADS) loc_exact_mono_kernel(const LocalParams P) {
    constexpr int PR = DP + 4;
    __shared__ float Lb[LOC_KNOTS * LOC_THREADS];
    __shared__ double T64[LOC_KNOTS];
    __shared__ float Tup[LOC_KNOTS];
    const int tid = threadIdx.x;
    const int64_t k = (int64_t)blockIdx.x * LOC_THREADS + tid;
    if (tid < LOC_KNOTS) {
        T64[tid] = P.T64[tid];
        Tup[tid] = P.Tf[2 * LOC_KNOTS + tid];
    }
    const bool valid = k < P.N && P.ncand[k] <= LOC_CAND;
    if (valid)
        for (int s = 0; s < LOC_KNOTS; ++s) Lb[s * LOC_THREADS + tid] = P.mt[k * LOC_KNOTS + s];
    __syncthreads();
    if (!valid) return;
    float xk[DP];
#pragma unroll
    for (int i = 0; i < DP; ++i) xk[i] = P.rec[k * PR + i];
    const float yk = P.rec[k * PR + DP], U = P.ubound[k];
    const float scale = P.meta->scale;
    const int m = P.meta->m;
    const ScreenConsts c = screen_consts(P);
    const double yk64 = ldv(P.y0, P.es, k);
    const int cnt = P.ncand[k];
    const int* list = P.cand + k * LOC_CAND;
    ExactRow r;
    r.d1 = INFINITY;
    r.F = 0.0;
    for (int s = 0; s < LOC_KNOTS; ++s) r.E[s] = 0.0;
    for (int i = 0; i < cnt; ++i) {
        const int64_t jj = list[i];
        const float* xj = P.rec + jj * PR;
        if (!mono_candidate<NORM, DP, Y64, BK>(xk, yk, xj, P.cmask, U, Lb + tid, P.bpack, Tup, scale, c)) continue;
        exact_pair_mono(P, k, jj, yk64, T64, m, r);
    }
    write_row<PR>(P, k, m, r);
}

// Exact rows of the data whose lists overflowed (monotone coordinates): a full scan
// against the final bounds.
template <int NORM, int DP, bool Y64, bool BK>
__global__ void __launch_bounds__(LOC_THREADS) loc_pass2_mono_kernel(const LocalParams P) {
    constexpr int PR = DP + 4;
    if ((int64_t)blockIdx.x * LOC_THREADS >= P.meta->n_over) return;   // the whole block
    extern __shared__ float4 sm4[];
    float* tile = reinterpret_cast<float*>(sm4);
    float* Lb = tile + LOC_TILE * PR;
    unsigned* bk = reinterpret_cast<unsigned*>(Lb + LOC_KNOTS * LOC_THREADS);
    float* Tup = reinterpret_cast<float*>(bk + (BK ? LOC_BUCKETS : 0)) + LOC_KNOTS;
    __shared__ double T64[LOC_KNOTS];
    const int tid = threadIdx.x;
    const int64_t slot = (int64_t)blockIdx.x * LOC_THREADS + tid;
    const bool valid = slot < P.meta->n_over;
    const int64_t k = valid ? P.over[slot] : 0;
    float xk[DP];
    float yk = 0.f, U = 0.f;
#pragma unroll
    for (int i = 0; i < DP; ++i) xk[i] = valid ? P.rec[k * PR + i] : 0.f;
    if (valid) {
        yk = P.rec[k * PR + DP];
        U = P.ubound[k];
        for (int s = 0; s < LOC_KNOTS; ++s) Lb[s * LOC_THREADS + tid] = P.mt[k * LOC_KNOTS + s];
    }
    if (BK)
        for (int b = tid; b < LOC_BUCKETS; b += LOC_THREADS) bk[b] = P.bpack[b];
    if (tid < LOC_KNOTS) {
        Tup[tid] = P.Tf[2 * LOC_KNOTS + tid];
        T64[tid] = P.T64[tid];
    }
    const float scale = P.meta->scale;
    const int m = P.meta->m;
    const ScreenConsts c = screen_consts(P);
    const double yk64 = valid ? ldv(P.y0, P.es, k) : 0.0;
    ExactRow r;
    r.d1 = INFINITY;
    r.F = 0.0;
    for (int s = 0; s < LOC_KNOTS; ++s) r.E[s] = 0.0;
    for (int64_t j0 = 0; j0 < P.N; j0 += LOC_TILE) {
        const int n = (int)lmin(LOC_TILE, P.N - j0);
        __syncthreads();
        const float4* src = reinterpret_cast<const float4*>(P.rec + j0 * PR);
        for (int i = tid; i < n * PR / 4; i += LOC_THREADS) sm4[i] = src[i];
        __syncthreads();
        if (!valid) continue;
        for (int j = 0; j < n; ++j) {
            if (!mono_candidate<NORM, DP, Y64, BK>(xk, yk, tile + j * PR, P.cmask, U, Lb + tid, bk, Tup, scale, c))
                continue;
            exact_pair_mono(P, k, j0 + j, yk64, T64, m, r);
        }
    }
    if (valid) write_row<PR>(P, k, m, r);
}

// ------------------------------------------------------------------ evaluation

// The two queries a thread holds share every instruction that can be packed: their
// coordinates sit in the two halves of float2 registers, so the distance to a data point,
// the bucket scaling and both bound values are f32x2 operations.  The hot loop keeps only
// the running extrema (one min and one max per pair); the 64-point tile in which each
// query's extremum last strictly improved is remembered, and after the scan that tile is
// evaluated again by the same inlined function, from global memory, to recover the lowest
// index whose value equals the extremum bit for bit.
template <int NORM, int DP, bool BUCKET>
__device__ __forceinline__ void loc_pair_values(const float2 (&q2)[DP], const float* xj, const float* mtj,
                                                const unsigned* bk, const float* Tn, float scale, float2& vu,
                                                float2& vl) {
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < DP; ++i) {
        const float2 t = sub2(q2[i], make_float2(xj[i], xj[i]));
        if (NORM == LIP_L2) acc = fma2(t, t, acc);
        else if (NORM == LIP_L1) acc = make_float2(__fadd_rn(acc.x, fabsf(t.x)), __fadd_rn(acc.y, fabsf(t.y)));
        else acc = make_float2(fmaxf(acc.x, fabsf(t.x)), fmaxf(acc.y, fabsf(t.y)));
    }
    float2 t = acc;
    if (NORM == LIP_L2) t = make_float2(sqrt_approx(acc.x), sqrt_approx(acc.y));
    int s0, s1;
    if (BUCKET) {
        const float2 u = mul2(t, make_float2(scale, scale));
        const int b0 = __float_as_int(__fadd_rz(fminf(u.x, (float)(LOC_BUCKETS - 1)), 8388608.0f)) - 0x4B000000;
        const int b1 = __float_as_int(__fadd_rz(fminf(u.y, (float)(LOC_BUCKETS - 1)), 8388608.0f)) - 0x4B000000;
        s0 = packed_count(bk[b0], t.x);
        s1 = packed_count(bk[b1], t.y);
    } else {
        s0 = knot_count(Tn, t.x);
        s1 = knot_count(Tn, t.y);
    }
    const float y = xj[DP], d1 = xj[DP + 1], Fj = xj[DP + 2];
    const float2 M = make_float2(t.x <= d1 ? Fj : mtj[s0], t.y <= d1 ? Fj : mtj[s1]);
    const float2 y2 = make_float2(y, y);
    vu = fma2(M, t, y2);
    vl = fma2(make_float2(-M.x, -M.y), t, y2);
}

// G groups of two queries per thread (G = 2 for d <= 4: the data point's loads and the loop
// are shared by four queries).
template <int NORM, int DP, bool BUCKET, int G>
__global__ void __launch_bounds__(LOC_THREADS) loc_scan_kernel(const LocalScanParams P) {
    constexpr int PR = DP + 4;
    __shared__ float4 rec4[LOC_SCAN_TILE * PR / 4];
    __shared__ float4 mt4[LOC_SCAN_TILE * LOC_KNOTS / 4];
    __shared__ unsigned bk[BUCKET ? LOC_BUCKETS : 1];
    __shared__ float Tn[LOC_KNOTS];
    const float* rec = reinterpret_cast<const float*>(rec4);
    const float* mt = reinterpret_cast<const float*>(mt4);
    const int tid = threadIdx.x;
    const int split = blockIdx.y;
    float2 q2[G][DP];
    int64_t qi[G][2];
#pragma unroll
    for (int g = 0; g < G; ++g) {
#pragma unroll
        for (int h = 0; h < 2; ++h) qi[g][h] = (int64_t)blockIdx.x * LOC_THREADS * 2 * G + (2 * g + h) * LOC_THREADS + tid;
#pragma unroll
        for (int i = 0; i < DP; ++i) {
            const float a = (qi[g][0] < P.nq && i < P.d) ? (float)(P.w[i] * ldv(P.Q, P.es, qi[g][0] * P.d + i)) : 0.f;
            const float b = (qi[g][1] < P.nq && i < P.d) ? (float)(P.w[i] * ldv(P.Q, P.es, qi[g][1] * P.d + i)) : 0.f;
            q2[g][i] = make_float2(a, b);
        }
    }
    if (BUCKET) {
        for (int b = tid; b < LOC_BUCKETS; b += LOC_THREADS) bk[b] = P.bpack[b];
    } else if (tid < LOC_KNOTS) {
        Tn[tid] = P.Tf[tid];
    }
    const float scale = P.scale;
    float2 bu[G], bl[G];
    int tu[G][2], tl[G][2];                                   // tile of the last strict improvement
#pragma unroll
    for (int g = 0; g < G; ++g) {
        bu[g] = make_float2(INFINITY, INFINITY);
        bl[g] = make_float2(-INFINITY, -INFINITY);
        tu[g][0] = tu[g][1] = tl[g][0] = tl[g][1] = -1;
    }
    const int64_t j_begin = (int64_t)split * P.points_per_split;
    const int64_t j_end = lmin(j_begin + P.points_per_split, P.npad);
    for (int64_t j0 = j_begin; j0 < j_end; j0 += LOC_SCAN_TILE) {
        __syncthreads();
        const float4* rs = reinterpret_cast<const float4*>(P.rec + j0 * PR);
        for (int i = tid; i < LOC_SCAN_TILE * PR / 4; i += LOC_THREADS) rec4[i] = rs[i];
        const float4* ms = reinterpret_cast<const float4*>(P.mt + j0 * LOC_KNOTS);
        for (int i = tid; i < LOC_SCAN_TILE * LOC_KNOTS / 4; i += LOC_THREADS) mt4[i] = ms[i];
        __syncthreads();
        float2 cu[G], cl[G];
#pragma unroll
        for (int g = 0; g < G; ++g) { cu[g] = bu[g]; cl[g] = bl[g]; }
        // two data points per step, folded with the three-input min / max (NaN, i.e.
        // padding, is ignored)
        for (int j = 0; j < LOC_SCAN_TILE; j += 2) {
#pragma unroll
            for (int g = 0; g < G; ++g) {
                float2 vu0, vl0, vu1, vl1;
                loc_pair_values<NORM, DP, BUCKET>(q2[g], rec + j * PR, mt + j * LOC_KNOTS, bk, Tn, scale, vu0, vl0);
                loc_pair_values<NORM, DP, BUCKET>(q2[g], rec + (j + 1) * PR, mt + (j + 1) * LOC_KNOTS, bk, Tn, scale,
                                                  vu1, vl1);
                cu[g] = make_float2(min3f(cu[g].x, vu0.x, vu1.x), min3f(cu[g].y, vu0.y, vu1.y));
                cl[g] = make_float2(max3f(cl[g].x, vl0.x, vl1.x), max3f(cl[g].y, vl0.y, vl1.y));
            }
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (cu[g].x < bu[g].x) tu[g][0] = (int)j0;
            if (cu[g].y < bu[g].y) tu[g][1] = (int)j0;
            if (cl[g].x > bl[g].x) tl[g][0] = (int)j0;
            if (cl[g].y > bl[g].y) tl[g][1] = (int)j0;
            bu[g] = cu[g];
            bl[g] = cl[g];
        }
    }
    // lowest index in the remembered tile whose value equals the extremum
    PartialRec<float>* part = static_cast<PartialRec<float>*>(P.partial);
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int tiles[4] = {tu[g][0], tu[g][1], tl[g][0], tl[g][1]};
        int idx[4] = {-1, -1, -1, -1};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (tiles[c] < 0) continue;
            const float target = c == 0 ? bu[g].x : (c == 1 ? bu[g].y : (c == 2 ? bl[g].x : bl[g].y));
            for (int j = 0; j < LOC_SCAN_TILE; ++j) {
                const int64_t k = (int64_t)tiles[c] + j;
                float2 vu, vl;
                loc_pair_values<NORM, DP, BUCKET>(q2[g], P.rec + k * PR, P.mt + k * LOC_KNOTS, bk, Tn, scale, vu, vl);
                const float v = c == 0 ? vu.x : (c == 1 ? vu.y : (c == 2 ? vl.x : vl.y));
                if (v == target) { idx[c] = (int)k; break; }
            }
        }
        if (qi[g][0] < P.nq) {
            PartialRec<float> rr;
            rr.vu = bu[g].x; rr.iu = idx[0]; rr.vl = bl[g].x; rr.il = idx[2];
            part[(int64_t)split * P.nq + qi[g][0]] = rr;
        }
        if (qi[g][1] < P.nq) {
            PartialRec<float> rr;
            rr.vu = bu[g].y; rr.iu = idx[1]; rr.vl = bl[g].y; rr.il = idx[3];
            part[(int64_t)split * P.nq + qi[g][1]] = rr;
        }
    }
}

// ------------------------------------------------ k > 1 neighbours with local constants

// One query per thread; sorted lists of the K best upper and lower values per split, with
// strict comparisons so equal values stay in data-index order (the scan visits the data in
// increasing index).  The segment lookup is the bucket table or, when a bucket holds two
// knots, the binary search.
template <int NORM, int DP, int K>
__global__ void __launch_bounds__(LOC_THREADS) loc_topk_scan_kernel(const LocalScanParams P, int K_out) {
    constexpr int PR = DP + 4;
    __shared__ float4 rec4[LOC_SCAN_TILE * PR / 4];
    __shared__ float4 mt4[LOC_SCAN_TILE * LOC_KNOTS / 4];
    __shared__ unsigned bk[LOC_BUCKETS];
    __shared__ float Tn[LOC_KNOTS];
    const float* rec = reinterpret_cast<const float*>(rec4);
    const float* mt = reinterpret_cast<const float*>(mt4);
    const int tid = threadIdx.x;
    const int split = blockIdx.y;
    const int64_t qi = (int64_t)blockIdx.x * LOC_THREADS + tid;
    float q[DP];
#pragma unroll
    for (int i = 0; i < DP; ++i) q[i] = (qi < P.nq && i < P.d) ? (float)(P.w[i] * ldv(P.Q, P.es, qi * P.d + i)) : 0.f;
    for (int b = tid; b < LOC_BUCKETS; b += LOC_THREADS) bk[b] = P.bpack[b];
    if (tid < LOC_KNOTS) Tn[tid] = P.Tf[tid];
    const float scale = P.scale;
    const bool bucket = P.bucket_ok != 0;
    float bu[K], bl[K];
    int ku[K], kl[K];
#pragma unroll
    for (int e = 0; e < K; ++e) { bu[e] = INFINITY; bl[e] = -INFINITY; ku[e] = -1; kl[e] = -1; }
    const int64_t j_begin = (int64_t)split * P.points_per_split;
    const int64_t j_end = lmin(j_begin + P.points_per_split, P.npad);
    for (int64_t j0 = j_begin; j0 < j_end; j0 += LOC_SCAN_TILE) {
        __syncthreads();
        const float4* rs = reinterpret_cast<const float4*>(P.rec + j0 * PR);
        for (int i = tid; i < LOC_SCAN_TILE * PR / 4; i += LOC_THREADS) rec4[i] = rs[i];
        const float4* ms = reinterpret_cast<const float4*>(P.mt + j0 * LOC_KNOTS);
        for (int i = tid; i < LOC_SCAN_TILE * LOC_KNOTS / 4; i += LOC_THREADS) mt4[i] = ms[i];
        __syncthreads();
        for (int j = 0; j < LOC_SCAN_TILE; ++j) {
            const float* xj = rec + j * PR;
            float t = dist32<NORM, DP>(q, xj);
            if (NORM == LIP_L2) t = sqrt_approx(t);
            int s;
            if (bucket) {
                s = packed_count(bk[knot_bucket(t, scale)], t);
            } else {
                s = knot_count(Tn, t);
            }
            const float M = t <= xj[DP + 1] ? xj[DP + 2] : mt[j * LOC_KNOTS + s];
            float vu = fmaf(M, t, xj[DP]), vl = fmaf(-M, t, xj[DP]);   // NaN (padding) never enters
            const int idx = (int)(j0 + j);
            if (vu < bu[K - 1]) {
                int kk = idx;
#pragma unroll
                for (int p = 0; p < K; ++p)
                    if (vu < bu[p]) {
                        const float tv = bu[p]; bu[p] = vu; vu = tv;
                        const int tk = ku[p]; ku[p] = kk; kk = tk;
                    }
            }
            if (vl > bl[K - 1]) {
                int kk = idx;
#pragma unroll
                for (int p = 0; p < K; ++p)
                    if (vl > bl[p]) {
                        const float tv = bl[p]; bl[p] = vl; vl = tv;
                        const int tk = kl[p]; kl[p] = kk; kk = tk;
                    }
            }
        }
    }
    if (qi >= P.nq) return;
    float* pv = static_cast<float*>(P.partial);
    int* pk = reinterpret_cast<int*>(pv + (int64_t)gridDim.y * P.nq * 2 * K);
    const int64_t base = ((int64_t)split * P.nq + qi) * 2 * K;
#pragma unroll
    for (int e = 0; e < K; ++e) {
        pv[base + e] = bu[e];
        pk[base + e] = ku[e];
        pv[base + K + e] = bl[e];
        pk[base + K + e] = kl[e];
    }
    (void)K_out;
}

// ------------------------------------------------ evaluation with monotone coordinates

// The segment of a non-negative FP32 distance: the packed bucket table, or the binary
// search over the knots when a bucket holds two of them.
__device__ __forceinline__ int loc_segment(float t, bool bucket, const unsigned* bk, const float* Tn, float scale) {
    return bucket ? packed_count(bk[knot_bucket(t, scale)], t) : knot_count(Tn, t);
}

// Bound values of query q (mirrored and scaled) against record xj with its table row: the
// upper with M_j(dist_up(q, x^j)), the lower with M_j(dist_lo(q, x^j)).
template <int NORM, int DP>
__device__ __forceinline__ void mono_values(const float* q, const float* xj, const float* mtj, unsigned cmask,
                                            bool bucket, const unsigned* bk, const float* Tn, float scale, float& vu,
                                            float& vl) {
    float tu, tl;
    mdist32<NORM, DP>(q, xj, cmask, tu, tl);                 // t = q - x^j
    const float y = xj[DP], d1 = xj[DP + 1], Fj = xj[DP + 2];
    const float Mu = tu <= d1 ? Fj : mtj[loc_segment(tu, bucket, bk, Tn, scale)];
    const float Ml = tl <= d1 ? Fj : mtj[loc_segment(tl, bucket, bk, Tn, scale)];
    vu = fmaf(Mu, tu, y);
    vl = fmaf(-Ml, tl, y);                                    // NaN (padding) never enters
}

// One query per thread; the running extrema with their indices (strict comparisons, so the
// lowest index on ties), per data split.
template <int NORM, int DP>
__global__ void __launch_bounds__(LOC_THREADS) loc_scan_mono_kernel(const LocalScanParams P) {
    constexpr int PR = DP + 4;
    __shared__ float4 rec4[LOC_SCAN_TILE * PR / 4];
    __shared__ float4 mt4[LOC_SCAN_TILE * LOC_KNOTS / 4];
    __shared__ unsigned bk[LOC_BUCKETS];
    __shared__ float Tn[LOC_KNOTS];
    const float* rec = reinterpret_cast<const float*>(rec4);
    const float* mt = reinterpret_cast<const float*>(mt4);
    const int tid = threadIdx.x;
    const int split = blockIdx.y;
    const int64_t qi = (int64_t)blockIdx.x * LOC_THREADS + tid;
    float q[DP];
#pragma unroll
    for (int i = 0; i < DP; ++i) q[i] = (qi < P.nq && i < P.d) ? (float)(P.w[i] * ldv(P.Q, P.es, qi * P.d + i)) : 0.f;
    for (int b = tid; b < LOC_BUCKETS; b += LOC_THREADS) bk[b] = P.bpack[b];
    if (tid < LOC_KNOTS) Tn[tid] = P.Tf[tid];
    const float scale = P.scale;
    const bool bucket = P.bucket_ok != 0;
    float bu = INFINITY, bl = -INFINITY;
    int iu = -1, il = -1;
    const int64_t j_begin = (int64_t)split * P.points_per_split;
    const int64_t j_end = lmin(j_begin + P.points_per_split, P.npad);
    for (int64_t j0 = j_begin; j0 < j_end; j0 += LOC_SCAN_TILE) {
        __syncthreads();
        const float4* rs = reinterpret_cast<const float4*>(P.rec + j0 * PR);
        for (int i = tid; i < LOC_SCAN_TILE * PR / 4; i += LOC_THREADS) rec4[i] = rs[i];
        const float4* ms = reinterpret_cast<const float4*>(P.mt + j0 * LOC_KNOTS);
        for (int i = tid; i < LOC_SCAN_TILE * LOC_KNOTS / 4; i += LOC_THREADS) mt4[i] = ms[i];
        __syncthreads();
        for (int j = 0; j < LOC_SCAN_TILE; ++j) {
            float vu, vl;
            mono_values<NORM, DP>(q, rec + j * PR, mt + j * LOC_KNOTS, P.cmask, bucket, bk, Tn, scale, vu, vl);
            if (vu < bu) { bu = vu; iu = (int)(j0 + j); }
            if (vl > bl) { bl = vl; il = (int)(j0 + j); }
        }
    }
    if (qi >= P.nq) return;
    PartialRec<float> rr;
    rr.vu = bu; rr.iu = iu; rr.vl = bl; rr.il = il;
    static_cast<PartialRec<float>*>(P.partial)[(int64_t)split * P.nq + qi] = rr;
}

// k > 1 neighbours with monotone coordinates: the sorted K-lists of loc_topk_scan_kernel
// over the one-sided bound values.
template <int NORM, int DP, int K>
__global__ void __launch_bounds__(LOC_THREADS) loc_topk_scan_mono_kernel(const LocalScanParams P) {
    constexpr int PR = DP + 4;
    __shared__ float4 rec4[LOC_SCAN_TILE * PR / 4];
    __shared__ float4 mt4[LOC_SCAN_TILE * LOC_KNOTS / 4];
    __shared__ unsigned bk[LOC_BUCKETS];
    __shared__ float Tn[LOC_KNOTS];
    const float* rec = reinterpret_cast<const float*>(rec4);
    const float* mt = reinterpret_cast<const float*>(mt4);
    const int tid = threadIdx.x;
    const int split = blockIdx.y;
    const int64_t qi = (int64_t)blockIdx.x * LOC_THREADS + tid;
    float q[DP];
#pragma unroll
    for (int i = 0; i < DP; ++i) q[i] = (qi < P.nq && i < P.d) ? (float)(P.w[i] * ldv(P.Q, P.es, qi * P.d + i)) : 0.f;
    for (int b = tid; b < LOC_BUCKETS; b += LOC_THREADS) bk[b] = P.bpack[b];
    if (tid < LOC_KNOTS) Tn[tid] = P.Tf[tid];
    const float scale = P.scale;
    const bool bucket = P.bucket_ok != 0;
    float bu[K], bl[K];
    int ku[K], kl[K];
#pragma unroll
    for (int e = 0; e < K; ++e) { bu[e] = INFINITY; bl[e] = -INFINITY; ku[e] = -1; kl[e] = -1; }
    const int64_t j_begin = (int64_t)split * P.points_per_split;
    const int64_t j_end = lmin(j_begin + P.points_per_split, P.npad);
    for (int64_t j0 = j_begin; j0 < j_end; j0 += LOC_SCAN_TILE) {
        __syncthreads();
        const float4* rs = reinterpret_cast<const float4*>(P.rec + j0 * PR);
        for (int i = tid; i < LOC_SCAN_TILE * PR / 4; i += LOC_THREADS) rec4[i] = rs[i];
        const float4* ms = reinterpret_cast<const float4*>(P.mt + j0 * LOC_KNOTS);
        for (int i = tid; i < LOC_SCAN_TILE * LOC_KNOTS / 4; i += LOC_THREADS) mt4[i] = ms[i];
        __syncthreads();
        for (int j = 0; j < LOC_SCAN_TILE; ++j) {
            float vu, vl;
            mono_values<NORM, DP>(q, rec + j * PR, mt + j * LOC_KNOTS, P.cmask, bucket, bk, Tn, scale, vu, vl);
            const int idx = (int)(j0 + j);
            if (vu < bu[K - 1]) {
                int kk = idx;
#pragma unroll
                for (int p = 0; p < K; ++p)
                    if (vu < bu[p]) {
                        const float tv = bu[p]; bu[p] = vu; vu = tv;
                        const int tk = ku[p]; ku[p] = kk; kk = tk;
                    }
            }
            if (vl > bl[K - 1]) {
                int kk = idx;
#pragma unroll
                for (int p = 0; p < K; ++p)
                    if (vl > bl[p]) {
                        const float tv = bl[p]; bl[p] = vl; vl = tv;
                        const int tk = kl[p]; kl[p] = kk; kk = tk;
                    }
            }
        }
    }
    if (qi >= P.nq) return;
    float* pv = static_cast<float*>(P.partial);
    int* pk = reinterpret_cast<int*>(pv + (int64_t)gridDim.y * P.nq * 2 * K);
    const int64_t base = ((int64_t)split * P.nq + qi) * 2 * K;
#pragma unroll
    for (int e = 0; e < K; ++e) {
        pv[base + e] = bu[e];
        pk[base + e] = ku[e];
        pv[base + K + e] = bl[e];
        pk[base + K + e] = kl[e];
    }
}

__device__ __forceinline__ double local_M64(const LocalMergeParams& P, int64_t k, double t);

// The k best over the splits by (value, index), their exact FP64 values with the exact
// table, sorted again by (exact value, index), and the weighted sums.
__global__ void loc_topk_merge_kernel(const LocalMergeParams P, int k, int K, LocalTopkWeights W) {
    const int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= P.nq) return;
    const float* pv = static_cast<const float*>(P.partial);
    const int* pk = reinterpret_cast<const int*>(pv + (int64_t)P.nsplit * P.nq * 2 * K);
    const int64_t q0 = qi * P.d;
    bool finite = true;
    for (int i = 0; i < P.d; ++i) finite = finite && isfinite(ldv(P.Q, P.es, q0 + i));
    double res[2];
    for (int side = 0; side < 2; ++side) {
        float sv[8];
        int sk[8];
        for (int e = 0; e < k; ++e) { sv[e] = side == 0 ? INFINITY : -INFINITY; sk[e] = -1; }
        for (int s = 0; s < P.nsplit; ++s) {
            const int64_t base = ((int64_t)s * P.nq + qi) * 2 * K + side * K;
            for (int e = 0; e < K; ++e) {
                float v = pv[base + e];
                int kk = pk[base + e];
                if (kk < 0) break;
                for (int p = 0; p < k; ++p) {
                    const bool better = sk[p] < 0 || (side == 0 ? v < sv[p] : v > sv[p]) || (v == sv[p] && kk < sk[p]);
                    if (better) {
                        const float tv = sv[p]; sv[p] = v; v = tv;
                        const int tk = sk[p]; sk[p] = kk; kk = tk;
                        if (kk < 0) break;
                    }
                }
            }
        }
        double ev[8];
        int ek[8];
        bool all = finite;
        for (int e = 0; e < k; ++e) {
            ek[e] = sk[e];
            if (sk[e] < 0) { all = false; ev[e] = 0.0; continue; }
            const double t = P.mono ? loc_mdist64(P.Q, q0, P.X0, (int64_t)sk[e] * P.d, P.es, P.d, P.norm, P.w, P.mon,
                                                  side == 0 ? +1 : -1)
                                    : loc_dist64(P.Q, q0, P.X0, (int64_t)sk[e] * P.d, P.es, P.d, P.norm, P.w);
            const double yy = ldv(P.y0, P.es, sk[e]), Mt = __dmul_rn(local_M64(P, sk[e], t), t);
            ev[e] = side == 0 ? __dadd_rn(yy, Mt) : __dsub_rn(yy, Mt);
        }
        for (int a = 1; a < k; ++a)
            for (int b = a; b > 0; --b) {
                const bool sw = side == 0 ? (ev[b] < ev[b - 1] || (ev[b] == ev[b - 1] && ek[b] < ek[b - 1]))
                                          : (ev[b] > ev[b - 1] || (ev[b] == ev[b - 1] && ek[b] < ek[b - 1]));
                if (!sw) break;
                const double tv = ev[b]; ev[b] = ev[b - 1]; ev[b - 1] = tv;
                const int tk = ek[b]; ek[b] = ek[b - 1]; ek[b - 1] = tk;
            }
        double sum = 0.0;
        for (int e = 0; e < k; ++e) sum += W.wk[e] * ev[e];
        res[side] = all ? sum : __longlong_as_double(0x7ff8000000000000ll);
        int32_t* out = side == 0 ? P.idx_up : P.idx_lo;
        if (out)
            for (int e = 0; e < k; ++e) out[qi * k + e] = all ? ek[e] : -1;
    }
    if (P.g) stv(P.g, P.es, qi, 0.5 * (res[0] + res[1]));
    if (P.hi) stv(P.hi, P.es, qi, res[0]);
    if (P.lo) stv(P.lo, P.es, qi, res[1]);
}

__device__ __forceinline__ double local_M64(const LocalMergeParams& P, int64_t k, double t) {
    if (t <= P.d1[k]) return P.F[k];
    int s = 0;
    while (s < P.m && P.T64[s] < t) ++s;
    return P.mt64[k * LOC_KNOTS + s];
}

__global__ void loc_merge_kernel(const LocalMergeParams P) {
    const int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= P.nq) return;
    float bu = 0.f, bl = 0.f;
    int iu = -1, il = -1;
    const PartialRec<float>* part = static_cast<const PartialRec<float>*>(P.partial);
    for (int s = 0; s < P.nsplit; ++s) {
        const PartialRec<float> r = part[(int64_t)s * P.nq + qi];
        if (r.iu >= 0 && (iu < 0 || r.vu < bu)) { bu = r.vu; iu = r.iu; }
        if (r.il >= 0 && (il < 0 || r.vl > bl)) { bl = r.vl; il = r.il; }
    }
    const int64_t q0 = qi * P.d;
    bool finite = true;
    for (int i = 0; i < P.d; ++i) finite = finite && isfinite(ldv(P.Q, P.es, q0 + i));
    double hi, lo;
    if (!finite || iu < 0 || il < 0) {
        hi = lo = __longlong_as_double(0x7ff8000000000000ll);
        iu = il = -1;
    } else {
        // with monotone coordinates the upper bound's datum at dist_up, the lower's at dist_lo
        const double tu = P.mono ? loc_mdist64(P.Q, q0, P.X0, (int64_t)iu * P.d, P.es, P.d, P.norm, P.w, P.mon, +1)
                                 : loc_dist64(P.Q, q0, P.X0, (int64_t)iu * P.d, P.es, P.d, P.norm, P.w);
        const double tl = P.mono ? loc_mdist64(P.Q, q0, P.X0, (int64_t)il * P.d, P.es, P.d, P.norm, P.w, P.mon, -1)
                                 : loc_dist64(P.Q, q0, P.X0, (int64_t)il * P.d, P.es, P.d, P.norm, P.w);
        hi = __dadd_rn(ldv(P.y0, P.es, iu), __dmul_rn(local_M64(P, iu, tu), tu));
        lo = __dsub_rn(ldv(P.y0, P.es, il), __dmul_rn(local_M64(P, il, tl), tl));
    }
    if (P.g) stv(P.g, P.es, qi, 0.5 * (hi + lo));
    if (P.lo) stv(P.lo, P.es, qi, lo);
    if (P.hi) stv(P.hi, P.es, qi, hi);
    if (P.idx_up) P.idx_up[qi] = iu;
    if (P.idx_lo) P.idx_lo[qi] = il;
}

}  // namespace

// Coordinates per record: d rounded up to 4, and 32 for every d above 16 (one wide shape).
int local_dim_pad(int d) { return d <= 16 ? (d + 3) / 4 * 4 : 32; }
int local_record_floats(int d) { return local_dim_pad(d) + 4; }
int64_t local_pad(int64_t N) { return (N + LOC_TILE - 1) / LOC_TILE * LOC_TILE; }
int local_scan_tile() { return LOC_SCAN_TILE; }
int local_queries_per_block(int d) { return LOC_THREADS * 2 * local_scan_groups(local_dim_pad(d)); }
int local_queries_per_block_mono() { return LOC_THREADS; }

cudaError_t launch_local_layout(const LocalParams& P, cudaStream_t st) {
    const unsigned blocks = (unsigned)((P.npad + 255) / 256);
    loc_layout_kernel<<<blocks, 256, 0, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_local_knots(const LocalParams& P, bool sampled, cudaStream_t st) {
    if (sampled && P.S > 0) {
        const unsigned blocks = (unsigned)((P.S + LOC_THREADS - 1) / LOC_THREADS);
        loc_sample_kernel<<<blocks, LOC_THREADS, 0, st>>>(P);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = cudaMemsetAsync(P.counts, 0, (size_t)P.S * 2 * sizeof(int), st);
        if (e != cudaSuccess) return e;
        loc_rank_kernel<<<dim3(blocks, LOC_RANK_SLICES), LOC_THREADS, 0, st>>>(P);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        loc_pick_kernel<<<blocks, LOC_THREADS, 0, st>>>(P);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    loc_knots_kernel<<<1, 256, 0, st>>>(P, sampled ? 1 : 0);
    return cudaGetLastError();
}

template <int NORM, int DP, bool Y64, bool BK>
static cudaError_t table_run_mono(const LocalParams& P, int m, cudaStream_t st) {
    const unsigned blocks = (unsigned)((P.N + LOC_THREADS - 1) / LOC_THREADS);
    loc_screen_mono_kernel<NORM, DP, Y64, BK><<<blocks, LOC_THREADS, table_smem(DP + 4, m + 1, BK), st>>>(P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    loc_exact_mono_kernel<NORM, DP, Y64, BK><<<blocks, LOC_THREADS, 0, st>>>(P);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    loc_pass2_mono_kernel<NORM, DP, Y64, BK><<<blocks, LOC_THREADS, table_smem(DP + 4, LOC_KNOTS, BK), st>>>(P);
    return cudaGetLastError();
}

template <int NORM, int DP, bool Y64, bool BK>
static cudaError_t table_run(const LocalParams& P, int m, cudaStream_t st) {
    if (P.mono) return table_run_mono<NORM, DP, Y64, BK>(P, m, st);
    const unsigned blocks = (unsigned)((P.N + LOC_THREADS - 1) / LOC_THREADS);
    loc_screen_kernel<NORM, DP, Y64, BK><<<blocks, LOC_THREADS, table_smem(DP + 4, m + 1, BK), st>>>(P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    loc_exact_kernel<NORM, DP, Y64, BK><<<blocks, LOC_THREADS, 0, st>>>(P);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    loc_pass2_kernel<NORM, DP, Y64, BK><<<blocks, LOC_THREADS, table_smem(DP + 4, LOC_KNOTS, BK), st>>>(P);
    return cudaGetLastError();
}

template <int NORM, int DP>
static cudaError_t table_shape(const LocalParams& P, bool bk, int m, cudaStream_t st) {
    if (P.es == 8) return bk ? table_run<NORM, DP, true, true>(P, m, st) : table_run<NORM, DP, true, false>(P, m, st);
    return bk ? table_run<NORM, DP, false, true>(P, m, st) : table_run<NORM, DP, false, false>(P, m, st);
}

template <int NORM>
static cudaError_t table_norm(const LocalParams& P, bool bk, int m, cudaStream_t st) {
    switch (P.dp) {
        case 4: return table_shape<NORM, 4>(P, bk, m, st);
        case 8: return table_shape<NORM, 8>(P, bk, m, st);
        case 12: return table_shape<NORM, 12>(P, bk, m, st);
        case 16: return table_shape<NORM, 16>(P, bk, m, st);
        default: return table_shape<NORM, 32>(P, bk, m, st);
    }
}

int local_candidates() { return LOC_CAND; }

cudaError_t launch_local_table(const LocalParams& P, bool bucket_ok, int m, cudaStream_t st) {
    if (P.norm == LIP_L1) return table_norm<LIP_L1>(P, bucket_ok, m, st);
    if (P.norm == LIP_L2) return table_norm<LIP_L2>(P, bucket_ok, m, st);
    return table_norm<LIP_LINF>(P, bucket_ok, m, st);
}

template <int NORM, int DP>
static void scan_shape(const LocalScanParams& S, dim3 grid, bool bucket, cudaStream_t st) {
    if (S.mono) {
        loc_scan_mono_kernel<NORM, DP><<<grid, LOC_THREADS, 0, st>>>(S);
        return;
    }
    constexpr int G = local_scan_groups(DP);
    if (bucket) loc_scan_kernel<NORM, DP, true, G><<<grid, LOC_THREADS, 0, st>>>(S);
    else loc_scan_kernel<NORM, DP, false, G><<<grid, LOC_THREADS, 0, st>>>(S);
}

template <int NORM>
static void scan_norm(const LocalScanParams& S, dim3 grid, bool bucket, cudaStream_t st) {
    switch (S.dp) {
        case 4: scan_shape<NORM, 4>(S, grid, bucket, st); break;
        case 8: scan_shape<NORM, 8>(S, grid, bucket, st); break;
        case 12: scan_shape<NORM, 12>(S, grid, bucket, st); break;
        case 16: scan_shape<NORM, 16>(S, grid, bucket, st); break;
        default: scan_shape<NORM, 32>(S, grid, bucket, st); break;
    }
}

template <int NORM, int DP>
static void topk_shape(int K, const LocalScanParams& S, dim3 grid, cudaStream_t st) {
    if (S.mono) {
        if (K == 2) loc_topk_scan_mono_kernel<NORM, DP, 2><<<grid, LOC_THREADS, 0, st>>>(S);
        else if (K == 4) loc_topk_scan_mono_kernel<NORM, DP, 4><<<grid, LOC_THREADS, 0, st>>>(S);
        else loc_topk_scan_mono_kernel<NORM, DP, 8><<<grid, LOC_THREADS, 0, st>>>(S);
        return;
    }
    if (K == 2) loc_topk_scan_kernel<NORM, DP, 2><<<grid, LOC_THREADS, 0, st>>>(S, K);
    else if (K == 4) loc_topk_scan_kernel<NORM, DP, 4><<<grid, LOC_THREADS, 0, st>>>(S, K);
    else loc_topk_scan_kernel<NORM, DP, 8><<<grid, LOC_THREADS, 0, st>>>(S, K);
}

template <int NORM>
static void topk_norm(int K, const LocalScanParams& S, dim3 grid, cudaStream_t st) {
    switch (S.dp) {
        case 4: topk_shape<NORM, 4>(K, S, grid, st); break;
        case 8: topk_shape<NORM, 8>(K, S, grid, st); break;
        case 12: topk_shape<NORM, 12>(K, S, grid, st); break;
        case 16: topk_shape<NORM, 16>(K, S, grid, st); break;
        default: topk_shape<NORM, 32>(K, S, grid, st); break;
    }
}

int local_topk_threads() { return LOC_THREADS; }

cudaError_t launch_local_eval_k(int norm, int k, int K, const LocalScanParams& S, int gx, int nsplit,
                                const LocalMergeParams& M, const LocalTopkWeights& W, cudaStream_t st) {
    if (nsplit > 0) {
        const dim3 grid((unsigned)gx, (unsigned)nsplit);
        if (norm == LIP_L1) topk_norm<LIP_L1>(K, S, grid, st);
        else if (norm == LIP_L2) topk_norm<LIP_L2>(K, S, grid, st);
        else topk_norm<LIP_LINF>(K, S, grid, st);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    loc_topk_merge_kernel<<<(unsigned)((M.nq + 127) / 128), 128, 0, st>>>(M, k, K, W);
    return cudaGetLastError();
}

cudaError_t launch_local_eval(int norm, const LocalScanParams& S, int gx, int nsplit, bool bucket,
                              const LocalMergeParams& M, cudaStream_t st) {
    if (nsplit > 0) {
        const dim3 grid((unsigned)gx, (unsigned)nsplit);
        if (norm == LIP_L1) scan_norm<LIP_L1>(S, grid, bucket, st);
        else if (norm == LIP_L2) scan_norm<LIP_L2>(S, grid, bucket, st);
        else scan_norm<LIP_LINF>(S, grid, bucket, st);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const unsigned gm = (unsigned)((M.nq + 255) / 256);
    loc_merge_kernel<<<gm, 256, 0, st>>>(M);
    return cudaGetLastError();
}

}  // namespace lip
