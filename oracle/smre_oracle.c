/*
 * FP64 CPU oracle for statistical multi-resolution projection (arXiv 1503.03492).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, obviously-correct
 * restatement of what the paper computes.  It exists so that tests, the smoke
 * check and the timed CPU baseline of the benchmark have something independent
 * to compare the CUDA path with.  The product library never links, loads or
 * calls it, and it shares no code, header or table with the CUDA path.
 *
 * Contents (every function cites the passage it follows):
 *   - weights c_s(alpha)               Sec. 2.1 (fourth-root transform of t_s)
 *   - single-set projection p_s        Sec. 2.3 (projection p_s)
 *   - Dykstra's cyclic projection      Sec. 2.3, Algorithm 2 (with the q-update
 *                                      of the incomplete listing in Sec. 3.2)
 *   - incomplete Dykstra (ICD)         Sec. 3.2 (sets Omega^i, P_incomplete)
 *   - checker: largest window violation of the constraint of Eq. (geq)
 *
 * Notation follows the paper: e is the residual being projected, q_s the
 * increment of set s, w_s = c_s(alpha) the weight of Eq. (tau_s), so the
 * feasible set of window s is { e : w_s * sum_{i in s} e_i^2 <= 1 }.  Callers
 * pass the bound cS = 1 / w_s (the radius squared); the code converts once.
 *
 * Sign convention of q (paper's incomplete listing, Sec. 3.2): before a set is
 * projected, s1 = e - q_s; then q_s = p_s(s1) - s1 and e = p_s(s1).  This is
 * standard Dykstra with the increment stored with the opposite sign.
 *
 * Readings of passages that are garbled or silent (each is listed in the
 * design notes of the repository):
 *   R1  Algorithm 2 prints no loop over s; the update used is the one of the
 *       incomplete listing, applied to every set in turn.
 *   R4  Set order of one cycle: sides in descending order; for each side L the
 *       L*L tilings (L, a, b), a and b in 0..L-1, a outer, b inner; windows of
 *       one tiling are disjoint, so their order is immaterial.  Callers may pass
 *       any other order of tilings explicitly.
 *   R5  Windows lie fully inside the image; no wrap-around, no partial windows.
 *   R6  Standard stopping test: unsquared L2 change of e over one cycle, either
 *       absolute or relative to |e| before the cycle; tol < 0 runs exactly
 *       max_cycles cycles.  ICD: per-tile L1 change of one sweep <= tol * B^2,
 *       at least one sweep, at most max_sweeps.
 *   R7  ICD: Omega^i is the union over levels k = i..K; passes i = 0..K;
 *       offset of pass i is (1 << i) mod B with B = 2^K; tiles lie fully
 *       inside the image.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Sec. 2.1: weights                                                          */
/* ------------------------------------------------------------------------ */

/* Standard normal CDF written with the C library's erfc (a library primitive). */
static double normal_cdf(double z) { return 0.5 * erfc(-z / sqrt(2.0)); }

/* alpha-quantile of N(0,1): plain bisection on the CDF. */
double oracle_normal_quantile(double alpha)
{
    double lo = -40.0, hi = 40.0;
    for (int it = 0; it < 300; ++it) {
        double mid = 0.5 * (lo + hi);
        if (normal_cdf(mid) < alpha) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* Upper tail Q(x; k) = P(chi2_k > x) for an integer number k of degrees of
 * freedom, written out as the textbook finite sums (Abramowitz & Stegun
 * 26.4.4 for odd k, 26.4.5 for even k). */
static double chi2_upper_tail(double x, int k)
{
    if (x <= 0.0) return 1.0;
    if (k % 2 == 0) {
        /* Q = exp(-x/2) * sum_{j=0}^{k/2-1} (x/2)^j / j! */
        double term = 1.0, sum = 1.0;
        for (int j = 1; j < k / 2; ++j) { term *= (x / 2.0) / j; sum += term; }
        return exp(-x / 2.0) * sum;
    } else {
        /* Q = 2 Q_N(sqrt x) + sqrt(2x/pi) exp(-x/2) * sum_{j=1}^{(k-1)/2} x^{j-1}/(1*3*...*(2j-1)) */
        double r = sqrt(x);
        double q = erfc(r / sqrt(2.0));
        double term = 1.0, sum = 0.0;
        for (int j = 1; j <= (k - 1) / 2; ++j) {
            if (j > 1) term *= x / (2.0 * j - 1.0);
            sum += term;
        }
        return q + sqrt(2.0 * x / M_PI) * exp(-x / 2.0) * sum;
    }
}

/* alpha-quantile of chi2_k: bisection on the CDF 1 - Q. */
double oracle_chi2_quantile(double alpha, int k)
{
    double lo = 0.0, hi = 10.0 * k + 100.0;
    for (int it = 0; it < 300; ++it) {
        double mid = 0.5 * (lo + hi);
        if (1.0 - chi2_upper_tail(mid, k) < alpha) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* Fourth-root transform of Sec. 2.1 for a set of |s| = n pixels:
 * t_s^{1/4} ~ N(mu_s, sigma_s^2), mu_s = (|s| - 0.5)^{1/4}, sigma_s^2 = 1/(8 sqrt|s|). */
static double mu_s(int n) { return pow(n - 0.5, 0.25); }
static double sigma_s(int n) { return sqrt(1.0 / (8.0 * sqrt((double)n))); }

/* Bound cS = 1/c_s(alpha) = (q sigma_s + mu_s)^4 of Sec. 2.1 for a square
 * window of side L, given the quantile q. */
double oracle_bound_from_quantile(double q, int L)
{
    int n = L * L;
    double r = q * sigma_s(n) + mu_s(n);
    return r * r * r * r;
}

/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) used as a counter-based
 * generator: value(i) = mix(seed + (i + 1) * golden_gamma). */
static uint64_t splitmix64_at(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1u) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Uniform in (0, 1]: the top 53 bits, shifted by one ulp away from zero. */
static double uniform_open0(uint64_t seed, uint64_t i)
{
    return ((double)(splitmix64_at(seed, i) >> 11) + 1.0) * (1.0 / 9007199254740992.0);
}

/* Standard normal number n(seed, j) by Box-Muller (Box & Muller 1958) from the
 * two uniforms with counters 2j and 2j+1 (cosine branch). */
double oracle_normal_sample(uint64_t seed, uint64_t j)
{
    double u1 = uniform_open0(seed, 2u * j);
    double u2 = uniform_open0(seed, 2u * j + 1u);
    return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Monte Carlo estimate of q_alpha, the alpha-quantile of the extreme value
 * statistic Q_Omega = max_s (t_s^{1/4} - mu_s) / sigma_s of Sec. 2.1, over all
 * square windows of the given sides at all positions of an H x W image of iid
 * N(0,1) noise.  Draw d uses pixels j = d*H*W + p of oracle_normal_sample.
 * The empirical quantile is the ceil(alpha*D)-th smallest of the D maxima. */
double oracle_maxstat_quantile(int H, int W, int n_sides, const int *sides,
                               double alpha, int draws, uint64_t seed)
{
    double *img = (double *)malloc(sizeof(double) * (size_t)H * W);
    double *qmax = (double *)malloc(sizeof(double) * (size_t)draws);
    for (int d = 0; d < draws; ++d) {
        for (int p = 0; p < H * W; ++p)
            img[p] = oracle_normal_sample(seed, (uint64_t)d * H * W + p);
        double best = -INFINITY;
        for (int si = 0; si < n_sides; ++si) {
            int L = sides[si], n = L * L;
            double mu = mu_s(n), sg = sigma_s(n);
            for (int r = 0; r + L <= H; ++r)
                for (int c = 0; c + L <= W; ++c) {
                    double t = 0.0;
                    for (int i = 0; i < L; ++i)
                        for (int j = 0; j < L; ++j) {
                            double e = img[(r + i) * W + (c + j)];
                            t += e * e;
                        }
                    double z = (pow(t, 0.25) - mu) / sg;
                    if (z > best) best = z;
                }
        }
        qmax[d] = best;
    }
    qsort(qmax, (size_t)draws, sizeof(double), cmp_double);
    int idx = (int)ceil(alpha * draws) - 1;
    if (idx < 0) idx = 0;
    if (idx >= draws) idx = draws - 1;
    double q = qmax[idx];
    free(img);
    free(qmax);
    return q;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.3, projection p_s: projection of one set, in place on s1            */
/* ------------------------------------------------------------------------ */

/* Project the L x L window at (r, c) of the pitch-W array s1 onto
 * { w * sum s1_i^2 <= 1 }:  s1_i <- s1_i / (sqrt(w) |s1|_{2,s}) if w |s1|^2 > 1. */
static void project_window(double *s1, int W, int r, int c, int L, double w)
{
    double t = 0.0;
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < L; ++j) {
            double v = s1[(r + i) * W + (c + j)];
            t += v * v;
        }
    if (w * t > 1.0) {
        double den = sqrt(w) * sqrt(t);
        for (int i = 0; i < L; ++i)
            for (int j = 0; j < L; ++j) s1[(r + i) * W + (c + j)] /= den;
    }
}

/* One Dykstra step on window s (Sec. 3.2 listing semantics, reading R1):
 * s1 = e - q_s; q_s = -s1; s1 = p_s(s1); q_s += s1; e = s1.
 * q is the pitch-W plane that holds q_s at the pixels of s.  Returns the L1
 * change of e over the window (the listing's increment). */
static double dykstra_step(double *e, double *q, double *s1, int W, int r, int c, int L, double w)
{
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < L; ++j) {
            size_t p = (size_t)(r + i) * W + (c + j);
            s1[p] = e[p] - q[p];
            q[p] = -s1[p];
        }
    project_window(s1, W, r, c, L, w);
    double delta = 0.0;
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < L; ++j) {
            size_t p = (size_t)(r + i) * W + (c + j);
            q[p] += s1[p];
            delta += fabs(e[p] - s1[p]);
            e[p] = s1[p];
        }
    return delta;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.3, Algorithm 2: Dykstra's cyclic projection onto tau_G               */
/* ------------------------------------------------------------------------ */

/*
 * Project x0 (H x W, row-major) onto the intersection of the balls of all
 * L x L windows of the listed tilings.  Tiling k is (Ls[k], as[k], bs[k]): the
 * windows with top-left corner (a + L u, b + L v) fully inside the image.  One
 * cycle visits the tilings in the given order (reading R4 gives the default),
 * each set once.  cS_of_tiling[k] is the bound of tiling k's windows.
 *
 * Stops after the first cycle whose L2 change d satisfies d <= tol (abs) or
 * d <= tol * |x_prev| (rel), or after max_cycles cycles (reading R6).
 *
 * Outputs: x_out (H x W); returns the number of cycles run.  If hist is not
 * NULL it receives (d, |x_prev|) per cycle.  If q_out is not NULL it receives
 * the n_tilings planes (H x W each) of increments in the paper's sign
 * convention.  n_threads > 1 splits the windows of one tiling over OpenMP
 * threads; since the windows are disjoint this is bitwise identical to serial.
 * Returns -1 if memory runs out.
 */
int oracle_dykstra(int H, int W, const double *x0,
                   int n_tilings, const int *Ls, const int *as, const int *bs,
                   const double *cS_of_tiling,
                   int max_cycles, double tol, int tol_relative, int n_threads,
                   double *x_out, double *hist, double *q_out)
{
    size_t npx = (size_t)H * W;
    double *q = q_out ? q_out : (double *)malloc(sizeof(double) * npx * (size_t)n_tilings);
    double *s1 = (double *)malloc(sizeof(double) * npx);
    double *prev = (double *)malloc(sizeof(double) * npx);
    if (!q || !s1 || !prev) { if (!q_out) free(q); free(s1); free(prev); return -1; }
    memset(q, 0, sizeof(double) * npx * (size_t)n_tilings);  /* q_{0,s} = 0 */
    memcpy(x_out, x0, sizeof(double) * npx);
    (void)n_threads;

    int cycles = 0;
    while (cycles < max_cycles) {
        memcpy(prev, x_out, sizeof(double) * npx);
        for (int k = 0; k < n_tilings; ++k) {
            int L = Ls[k], a = as[k], b = bs[k];
            double w = 1.0 / cS_of_tiling[k];
            double *qk = q + npx * (size_t)k;
            int nu = (H - a) / L, nv = (W - b) / L;
#ifdef _OPENMP
#pragma omp parallel for num_threads(n_threads > 0 ? n_threads : 1) schedule(static)
#endif
            for (int u = 0; u < nu; ++u)
                for (int v = 0; v < nv; ++v)
                    dykstra_step(x_out, qk, s1, W, a + L * u, b + L * v, L, w);
        }
        ++cycles;
        double d2 = 0.0, n2 = 0.0;
        for (size_t p = 0; p < npx; ++p) {
            double dd = x_out[p] - prev[p];
            d2 += dd * dd;
            n2 += prev[p] * prev[p];
        }
        double d = sqrt(d2), n = sqrt(n2);
        if (hist) { hist[2 * (cycles - 1)] = d; hist[2 * (cycles - 1) + 1] = n; }
        if (tol >= 0.0 && (tol_relative ? d <= tol * n : d <= tol)) break;
    }
    if (!q_out) free(q);
    free(s1);
    free(prev);
    return cycles;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.2: incomplete Dykstra                                                */
/* ------------------------------------------------------------------------ */

/* Number of tiles of pass i along an extent n (reading R7: tiles of side B
 * start at off + B t and lie fully inside). */
static int icd_tiles(int n, int off, int B) { return n - off >= B ? (n - off) / B : 0; }

/*
 * P_incomplete = prod_{i=0}^{K} P_{Omega^i} (Sec. 3.2, readings R6, R7).
 * Pass i covers the image with B x B tiles (B = 2^K) whose origins are
 * (off + B ti, off + B tj), off = (1 << i) mod B.  Inside one tile it runs
 * Dykstra's algorithm over the sets of Omega^i: for k = K down to i, the
 * non-overlapping 2^k x 2^k squares that tile the tile.  The increments of all
 * levels start at zero for every tile of every pass.  A tile repeats sweeps
 * (one sweep = all levels once) until the sweep's L1 change of e is
 * <= tol * B^2 (at least one sweep, at most max_sweeps).
 *
 * cS_level[k] is the bound of side 2^k.  sweeps_out (optional) receives the
 * sweep count of every tile, pass by pass, tiles row-major.  Returns the
 * total number of tiles over all passes, or -1 on bad arguments.
 */
int oracle_icd(int H, int W, const double *x0, int K, const double *cS_level,
               double tol, int max_sweeps, double *x_out, int *sweeps_out)
{
    if (K < 0 || K > 12 || max_sweeps < 1) return -1;
    int B = 1 << K;
    size_t npx = (size_t)H * W;
    double *q = (double *)malloc(sizeof(double) * npx * (size_t)(K + 1));
    double *s1 = (double *)malloc(sizeof(double) * npx);
    if (!q || !s1) { free(q); free(s1); return -1; }
    memcpy(x_out, x0, sizeof(double) * npx);
    int tile_count = 0;
    for (int i = 0; i <= K; ++i) {
        int off = (1 << i) % B;
        int nti = icd_tiles(H, off, B), ntj = icd_tiles(W, off, B);
        for (int ti = 0; ti < nti; ++ti)
            for (int tj = 0; tj < ntj; ++tj) {
                int r0 = off + B * ti, c0 = off + B * tj;
                /* q_k := 0 on this tile for every level of the pass */
                for (int k = i; k <= K; ++k)
                    for (int r = 0; r < B; ++r)
                        for (int c = 0; c < B; ++c)
                            q[npx * (size_t)k + (size_t)(r0 + r) * W + (c0 + c)] = 0.0;
                int sweeps = 0;
                double delta;
                do {
                    delta = 0.0;
                    for (int k = K; k >= i; --k) {
                        int side = 1 << k;
                        double w = 1.0 / cS_level[k];
                        for (int m = 0; m < B / side; ++m)
                            for (int n = 0; n < B / side; ++n)
                                delta += dykstra_step(x_out, q + npx * (size_t)k, s1, W,
                                                      r0 + side * m, c0 + side * n, side, w);
                    }
                    ++sweeps;
                } while (delta > tol * (double)B * (double)B && sweeps < max_sweeps);
                if (sweeps_out) sweeps_out[tile_count] = sweeps;
                ++tile_count;
            }
    }
    free(q);
    free(s1);
    return tile_count;
}

/* ------------------------------------------------------------------------ */
/* Checker: constraint of Eq. (geq)                                            */
/* ------------------------------------------------------------------------ */

/* Largest relative violation max_s (sum_{i in s} e_i^2 - cS) / cS over all
 * L x L windows at all positions, for each listed side. */
double oracle_max_violation(int H, int W, const double *e, int n_sides, const int *sides,
                            const double *cS_of_side)
{
    double worst = -INFINITY;
    for (int si = 0; si < n_sides; ++si) {
        int L = sides[si];
        for (int r = 0; r + L <= H; ++r)
            for (int c = 0; c + L <= W; ++c) {
                double t = 0.0;
                for (int i = 0; i < L; ++i)
                    for (int j = 0; j < L; ++j) {
                        double v = e[(size_t)(r + i) * W + (c + j)];
                        t += v * v;
                    }
                double viol = (t - cS_of_side[si]) / cS_of_side[si];
                if (viol > worst) worst = viol;
            }
    }
    return worst;
}

/* Number of threads OpenMP would use (1 if built without it). */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
