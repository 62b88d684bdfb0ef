/*
 * ncf_oracle.c -- FP64 CPU oracle for the kernel-weighted ACF/CCF estimator.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA library is checked against.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it; the product path never
 * does.  It shares no code, header or table with the CUDA library.
 *
 * Two evaluators of the same quantity:
 *
 *  O1  oracle_corr_direct   -- the definition written out (Sec. 2.3,
 *      Eq. kernel_estimator): for every requested lag, a double loop over all
 *      pairs (i, j) accumulating x_i*y_j*b(d) and b(d) with Neumaier
 *      compensated sums.  O(n_x * n_y * K).
 *
 *  O2  oracle_corr_windowed -- the paper's real-space algorithms
 *      (Appendix "Real-space ACF/CCF algorithms", Algorithms 5-8): a
 *      two-pointer window scan per lag over sorted times, Gaussian weights
 *      summed inside the half-open window [c - R h, c + R h), rectangle counts
 *      and prefix-sum numerators inside the closed window [c - h, c + h].
 *      O((n_x + n_y) * K).  Used where O1's n^2 K is too slow.
 *
 * Conventions, with the reading taken where the paper leaves a choice open:
 *  - outer index j runs over (s, y), window index i over (t, x); the window
 *    centre is c_j = s_j + eps * tau_k with eps = +1 for the ACF (s = t, y = x)
 *    and eps = -1 for the CCF (Sec. "Effective pair count algorithms"), so a
 *    positive lag pairs s_j with t_i near s_j - tau: y lags x;
 *  - rectangle: h is the half-width, as in Algorithms 6 and 8, whose window is
 *    [c - h, c + h] (Eq. rectangle_kernel writes |d| <= h/2 with h the full
 *    width; the package's parameter is the algorithms' half-width).  A pair
 *    counts iff fl(c_j - h) <= t_i <= fl(c_j + h), closed at both ends as in
 *    Algorithm 6, every operation one FP64 rounding on the caller's own times
 *    (compile with -ffp-contract=off so no FMA changes a rounding), so that the
 *    exact integer counts have one definition;
 *  - Gaussian: b(d) = exp(-d^2 / (2 h^2)) / (sqrt(2 pi) h), Eq. Gaussian_kernel,
 *    with d = t_i - c_j.  trunc_R == 0 means untruncated (all pairs), as the
 *    equation is written; trunc_R > 0 keeps only
 *    fl(c_j - fl(R h)) <= t_i < fl(c_j + fl(R h)), the half-open window of
 *    Algorithm 5 (which takes R = 6).
 *
 * All inputs are standardised values already (the Python wrapper does the
 * standardisation in FP64, Sec. "Prior standardization").
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_SQRT_2PI 2.50662827463100050241576528481104525

/* Neumaier's improved Kahan summation. */
typedef struct { double s, c; } nsum;

static inline void nsum_add(nsum *a, double v) {
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}
static inline double nsum_get(const nsum *a) { return a->s + a->c; }

/* mean and population standard deviation (ddof = 0), both with compensated
 * sums: x_std = (x - mean) / std is step 1 of Algorithms 2, 4, 9 and 10. */
void oracle_stats(const double *x, int64_t n, double *mean, double *std_) {
    nsum a = {0.0, 0.0};
    for (int64_t i = 0; i < n; ++i) nsum_add(&a, x[i]);
    double m = nsum_get(&a) / (double)n;
    nsum v = {0.0, 0.0};
    for (int64_t i = 0; i < n; ++i) { double d = x[i] - m; nsum_add(&v, d * d); }
    *mean = m;
    *std_ = sqrt(nsum_get(&v) / (double)n);
}

#define ORACLE_PI 3.14159265358979323846264338327950288

static inline double gauss_b(double d, double h) {
    return exp(-(d * d) / (2.0 * h * h)) / (ORACLE_SQRT_2PI * h);
}

/* Hann window of half-width h and unit mass, b(d) = cos^2(pi d / (2 h)) / h on
 * |d| <= h (the Hanning kernel named in Sec. 2.3 and left undefined there). */
static inline double hann_b(double d, double h) {
    const double c = cos(ORACLE_PI * d / (2.0 * h));
    return c * c / h;
}

/*
 * O1: direct double sum of Eq. kernel_estimator for each lag.
 *   kernel: 0 = Gaussian, 1 = rectangle, 2 = Hanning (the rectangle's closed
 *   window with Hann weights).  eps: +1 ACF, -1 CCF.
 * Outputs per lag k: num[k] = sum x_i y_j b, den[k] = sum b, cnt[k] = number
 * of pairs with nonzero weight (rectangle: the exact integer pair count).
 */
void oracle_corr_direct(const double *t, const double *x, int64_t nx,
                        const double *s, const double *y, int64_t ny,
                        const double *lags, int64_t K, int kernel, double h,
                        double trunc_R, int eps,
                        double *num, double *den, int64_t *cnt) {
    const double Rh = trunc_R * h;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < K; ++k) {
        nsum N = {0.0, 0.0}, B = {0.0, 0.0};
        int64_t C = 0;
        for (int64_t j = 0; j < ny; ++j) {
            const double c = s[j] + (double)eps * lags[k];
            if (kernel == 1) {
                const double lo = c - h, hi = c + h;
                for (int64_t i = 0; i < nx; ++i) {
                    if (lo <= t[i] && t[i] <= hi) {
                        nsum_add(&N, x[i] * y[j]);
                        C += 1;
                    }
                }
            } else if (kernel == 2) {
                const double lo = c - h, hi = c + h;
                for (int64_t i = 0; i < nx; ++i) {
                    if (lo <= t[i] && t[i] <= hi) {
                        const double w = hann_b(t[i] - c, h);
                        nsum_add(&N, w * x[i] * y[j]);
                        nsum_add(&B, w);
                        C += 1;
                    }
                }
            } else {
                const double lo = c - Rh, hi = c + Rh;
                for (int64_t i = 0; i < nx; ++i) {
                    if (trunc_R > 0.0 && !(lo <= t[i] && t[i] < hi)) continue;
                    const double w = gauss_b(t[i] - c, h);
                    nsum_add(&N, w * x[i] * y[j]);
                    nsum_add(&B, w);
                    C += 1;
                }
            }
        }
        num[k] = nsum_get(&N);
        den[k] = (kernel == 1) ? (double)C : nsum_get(&B);
        cnt[k] = C;
    }
}

/*
 * O2: the paper's two-pointer real-space scan (Algorithms 5-8), one lag per
 * OpenMP task.  Gaussian: PairCount (Alg. 5) and CorrSum (Alg. 7) share the
 * window; rectangle: PairCount (Alg. 6) and the prefix-sum CorrSum (Alg. 8).
 * The prefix sums cum[0..nx] are plain FP64 running sums as in Algorithm 8.
 */
void oracle_corr_windowed(const double *t, const double *x, int64_t nx,
                          const double *s, const double *y, int64_t ny,
                          const double *lags, int64_t K, int kernel, double h,
                          double trunc_R, int eps,
                          double *num, double *den, int64_t *cnt) {
    double *cum = NULL;
    if (kernel == 1) {
        cum = (double *)malloc((size_t)(nx + 1) * sizeof(double));
        cum[0] = 0.0;
        for (int64_t i = 0; i < nx; ++i) cum[i + 1] = cum[i] + x[i];
    }
    const double Rh = trunc_R * h;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < K; ++k) {
        int64_t lo = 0, hi = 0, C = 0;
        double N = 0.0, B = 0.0;
        for (int64_t j = 0; j < ny; ++j) {
            const double c = s[j] + (double)eps * lags[k];
            if (kernel == 1) {
                while (lo < nx && t[lo] < c - h) ++lo;
                if (hi < lo) hi = lo;
                while (hi < nx && t[hi] <= c + h) ++hi;
                C += hi - lo;
                N += y[j] * (cum[hi] - cum[lo]);
            } else if (kernel == 2) {
                while (lo < nx && t[lo] < c - h) ++lo;
                if (hi < lo) hi = lo;
                while (hi < nx && t[hi] <= c + h) ++hi;
                for (int64_t i = lo; i < hi; ++i) {
                    const double w = hann_b(t[i] - c, h);
                    B += w;
                    N += w * x[i] * y[j];
                }
                C += hi - lo;
            } else {
                while (lo < nx && t[lo] < c - Rh) ++lo;
                while (hi < nx && t[hi] < c + Rh) ++hi;
                for (int64_t i = lo; i < hi; ++i) {
                    const double w = gauss_b(t[i] - c, h);
                    B += w;
                    N += w * x[i] * y[j];
                }
                C += (hi > lo) ? hi - lo : 0;
            }
        }
        num[k] = N;
        den[k] = (kernel == 1) ? (double)C : B;
        cnt[k] = C;
    }
    free(cum);
}
