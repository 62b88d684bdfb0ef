/*
 * synth.c -- seeded synthetic irregularly sampled light curves.
 *
 * Input generators only: nothing here computes any part of the correlation
 * estimator.  Every random draw comes from a counter-style generator
 * (SplitMix64, Steele, Lea & Flood 2014) keyed by (seed, stream), turned into
 * uniforms on (0, 1) and into normals by the Box-Muller transform, so a given
 * (seed, stream) always yields the same numbers on any host.
 *
 * Processes:
 *  - exact Ornstein-Uhlenbeck transitions at arbitrary sorted times:
 *    X_k = phi_k X_{k-1} + sigma sqrt(1 - phi_k^2) eta_k, phi_k = exp(-dt_k/tau),
 *    started from the stationary law N(0, sigma^2) (the exact discretisation
 *    used for the paper's OU test series, Sec. 3.1 footnote);
 *  - nightly ground-based cadence with an observing season and weather
 *    losses (Sec. 4.1), several epochs per night for long series.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

typedef struct { uint64_t s; } rng_t;

static inline uint64_t splitmix64(rng_t *r) {
    uint64_t z = (r->s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static inline rng_t rng_make(uint64_t seed, uint64_t stream) {
    rng_t r = {seed * 0xD1342543DE82EF95ULL + stream};
    (void)splitmix64(&r);
    r.s ^= stream * 0x9E3779B97F4A7C15ULL;
    (void)splitmix64(&r);
    return r;
}
/* uniform on the open interval (0, 1) from the top 53 bits */
static inline double unif(rng_t *r) {
    return ((double)(splitmix64(r) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}
static inline double normal(rng_t *r) {
    double u1 = unif(r), u2 = unif(r);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925286766559 * u2);
}

/* Exact OU at sorted times t[0..n), mean 0, stationary std sigma, added into
 * out (accumulate = 1) or written (accumulate = 0). */
void synth_ou(const double *t, int64_t n, double tau, double sigma,
              uint64_t seed, uint64_t stream, double *out, int accumulate) {
    rng_t r = rng_make(seed, stream);
    double v = sigma * normal(&r);
    for (int64_t k = 0; k < n; ++k) {
        if (k > 0) {
            double phi = exp(-(t[k] - t[k - 1]) / tau);
            v = phi * v + sigma * sqrt(fmax(0.0, 1.0 - phi * phi)) * normal(&r);
        }
        out[k] = accumulate ? out[k] + v : v;
    }
}

/* n normals N(0, 1) */
void synth_normals(int64_t n, uint64_t seed, uint64_t stream, double *out) {
    rng_t r = rng_make(seed, stream);
    for (int64_t k = 0; k < n; ++k) out[k] = normal(&r);
}

/* n uniforms on (lo, hi) */
void synth_uniforms(int64_t n, double lo, double hi, uint64_t seed, uint64_t stream,
                    double *out) {
    rng_t r = rng_make(seed, stream);
    for (int64_t k = 0; k < n; ++k) out[k] = lo + (hi - lo) * unif(&r);
}

/*
 * Ground-based nightly cadence over `years` years: nights d = 365*y + i for
 * i < season_days are observable, each lost to weather with probability
 * p_weather.  n epochs are placed in night windows [d, d + night_len):
 * n <= nights -> one epoch on each of n nights chosen without replacement;
 * otherwise every night gets floor(n / nights) or one more epoch, at sorted
 * uniform offsets (exponential spacings, so no sort is needed).
 * Writes n sorted times into t.  Returns the number of observable nights.
 */
int64_t synth_cadence(int64_t n, int years, int season_days, double p_weather,
                      double night_len, uint64_t seed, uint64_t stream, double *t) {
    rng_t r = rng_make(seed, stream);
    int64_t cap = (int64_t)years * season_days;
    int64_t *nights = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
    int64_t nn = 0;
    for (int y = 0; y < years; ++y)
        for (int i = 0; i < season_days; ++i)
            if (unif(&r) >= p_weather) nights[nn++] = 365 * (int64_t)y + i;
    int64_t w = 0;
    if (n <= nn) {
        /* selection sampling (Knuth, TAOCP vol. 2, Algorithm S) keeps order */
        int64_t need = n;
        for (int64_t q = 0; q < nn && need > 0; ++q) {
            if ((double)(nn - q) * unif(&r) < (double)need) {
                t[w++] = (double)nights[q] + night_len * unif(&r);
                --need;
            }
        }
    } else {
        int64_t base = n / nn, extra = n - base * nn;
        int64_t need = extra;
        double *e = (double *)malloc((size_t)(base + 2) * sizeof(double));
        for (int64_t q = 0; q < nn; ++q) {
            int64_t c = base;
            if (need > 0 && (double)(nn - q) * unif(&r) < (double)need) { ++c; --need; }
            double tot = 0.0;
            for (int64_t a = 0; a <= c; ++a) { e[a] = -log(unif(&r)); tot += e[a]; }
            double acc = 0.0;
            for (int64_t a = 0; a < c; ++a) {
                acc += e[a];
                t[w++] = (double)nights[q] + night_len * (acc / tot);
            }
        }
        free(e);
    }
    free(nights);
    return nn;
}
