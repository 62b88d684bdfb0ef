/*
 * ncf.h -- C ABI of libncf: kernel-weighted auto/cross-correlation of
 * irregularly sampled time series on one NVIDIA B300 (sm_103a).
 *
 * What is computed (arXiv 2609.03866, Sec. 2.3, Eq. kernel_estimator):
 *
 *     N_k = sum_i sum_j x_std,i * y_std,j * b(s_j - t_i - tau_k)
 *     B_k = sum_i sum_j b(s_j - t_i - tau_k)
 *     c_k = N_k / max(B_k, 1e-16)                       (Algorithms 5-6 clamp)
 *
 * for K requested lags tau_k, where x_std = (x - mean(x)) / std(x) with ddof 0
 * (Appendix, "Prior standardization"), and b is
 *   - the Gaussian kernel exp(-d^2 / 2h^2) / (sqrt(2 pi) h)  (Eq. Gaussian_kernel), or
 *   - the rectangle kernel, 1 for |d| <= h, 0 otherwise, h the HALF-width
 *     (the half-width convention of Algorithms 6 and 8).
 * The ACF is the case s = t, y = x.  Lag tau > 0 pairs points with
 * s_j - t_i ~ tau, i.e. y lagging x (Appendix, sign convention).
 *
 * Rectangle windows use the predicate of Algorithm 6 evaluated in IEEE FP64
 * round-to-nearest on the caller's own values: with c = s_j + e*tau_k
 * (e = +1 for the ACF, -1 for the CCF), a pair counts iff
 * fl(c - h) <= t_i <= fl(c + h).  Pair counts are exact 64-bit integers.
 *
 * Evaluation paths:
 *   NCF_PATH_SPECTRAL  Wiener-Khinchin (Sec. 2.6): type-1 NUFFT of the values
 *                      and of unit weights onto a uniform grid, FFT, cross-
 *                      spectrum times the kernel's Fourier transform, sum of
 *                      the modes at the K lags.  For the rectangle this is the
 *                      spectral-sinc variant, taken only when asked for: its
 *                      transform sin(2 pi f h)/(pi f) decays as 1/f, so the sum
 *                      over |m| <= L/(h tol) modes (tol default 1e-3) carries
 *                      an error of order tol of a pair's weight near the window
 *                      edges (reported by the tests, not gated); count_out is 0.
 *                      It keeps a mode-by-lag table, so it suits single series
 *                      and moderate L/(h tol) (NCF_ENOMEM otherwise).
 *   NCF_PATH_WINDOWED  the two-pointer real-space scan (Algorithms 5-8).
 *   NCF_PATH_AUTO      spectral for the Gaussian, windowed for the rectangle.
 *
 * Precision:
 *   NCF_FP64           FP64 throughout (results within 1e-10 of the FP64
 *                      definition for the documented workloads).
 *   NCF_FP32           batched FP32 form: spreading, FFT and the mode-to-lag
 *                      contraction in FP32 (the contraction on tensor cores
 *                      where available); FP64 for standardisation, time-to-
 *                      phase reduction and normalisation.  Rectangle results
 *                      are identical in both precisions (exact scan).
 *
 * Memory and streams: every array argument of ncf_corr and ncf_corr_batch is
 * a DEVICE pointer owned by the caller, except the CSR offsets of
 * ncf_corr_batch, which are HOST arrays.  `stream` is a cudaStream_t (NULL =
 * legacy default stream).  The library owns a workspace per context, grown on
 * demand with cudaMalloc.  A call validates its inputs, synchronises `stream`
 * once to read back per-series statistics (time span, variance), then
 * enqueues its kernels on `stream` and returns; results are ready when the
 * stream reaches that point.  Validation errors are returned before any
 * output is written.  No exception crosses the ABI.  A context is not
 * thread-safe: use one per host thread.
 */
#ifndef NCF_H
#define NCF_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define NCF_API __attribute__((visibility("default")))
#else
#define NCF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NCF_OK = 0,
    NCF_EINVAL = 1,        /* bad argument: NULL pointer, n < 2, K < 1, h <= 0, bad enum */
    NCF_ENOTSORTED = 2,    /* times decrease somewhere (equal times are allowed) */
    NCF_EDEGENERATE = 3,   /* a series has zero variance: x_std undefined */
    NCF_ENOMEM = 4,        /* workspace allocation failed */
    NCF_ECUDA = 5,         /* a CUDA runtime call failed; see ncf_last_error */
    NCF_ETIMEOUT = 6,      /* a bounded device-side wait gave up */
    NCF_EBUSY = 7,         /* serving: admission budget exhausted */
    NCF_ENONFINITE = 8,    /* a time, value or lag is NaN or infinite */
    NCF_EUNSUPPORTED = 9   /* option combination not provided (see ncf_last_error) */
} ncf_status;

/* NCF_HANNING: the Hann window b(d) = cos^2(pi d / (2 h)) / h for |d| <= h (unit
 * mass), the kernel Sec. 2.3 names without defining; the rectangle's closed
 * window with Hann weights, FP64 windowed path (and the regular-grid path) only. */
typedef enum { NCF_GAUSSIAN = 0, NCF_RECTANGLE = 1, NCF_HANNING = 2 } ncf_kernel;
typedef enum { NCF_PATH_AUTO = 0, NCF_PATH_SPECTRAL = 1, NCF_PATH_WINDOWED = 2 } ncf_path;
typedef enum { NCF_FP64 = 0, NCF_FP32 = 1 } ncf_precision;
typedef enum {
    NCF_NORM_NONE = 0,     /* c = N / max(B, 1e-16), Eq. kernel_estimator as written */
    NCF_NORM_LAG0 = 1      /* Pearson: ACF / ACF(0) (Algorithm 4); CCF / sqrt(ACF_x(0) ACF_y(0)) (Algorithm 10) */
} ncf_norm;

typedef struct {
    int32_t kernel;     /* ncf_kernel */
    int32_t path;       /* ncf_path */
    int32_t precision;  /* ncf_precision */
    int32_t norm;       /* ncf_norm */
    double h;           /* Gaussian sigma, or rectangle half-width; > 0 */
    double trunc_R;     /* Gaussian windowed path: window [c - R h, c + R h) as in
                           Algorithm 5 with 6 replaced by R; 0 selects 8 */
    double tol;         /* spectral path tolerance on the kernel transform and the
                           spreading; 0 selects 1e-14 (FP64) or 1e-7 (FP32), and
                           1e-3 for the spectral-sinc rectangle (its mode count
                           L / (h tol)) */
} ncf_options;

/* Fills *o with: Gaussian, AUTO path, FP64, NORM_NONE, h = 1, trunc_R = 0, tol = 0. */
NCF_API void ncf_options_default(ncf_options *o);

typedef struct ncf_ctx ncf_ctx;

/* Creates a context bound to CUDA device `device`.  *out is NULL on failure. */
NCF_API ncf_status ncf_create(ncf_ctx **out, int device);
/* Frees the context and its workspace (synchronises the device first). */
NCF_API void ncf_destroy(ncf_ctx *ctx);
/* Message of the last failed call on ctx ("" if none).  Owned by ctx. */
NCF_API const char *ncf_last_error(const ncf_ctx *ctx);
/* Static name of a status code. */
NCF_API const char *ncf_status_string(ncf_status s);
/* Number of kernels this context has launched so far. */
NCF_API uint64_t ncf_launch_count(const ncf_ctx *ctx);
/* High-water mark of the device memory the context's workspaces have held (bytes;
 * workspaces grow on demand and are kept until ncf_destroy).  Plans and servers
 * report their own memory (ncf_plan_device_bytes, the server's budget).  No
 * counterpart in the paper: a serving metric. */
NCF_API size_t ncf_device_bytes(const ncf_ctx *ctx);

/*
 * Geometry of the most recent spectral call on this context: the common
 * period L of the Fourier series, the number of modes kept (m = 0 .. modes-1),
 * the oversampled grid size n_f, the spreading kernel width (cells), and the
 * batch size B and lag count K it served.  A batch whose series need grids of
 * very different sizes is split into `buckets` of series sharing a grid size,
 * each on its own period and grid (per-series grid sizing; Algorithm 1 applied
 * to each bucket's spans); period, modes and grid then describe the largest
 * bucket, and buckets = 1 means one grid for the batch.  All zero before any
 * spectral call.
 */
typedef struct {
    double period;
    int64_t modes, grid, width, B, K, buckets;
} ncf_plan_info;
NCF_API ncf_status ncf_last_plan(const ncf_ctx *ctx, ncf_plan_info *out);

/*
 * The autotuner's choices for the most recent evaluation of each kind on this
 * context (-1: none made yet).  rect_variant: the exact rectangle scan's design
 * (0, 1, 2: lags on lanes with runs of 16, 32, 64 outer points; 3: outer points
 * on lanes).  For the FP32 spectral form: fft_variant 0 = the FFT of an ACF grid
 * of 2^7..2^14 cells in shared memory, fused with its spectrum, 1 = global
 * Stockham passes (the only choice for larger grids and for CCFs);
 * contract_variant 0 = mode-to-lag contraction on tensor cores, 1 = on the FP32
 * pipe; spread_variant bit 0 = spreading by CTAs of 2048 points instead of 4096
 * (half the shared memory, more CTAs per SM), bit 1 = the CTA's tile summed in
 * fixed point by integer atomics instead of in FP32 by compare-and-swap.  Each
 * choice is the fastest of its candidates when first timed for a problem bucket
 * (device, sizes in powers of two, ACF/CCF), and is kept for the process;
 * NCF_RECT_VARIANT and NCF_SPEC_VARIANT (fft + 2 contraction + 4 spreading,
 * 0..15) in the environment pin them.  The estimators' results agree between variants:
 * bit for bit on the rectangle scan, within the FP32 form's error otherwise.
 * No counterpart in the paper (an implementation choice).
 */
typedef struct {
    int32_t rect_variant, fft_variant, contract_variant, spread_variant;
} ncf_tuning;
NCF_API ncf_status ncf_last_tuning(const ncf_ctx *ctx, ncf_tuning *out);

/*
 * Kernel profiler.  While enabled, every kernel the context launches is
 * bracketed by two CUDA events recorded on its launch stream.
 * ncf_profile_report synchronises on the recorded events, folds them into
 * per-kernel totals and writes lines "name launches total_ms\n" into buf
 * (NUL-terminated, truncated to len); it returns the full text length, or -1
 * for a NULL context.  ncf_profile_reset clears the totals.
 */
NCF_API ncf_status ncf_profile_enable(ncf_ctx *ctx, int on);
NCF_API int64_t ncf_profile_report(ncf_ctx *ctx, char *buf, size_t len);
NCF_API void ncf_profile_reset(ncf_ctx *ctx);

/*
 * One ACF (s == NULL and y == NULL) or CCF (x at t with y at s).
 *   t, x   [nx]  device FP64, t non-decreasing, nx >= 2
 *   s, y   [ny]  device FP64, s non-decreasing, ny >= 2 (ignored for the ACF)
 *   lags   [K]   device FP64, any order, repeats allowed, K >= 1
 *   c_out  [K]   device FP64: the estimate c_k, in the order of `lags`
 *   b_out  [K]   device FP64 or NULL: the effective pair count B_k (unclamped)
 *   count_out [K] device int64 or NULL: rectangle pair counts (exact); for the
 *                 Gaussian the number of pairs inside the window (windowed
 *                 path) or 0 (spectral path)
 */
NCF_API ncf_status ncf_corr(ncf_ctx *ctx,
                    const double *t, const double *x, int64_t nx,
                    const double *s, const double *y, int64_t ny,
                    const double *lags, int64_t K, const ncf_options *opt,
                    double *c_out, double *b_out, int64_t *count_out, void *stream);

/*
 * B independent ACFs (s == NULL) or CCFs on one shared lag grid, packed CSR:
 * series b is t[offs_x[b] .. offs_x[b+1]) (and s[offs_y[b] .. offs_y[b+1])).
 *   offs_x, offs_y  HOST int64 [B+1], offs[0] = 0, non-decreasing, each
 *                   series of length >= 2
 *   t, x, s, y      device FP64 arrays of length offs[B]
 *   lags [K]        device FP64 shared by every series
 *   c_out, b_out, count_out  device [B*K], row b holds series b (b_out,
 *                   count_out may be NULL)
 */
NCF_API ncf_status ncf_corr_batch(ncf_ctx *ctx, const int64_t *offs_x, const double *t, const double *x,
                          const int64_t *offs_y, const double *s, const double *y, int64_t B,
                          const double *lags, int64_t K, const ncf_options *opt,
                          double *c_out, double *b_out, int64_t *count_out, void *stream);

/*
 * ncf_corr_batch on HOST buffers: copies t, x (s, y) and lags to device
 * memory owned by the context, runs the batch, copies c (b, count) back and
 * synchronises the stream before returning.  Host buffers should be pinned
 * (cudaHostAlloc / torch pin_memory) for full copy bandwidth; pageable memory
 * works but copies synchronously.  Same argument meanings as ncf_corr_batch.
 */
NCF_API ncf_status ncf_corr_batch_host(ncf_ctx *ctx, const int64_t *offs_x, const double *t, const double *x,
                               const int64_t *offs_y, const double *s, const double *y, int64_t B,
                               const double *lags, int64_t K, const ncf_options *opt,
                               double *c_out, double *b_out, int64_t *count_out, void *stream);

/*
 * ncf_corr_batch with several option sets (estimators) on one batch whose
 * arrays are already on the device: the per-series statistics (the prior
 * standardisation step of Algorithms 2, 4, 9 and 10, which does not depend on
 * the kernel) are computed and validated once, then each option set runs its
 * own path on them.  Arguments as ncf_corr_batch, with opts[n_opts] and
 * c_out[o], b_out[o], count_out[o] DEVICE buffers of [B x K] (b_out,
 * count_out and any of their entries may be NULL).  Every result equals the one
 * ncf_corr_batch gives for that option set.  Errors as ncf_corr_batch; the
 * first failing option set ends the call.  n_opts < 1, a NULL opts or a NULL
 * c_out[o] gives NCF_EINVAL.
 */
NCF_API ncf_status ncf_corr_batch_multi(ncf_ctx *ctx, const int64_t *offs_x, const double *t, const double *x,
                                        const int64_t *offs_y, const double *s, const double *y, int64_t B,
                                        const double *lags, int64_t K, const ncf_options *opts, int n_opts,
                                        double *const *c_out, double *const *b_out, int64_t *const *count_out,
                                        void *stream);

/*
 * One very long series over several GPUs (or several passes of one GPU): the
 * estimator's sums are additive over the outer points, N_k = sum_j y_j
 * sum_i x_i b(s_j - t_i - tau_k) (Eq. kernel_estimator), so a series can be cut
 * into contiguous ranges of its outer points s_j, each evaluated against the
 * inner points t_i within reach of it (max|tau| plus the kernel's half-width),
 * and the ranges' partial N_k, B_k and pair counts summed.  Both need the
 * standardisation of the whole series (Appendix, "Prior standardization"),
 * pooled from the ranges' own statistics.
 *
 * ncf_series_stats runs the statistics pass of ONE series (device t, x, n >= 1
 * points) and returns, in *out (host): n, the mean, m2 = sum (x - mean)^2
 * (population variance m2 / n), the first and last times, and validation flags
 * (nonzero: 1 NaN or Inf present, 2 times decrease).  Pooling ranges a and b:
 * n = n_a + n_b, mean = mean_a + (mean_b - mean_a) n_b / n,
 * m2 = m2_a + m2_b + (mean_b - mean_a)^2 n_a n_b / n (Chan, Golub and LeVeque's
 * pairwise update).  Synchronises `stream`.
 *
 * ncf_corr_pooled is ncf_corr with the standardisation taken from *pooled
 * (the means, population standard deviations and total sizes of the whole
 * series, pooled as above) instead of from the given points; the given points'
 * own statistics pass still validates them (a range of constant values is
 * allowed).  Only NORM_NONE (normalise after summing the ranges); NCF_EINVAL for
 * means or std that are not finite and positive.  Results and errors otherwise
 * as ncf_corr; b_out and count_out (the range's B_k and exact pair counts) sum
 * over the ranges, and N_k = c_k max(B_k, 1e-16).
 */
typedef struct {
    int64_t n;
    double mean, m2, t_first, t_last;
    int32_t flags, pad;
} ncf_series_summary;
typedef struct {
    double mean_x, std_x;  /* pooled over every point of the x series */
    double mean_y, std_y;  /* the y series of a CCF (ignored for an ACF) */
    int64_t n_x, n_y;      /* total sizes of the series pooled over */
} ncf_pooled_stats;
NCF_API ncf_status ncf_series_stats(ncf_ctx *ctx, const double *t, const double *x, int64_t n,
                                    ncf_series_summary *out, void *stream);
NCF_API ncf_status ncf_corr_pooled(ncf_ctx *ctx, const double *t, const double *x, int64_t nx,
                                   const double *s, const double *y, int64_t ny, const double *lags,
                                   int64_t K, const ncf_options *opt, const ncf_pooled_stats *pooled,
                                   double *c_out, double *b_out, int64_t *count_out, void *stream);

/*
 * Several estimators of one batch from a single upload.  For example, the
 * Gaussian and the rectangle estimate of the same series (Eq. kernel_estimator
 * with Eq. Gaussian_kernel and Eq. rectangle_kernel).  It works as
 * ncf_corr_batch_host but takes n_opts option sets:
 *   - t, x (s, y) and lags are copied to the device once;
 *   - each chunk of series is evaluated with opts[0], ..., opts[n_opts - 1] in
 *     turn, on one statistics pass (the prior standardisation step of
 *     Algorithms 2, 4, 9 and 10 does not depend on the kernel);
 *   - the results are written to the HOST buffers c_out[o], b_out[o] and
 *     count_out[o], each [B x K].
 * b_out and count_out may be NULL, and so may any of their entries.
 * Every result equals the one ncf_corr_batch_host gives for that option set.
 * Errors are those of ncf_corr_batch_host.  The first failing option set ends
 * the call; the outputs of the other sets are then undefined.  n_opts < 1, a
 * NULL opts or a NULL c_out[o] gives NCF_EINVAL.
 */
NCF_API ncf_status ncf_corr_batch_host_multi(ncf_ctx *ctx, const int64_t *offs_x, const double *t,
                                             const double *x, const int64_t *offs_y, const double *s,
                                             const double *y, int64_t B, const double *lags, int64_t K,
                                             const ncf_options *opts, int n_opts, double *const *c_out,
                                             double *const *b_out, int64_t *const *count_out, void *stream);


/*
 * The paper's own NUFFT estimators, smoothing step included (Appendix
 * "NUFFT-based ACF/CCF algorithms", Algorithms 1-4), for users who need the
 * published package's numbers rather than Eq. kernel_estimator itself:
 *   Algorithm 1  L = span + 2 max|tau| (lag 0 included), t_c = t_min + span/2,
 *                N1 = round(32 n_max L / span) (Eq. N1_default; N1 > 0 overrides);
 *   Algorithm 2  CCF: type-1 transforms of the standardised x and y on the map
 *                t -> pi + 2 pi (t - t_c) / L (N1 modes k = -floor(N1/2) ..
 *                ceil(N1/2) - 1, exp(+i k t~)), cross spectrum conj(F1) F2, its
 *                type-2 transform (exp(-i k tau~)) at the sorted lags with lag 0
 *                prepended, the smoothing S_h along that sorted array, division
 *                by the pair count, unsorting, division by sqrt(ACF_x(0) ACF_y(0));
 *   Algorithm 3  ACF(0) of each series for that scale, smoothed at the centre of
 *                the array -n_h .. n_h, n_h = max(ceil(4h) + 2, 5);
 *   Algorithm 4  ACF: the same with |F|^2, normalised by the prepended lag 0.
 * S_h (the paper names it without fixing edges or truncation; this library
 * reads it as scipy.ndimage's defaults): Gaussian weights exp(-j^2 / 2h^2),
 * |j| <= int(4h + 0.5), unit sum; rectangle: the mean of round(2h) entries
 * j = -size/2 .. size - 1 - size/2 (round half to even, size >= 1); both with
 * half-sample reflection at the array ends.  PairCount (Algorithms 5, 6): the
 * Gaussian summed over [c - 6h, c + 6h), the rectangle counted in [c - h, c + h].
 * The smoothing acts on array positions, so the result matches Eq.
 * kernel_estimator only for integer times with unit lag spacing; the
 * transforms are evaluated to about 1e-13 relative (no FINUFFT tolerance).
 *
 * DEVICE pointers as ncf_corr: t, x [nx], s, y [ny] (both NULL for an ACF),
 * lags [K] (any order), c_out [K], b_out [K] or NULL (PairCount clamped below
 * at 1e-16).  kernel: NCF_GAUSSIAN or NCF_RECTANGLE (NCF_EUNSUPPORTED
 * otherwise).  The data must span a positive interval (NCF_EDEGENERATE) and
 * N1 must fit a grid of 2^27 cells, N1 <= about 6.7e7 (NCF_EUNSUPPORTED).
 * Other errors as ncf_corr.  Several host synchronisations (statistics, lags,
 * and the pair counts, which run through ncf_corr's windowed paths).
 */
NCF_API ncf_status ncf_corr_paper(ncf_ctx *ctx, const double *t, const double *x, int64_t nx,
                                  const double *s, const double *y, int64_t ny, const double *lags, int64_t K,
                                  ncf_kernel kernel, double h, int64_t N1, double *c_out, double *b_out,
                                  void *stream);

/*
 * Classic-FFT estimator for data on a regular grid (the paper's dedicated FFT
 * path for regularly sampled series, Table 1 and Sec. 5.2): every time is a
 * whole multiple of one step, t_i = m_x[i] dt and s_j = m_y[j] dt, so a pair's
 * separation is d dt for an integer d and Eq. kernel_estimator becomes
 * N(tau) = sum_d R(d) b(d dt - tau), B(tau) = sum_d C(d) b(d dt - tau), with R
 * the raw correlation of the standardised values and C the number of pairs at
 * separation d, both from FFTs of the zero-padded lattice; the cost does not
 * grow with K.  Gaussian (untruncated to within 1.3e-14: separations beyond
 * 8 h are dropped) or rectangle (|fl(d dt - tau)| <= h in FP64; exact int64
 * pair counts), NORM_NONE or NORM_LAG0, FP64 throughout; opt->path and
 * opt->precision are ignored.  It equals the general estimator on the times
 * m dt except where a rectangle bound falls exactly on a pair separation
 * (there the general path tests the rounded times, this path the lattice).
 *
 * DEVICE pointers: m_x [nx] (int64 lattice indices, non-decreasing; equal
 * indices are distinct samples at one time), x [nx]; for a CCF m_y, y [ny]
 * on the same lattice (both NULL for an ACF); lags [K] (any order); outputs
 * c_out, b_out (nullable), count_out (nullable; 0 for the Gaussian) [K].  The
 * lattice span plus the lags' reach, (max m - min m) + (max|tau| + reach)/dt,
 * must stay below 2^29 cells (NCF_EUNSUPPORTED otherwise).  Errors: NCF_EINVAL,
 * NCF_ENOTSORTED, NCF_ENONFINITE, NCF_EDEGENERATE, NCF_ENOMEM, NCF_ECUDA.  One
 * host synchronisation (statistics and lags are read back to size the grid).
 */
NCF_API ncf_status ncf_corr_regular(ncf_ctx *ctx, const int64_t *m_x, const double *x, int64_t nx,
                                    const int64_t *m_y, const double *y, int64_t ny, double dt,
                                    const double *lags, int64_t K, const ncf_options *opt,
                                    double *c_out, double *b_out, int64_t *count_out, void *stream);

/*
 * Self-test of failure detection (no counterpart in the paper): runs a kernel
 * whose mbarrier wait -- the bounded wait the tensor-core contraction uses --
 * is never satisfied, so it must give up after a short iteration limit, set
 * the timeout bit of a device status word and return normally.  *flags
 * receives that word (bit 1, the timeout bit of ncf_plan_status, expected).
 * Returns NCF_OK when the timeout was reported; the context stays usable
 * either way.
 */
NCF_API ncf_status ncf_selftest_bounded_wait(ncf_ctx *ctx, void *stream, int32_t *flags);

/*
 * Bootstrap replicates of one ACF (s = y = NULL) or CCF, for per-lag sampling
 * uncertainties.  The paper recommends weighing an estimate against its
 * sampling variance by resampling or Monte-Carlo over realisations (Sec. 4,
 * "Monte-Carlo over independent realizations"; Sec. 6) but provides no
 * resampler; this entry point has no counterpart in it.
 *
 * Replicate r (0 <= r < n_boot) resamples the nx points of (t, x) with
 * replacement, keeping time order, and for a CCF the ny points of (s, y)
 * independently, then evaluates the estimator with *opt exactly as
 * ncf_corr_batch would on the batch of replicates.  Draw j of replicate r on
 * the x side is point floor(nx * u / 2^64), u = the SplitMix64 output number
 * c = 2^32 r + j of the stream started at `seed` (output c is
 * mix(seed + (c + 1) 0x9E3779B97F4A7C15) with the mixing of Steele, Lea and
 * Flood); the y side uses the stream started at ~seed.
 *
 * All arrays are DEVICE pointers: t, x [nx] and s, y [ny] (t, s
 * non-decreasing), lags [K], outputs c_out, b_out, count_out [n_boot][K]
 * (b_out and count_out may be NULL).  nx, ny, n_boot < 2^32.  The replicates
 * live in a context buffer of 16 (nx + ny) n_boot + 4 max(nx, ny) n_boot
 * bytes.  Errors: NCF_EINVAL for NULL pointers or sizes out of range, the
 * statuses of ncf_corr_batch otherwise (NCF_EDEGENERATE when a replicate
 * drew a single distinct value, which short series make likely).
 */
NCF_API ncf_status ncf_corr_bootstrap(ncf_ctx *ctx, const double *t, const double *x, int64_t nx,
                                      const double *s, const double *y, int64_t ny,
                                      const double *lags, int64_t K, const ncf_options *opt,
                                      int64_t n_boot, uint64_t seed, double *c_out, double *b_out,
                                      int64_t *count_out, void *stream);
/*
 * Plans: the analysis of one batch layout, lag set and options, done once,
 * for repeated launches that neither synchronise nor allocate, so a launch
 * can be captured in a CUDA graph.
 *
 * ncf_plan_create runs exactly what ncf_corr_batch runs before its kernels
 * (argument and data validation, statistics read-back, geometry, tables) on
 * the given data, and allocates the plan's own device memory
 * (ncf_plan_device_bytes).  Same arguments as ncf_corr_batch; the lags are
 * copied into the plan.  Returns after synchronising `stream`.
 *
 * ncf_plan_execute launches the kernels on `stream` for data laid out like the
 * data of the plan (same CSR offsets, same lags): statistics and keys are
 * recomputed from the new t, x (s, y); nothing is allocated or copied from the
 * host and the host does not wait.  The plan's geometry (period, grid, key
 * scale) must still fit the new data; device-side checks set bits of a
 * status word instead of returning an error:
 *     1  a bounded device wait gave up           4  times beyond the key range
 *     2  a series outside the periodic domain    8  unsorted / non-finite / constant input
 * and every output of that launch is NaN (count -1).  ncf_plan_status
 * synchronises `stream`, stores the word in *flags and returns NCF_OK (0),
 * NCF_ETIMEOUT (bit 1), NCF_EINVAL (bit 8) or NCF_EUNSUPPORTED (bits 2, 4:
 * build a new plan).  A plan belongs to the context it was created with and,
 * like it, is not thread-safe; launches of one plan must not overlap.
 */
typedef struct ncf_plan ncf_plan;
NCF_API ncf_status ncf_plan_create(ncf_ctx *ctx, const int64_t *offs_x, const double *t, const double *x,
                                   const int64_t *offs_y, const double *s, const double *y, int64_t B,
                                   const double *lags, int64_t K, const ncf_options *opt, void *stream,
                                   ncf_plan **out);
NCF_API ncf_status ncf_plan_execute(ncf_plan *plan, const double *t, const double *x, const double *s,
                                    const double *y, double *c_out, double *b_out, int64_t *count_out,
                                    void *stream);
NCF_API ncf_status ncf_plan_status(ncf_plan *plan, void *stream, int32_t *flags);
/*
 * A plan of several option sets (estimators) on the same data: ncf_plan_create
 * with opts[n_opts].  ncf_plan_execute_multi runs the statistics pass once
 * (the prior standardisation step of Algorithms 2, 4, 9 and 10 does not depend
 * on the kernel) and then every option set's kernels, writing c_out[o], b_out[o]
 * and count_out[o] (DEVICE [B x K]; b_out, count_out and their entries may be
 * NULL).  Like ncf_plan_execute it neither allocates nor synchronises, so it can
 * be captured in a CUDA graph; one status word covers every set.
 * ncf_plan_execute on such a plan runs the first option set only;
 * ncf_plan_option_sets returns n_opts.
 */
NCF_API ncf_status ncf_plan_create_multi(ncf_ctx *ctx, const int64_t *offs_x, const double *t, const double *x,
                                         const int64_t *offs_y, const double *s, const double *y, int64_t B,
                                         const double *lags, int64_t K, const ncf_options *opts, int n_opts,
                                         void *stream, ncf_plan **out);
NCF_API ncf_status ncf_plan_execute_multi(ncf_plan *plan, const double *t, const double *x, const double *s,
                                          const double *y, double *const *c_out, double *const *b_out,
                                          int64_t *const *count_out, void *stream);
NCF_API int ncf_plan_option_sets(const ncf_plan *plan);
NCF_API size_t ncf_plan_device_bytes(const ncf_plan *plan);

/*
 * Device footprint of an evaluation, known before anything is allocated (the
 * paper's single calling convention, Sec. 2.6 "Unified API": the same options,
 * sizes and lag count as the call it sizes).  Host arithmetic only: no GPU work,
 * no allocation, no synchronisation; ctx may be NULL (no error text is kept).
 *   n_x        total points of the x side of the batch (sum over its B series)
 *   n_y        total points of the y side, or 0 for ACFs
 *   B, K       series and lags (K >= 1; each series needs >= 2 points)
 *   span       the largest time span of one series (for a CCF, of the union of
 *              its two series); the spectral grid grows with span / h
 *   max_abs_lag  the largest |tau_k|
 *   opt        the options of the call
 * *device_bytes receives an upper bound of the device memory that
 * ncf_corr_batch (or ncf_corr for B = 1) asks its context's workspace for, and
 * of what ncf_plan_create allocates (ncf_plan_device_bytes), for any batch of
 * these sizes whose largest span is at most `span`: the bound holds for every
 * split of the points into the B series.  With NCF_PATH_AUTO for the FP64
 * Gaussian, whose path is chosen from the data, it covers both paths.  The
 * request server admits requests against its budget with this bound.  *pinned_bytes (may be NULL)
 * receives the context's pinned host staging.  Not included: the caller's own
 * inputs and outputs, and what the host-buffer calls add: the uploaded copies
 * (16 bytes per point plus 8 per lag), and a second pre-statistics workspace and
 * pinned staging for the next chunk's statistics stage, which runs beside the
 * current chunk's evaluation (about 64 bytes per series plus 28 per 4096
 * points).  Returns NCF_EINVAL or NCF_EUNSUPPORTED for options
 * or sizes that the calls would refuse (a spectral grid beyond 2^28 cells).
 */
NCF_API ncf_status ncf_workspace_bytes(ncf_ctx *ctx, int64_t n_x, int64_t n_y, int64_t B, int64_t K,
                                       double span, double max_abs_lag, const ncf_options *opt,
                                       size_t *device_bytes, size_t *pinned_bytes);
NCF_API void ncf_plan_destroy(ncf_plan *plan);

/*
 * Serving: a continuous-batching request loop on one GPU.
 *
 * ncf_server_create starts `slots` worker threads, each with its own CUDA
 * stream and context, on `device`.  ncf_server_submit admits one ACF/CCF
 * request (HOST buffers, which must stay valid until ncf_server_wait returns
 * for its ticket) if a slot is free and the estimated device memory of all
 * admitted requests stays within mem_budget_bytes; otherwise it returns
 * NCF_EBUSY at once and the caller retries later.  Admitted requests run
 * concurrently, each exactly as ncf_corr on its own stream, so their kernels
 * overlap on the device and each result equals the request run alone (up to
 * floating-point summation order).  ncf_server_poll reports completion;
 * ncf_server_wait blocks until the request is done, copies c, b, count
 * (each [K], NULL to skip) to host memory, returns the request's status and
 * its latency (submit to completion).  ncf_server_latency reports the 50th
 * and 99th percentile latencies of all completed requests.
 *
 * Resident series: ncf_server_put copies a series (host t, x; n >= 2 points)
 * once into device memory owned by the server, charged to the memory budget
 * until ncf_server_drop, and returns its handle (NCF_EBUSY when the budget
 * cannot hold it).  A request names resident series through x_series /
 * y_series; their host pointers and sizes are then ignored and nothing is
 * copied per request.  ncf_server_drop returns NCF_EBUSY while an admitted
 * request still uses the series, NCF_EINVAL for an unknown handle.
 */
typedef struct {
    const double *t, *x;   /* HOST, nx points, t non-decreasing (ignored when x_series != 0) */
    int64_t nx;
    const double *s, *y;   /* HOST, ny points (NULL, NULL for an ACF; ignored when y_series != 0) */
    int64_t ny;
    const double *lags;    /* HOST [K] */
    int64_t K;
    ncf_options opt;
    uint64_t x_series;     /* 0, or a resident series used as (t, x) */
    uint64_t y_series;     /* 0, or a resident series used as (s, y): a CCF */
} ncf_request;
typedef struct ncf_server ncf_server;
NCF_API ncf_status ncf_server_create(int device, size_t mem_budget_bytes, int slots, ncf_server **out);
NCF_API ncf_status ncf_server_put(ncf_server *srv, const double *t, const double *x, int64_t n, uint64_t *series);
NCF_API ncf_status ncf_server_drop(ncf_server *srv, uint64_t series);
NCF_API ncf_status ncf_server_submit(ncf_server *srv, const ncf_request *req, uint64_t *ticket);
NCF_API ncf_status ncf_server_poll(ncf_server *srv, uint64_t ticket, int *done);
NCF_API ncf_status ncf_server_wait(ncf_server *srv, uint64_t ticket, double *c_out, double *b_out,
                                   int64_t *count_out, double *latency_ms);
NCF_API ncf_status ncf_server_latency(ncf_server *srv, double *p50_ms, double *p99_ms, uint64_t *completed);
NCF_API void ncf_server_destroy(ncf_server *srv);

/*
 * Allocation-free variant of the Gaussian windowed estimator (no counterpart
 * in the paper; it exists for callers that must not allocate device memory
 * while running, such as real-time or embedded pipelines with a fixed memory
 * plan, or plug-ins inside a framework whose allocator owns the device).
 *
 * Same arguments and results as ncf_corr with kernel = NCF_GAUSSIAN, path =
 * NCF_PATH_WINDOWED, precision = NCF_FP64, norm = NCF_NORM_NONE (window
 * [c - R h, c + R h), R = trunc_R, 0 selects 8), for ONE series (s, y NULL:
 * ACF) or one pair (CCF); all arrays are device pointers, b_out may be NULL.
 * No context is needed and nothing is allocated: the scratch is a fixed
 * 64 KiB array compiled into the library, present on every GPU that loads
 * the library until the process exits.
 *   Limits: nx, ny <= 262144 points, K <= 1024 lags; larger inputs return
 *   NCF_EUNSUPPORTED (use ncf_corr).  Other errors as for ncf_corr
 *   (NCF_EINVAL, NCF_ENOTSORTED, NCF_ENONFINITE, NCF_EDEGENERATE, NCF_ECUDA).
 *   The first call on a device looks up the scratch array's device address
 *   (cudaGetSymbolAddress) with that device current.  The call synchronises
 *   `stream` once (input validation).
 *   All calls share the one scratch array: calls that may overlap on the GPU
 *   (other streams or host threads) race and must be serialised by the caller.
 */
NCF_API ncf_status ncf_corr_window_static(const double *t, const double *x, int64_t nx,
                                          const double *s, const double *y, int64_t ny,
                                          const double *lags, int64_t K, double h, double trunc_R,
                                          double *c_out, double *b_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* NCF_H */
