// spectral.cuh -- the Wiener-Khinchin (NUFFT) path for the Gaussian kernel.
#pragma once

#include <string>
#include <memory>
#include <vector>

#include "common.cuh"

namespace ncf {

struct SpecSide {
    const double *t = nullptr, *v = nullptr;  // device times and values
    const int64_t *d_offs = nullptr;          // device CSR offsets [B+1]
    const SeriesStats *d_stats = nullptr;     // device per-series statistics
    const int64_t *h_offs = nullptr;          // host CSR offsets [B+1]
    const SeriesStats *h_stats = nullptr;     // host copy of the statistics
    int64_t n_total = 0, n_max = 0;
    const int64_t *d_chunk_base = nullptr;    // device chunk table of the statistics pass
    int64_t n_chunks = 0;
    const int32_t *d_cs = nullptr;            // series of each chunk
    const int64_t *d_offs_end = nullptr;      // device end offsets [B] (NULL: d_offs + 1)
};

struct SpectralArgs {
    bool acf = true, fp32 = false, lag0 = false;
    int kernel = 0;  // NCF_GAUSSIAN (b-hat Gaussian) or NCF_RECTANGLE (the spectral-sinc variant)
    int64_t B = 0, K = 0;
    double h = 1.0, tol = 1e-14, max_tau = 0.0;
    const double *lags = nullptr;    // device [K]
    const double *h_lags = nullptr;  // host copy [K]
    SpecSide x, y;
    double *c_out = nullptr, *b_out = nullptr;
    int64_t *count_out = nullptr;
    const int64_t *row_map = nullptr;  // device [B]: output row of series b (NULL: b)
    int sm_count = 148;
    bool no_buckets = false;           // plan one common grid (a bucket's own plan)
};

struct SpectralBucket;

// Geometry and host tables of a spectral evaluation (spectral_plan), kept by
// one-shot calls and by ncf_plan objects alike.  A batch whose series need grids
// of very different sizes is split into buckets of series sharing a grid size,
// each with its own plan (period, grid, lag table, workspace); the geometry
// fields then describe the largest bucket.
struct SpectralPrepared {
    double L = 0, beta = 0, R_alias = 0, h = 0, max_tau = 0;
    int64_t M = 0, Mp = 0, K1 = 0, Kp = 0, M2 = 0, B = 0, K = 0;
    int nf = 0, lg = 0, W = 8, nq = 64;
    bool fp32 = false, acf = true, lag0 = false;
    bool direct = false;  // one FP64 series: mode sums at the lags, no lag table
    // FP32 shapes chosen by the autotuner: FFT of an ACF grid of 2^7..2^14 cells in
    // shared memory fused with its spectrum (0) or as global passes (1); the
    // contraction on tensor cores (0) or on the FP32 pipe (1)
    int fft_variant = 0, contract_variant = 0;
    // FP32 spreading: bit 0, CTAs of half a statistics chunk of points (half the
    // shared memory, more CTAs per SM); bit 1, the CTA's tile of cells summed in
    // fixed point by native integer shared-memory atomics instead of in FP32 by
    // compare-and-swap loops
    int spread_variant = 0;
    double tap_sum = 0;  // an upper bound of sum_k phi_k(u) over the W taps of one point
    int kernel = 0;
    std::vector<double> tc, gx, gphi, poly;
    std::vector<unsigned long long> phi;
    std::vector<std::shared_ptr<SpectralBucket>> buckets;  // empty: one grid for the batch
};

// Host-side planning: geometry, tables, workspace sizes (device, pinned staging).
ncf_status spectral_plan(const SpectralArgs &a, SpectralPrepared *sp, size_t *ws_bytes,
                         size_t *pinned_bytes, std::string *msg);
// Host staging a plan split into grid-size buckets may need beyond one grid's.
size_t spectral_bucket_pinned_allowance(int64_t B, int64_t K, int64_t n_x, int64_t n_y, bool ccf);
// Uploads the host tables and builds the device tables (mode weights,
// twiddles, lag table) in `ws`.
void spectral_prepare(const SpectralPrepared &p, char *ws, char *pinned, cudaStream_t st);
// The per-data kernels: spreading, FFT, spectra, contraction, normalisation.
// *status is read by the normalisation (nonzero -> NaN results).
ncf_status spectral_launch(const SpectralArgs &a, const SpectralPrepared &p, char *ws, int *status,
                           cudaStream_t st, std::string *msg);
// Device check that the series still fit the plan's periodic domain.
void spectral_guard(const SpectralArgs &a, const SpectralPrepared &p, char *ws, int *status,
                    cudaStream_t st);

// Tensor-core contraction of the FP32 form (k_tc.cu): acc_c += A_c E over all
// modes, TF32 split products, FP32 TMEM accumulation per chunk of modes, FP64
// partial sums.  The operands are first packed into split, swizzled tiles
// (launch_tc_pack_a per execution, launch_tc_pack_e when the lag table is
// made).  *status becomes nonzero if a bounded wait gave up.
bool contract_tc_supported(int64_t M2);
size_t tc_a_tiles_bytes(int64_t B, int64_t M2);
size_t tc_e_tiles_bytes(int64_t M2, int64_t Kp);
void launch_tc_pack_a(const float *Anum, const float *Aden, int64_t B, int64_t M2, unsigned char *At,
                      cudaStream_t st);
void launch_tc_pack_e(const float *E, int64_t M2, int64_t Kp, unsigned char *Et, cudaStream_t st);
void launch_contract_tc(const unsigned char *At, const unsigned char *Et, int64_t B, int64_t M2, int64_t Kp,
                        int sm_count, double *acc_num, double *acc_den, int *status, cudaStream_t st);

// FP64 forward FFT passes shared with the regular-grid path (k_spectral.cu).
void fft_twiddles_f64(double2 *tw, int lg, cudaStream_t st);
double2 *fft_forward_f64(double2 *grid, double2 *scratch, const double2 *tw, int lg, int64_t B, cudaStream_t st);

// The paper's own NUFFT estimators (Algorithms 2-4 with the smoothing step):
// geometry of the type-1 transforms on the padded period L of Algorithm 1.
struct PaperModes {
    double L = 0.0, tc = 0.0;
    int64_t N1 = 0, Mh = 0;  // coefficients m = 0 .. Mh = floor(N1 / 2)
    int lg = 0, nf = 0, W = 16, nq = 128;
    double beta = 0.0;
    std::vector<double> gx, gphi, poly;
};
ncf_status paper_modes_plan(double L, double tc, int64_t N1, PaperModes *pm, std::string *msg);
size_t paper_modes_bytes(const PaperModes &pm, bool ccf);
size_t paper_modes_pinned_bytes(const PaperModes &pm);
// F_m = sum_j x_std,j exp(+2 pi i m (t_j - t_c) / L), m = 0 .. Mh, of side x
// (and y), by ES spreading, FFT and deconvolution; *Fx, *Fy point into ws.
void paper_modes_run(const PaperModes &pm, const SpecSide &x, const SpecSide *y, char *ws, char *pinned,
                     double2 **Fx, double2 **Fy, cudaStream_t st);
// c[k] = Re sum_{m=0}^{Mh} A_m exp(-2 pi i m tau_k / L) by a type-2 transform on the
// grid of paper_modes_run (after it): deconvolution, one FFT, W-tap interpolation at
// each lag from its phase phi[k] = frac(tau_k / L) 2^64.  Overwrites the grids.
void paper_type2(const PaperModes &pm, bool ccf, char *ws, const double2 *A, const unsigned long long *phi,
                 int64_t K, double *c, cudaStream_t st);

// k_paper.cu: A_m = fac_m conj(Fa_m) Fb_m (fac 1 at m = 0 and, N1 even, at
// m = N1/2; 2 otherwise); c[k] += sum_m Re(A_m exp(-2 pi i m tau_k / L)) with
// phi[k] = frac(tau_k / L) 2^64 (c zeroed by the caller); the smoothing,
// pair-count division, normalisation and unsorting of Algorithms 2-4.
void paper_spectrum(const double2 *Fa, const double2 *Fb, int64_t Mh, int64_t N1, double2 *A, cudaStream_t st);
// (with A1, c1: a second spectrum at the same lags in the same launch)
void paper_eval(const double2 *A, int64_t Mh, const unsigned long long *phi, int64_t K, double *c,
                cudaStream_t st, const double2 *A1 = nullptr, double *c1 = nullptr);
void paper_finish(const double *craw, const double *bsrt, int64_t K1, const int64_t *perm, int64_t pos0,
                  const double *w, int nw, int o0, bool acf, const double *craw_x, const double *craw_y,
                  int64_t nsym, const double *bx0, const double *by0, double *tmp, double *c_out,
                  double *b_out, cudaStream_t st);

// Self-test: a bounded mbarrier wait that nothing completes sets STATUS_TIMEOUT (k_tc.cu).
void launch_bounded_wait_selftest(int *status, cudaStream_t st);

}  // namespace ncf
