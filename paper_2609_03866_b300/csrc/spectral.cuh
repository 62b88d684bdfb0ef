// spectral.cuh -- the Wiener-Khinchin (NUFFT) path for the Gaussian kernel.
#pragma once

#include <string>

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
};

struct SpectralArgs {
    bool acf = true, fp32 = false, lag0 = false;
    int64_t B = 0, K = 0;
    double h = 1.0, tol = 1e-14, max_tau = 0.0;
    const double *lags = nullptr;    // device [K]
    const double *h_lags = nullptr;  // host copy [K]
    SpecSide x, y;
    double *c_out = nullptr, *b_out = nullptr;
    int64_t *count_out = nullptr;
    int sm_count = 148;
};

// Geometry chosen by the last run_spectral call (reported through ncf_last_plan).
struct SpectralGeometry { double L; int64_t M, nf, W; };

// Tensor-core contraction of the FP32 form (k_tc.cu): acc_c += A_c E over all
// modes, TF32 split products, FP32 TMEM accumulation per 512-mode chunk, FP64
// partial sums.  *status becomes nonzero if a bounded wait gave up.
bool contract_tc_supported(int64_t M2);
void launch_contract_tc(const float *Anum, const float *Aden, const float *E, int64_t B, int64_t M2,
                        int64_t Kp, double *acc_num, double *acc_den, int *status, cudaStream_t st);

// Runs the spectral path on `st`; grows *ws (device) and *pinned (host) as
// needed.  Returns NCF_OK or an error with *msg set.
ncf_status run_spectral(const SpectralArgs &a, char **ws, size_t *ws_cap, char **pinned,
                        size_t *pinned_cap, cudaStream_t st, std::string *msg,
                        SpectralGeometry *geom);

}  // namespace ncf
