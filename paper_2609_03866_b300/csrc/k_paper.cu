// k_paper.cu -- the paper's own NUFFT estimators (Appendix "NUFFT-based
// ACF/CCF algorithms": Algorithms 2-4, with the smoothing step S_h).
//
// Given the deconvolved type-1 coefficients F_m, m = 0 .. floor(N1/2), of the
// standardised series on the padded period L (k_spectral.cu), these kernels
//   spectrum  form A_m = fac_m conj(Fa_m) Fb_m: the cross spectrum of
//             Algorithm 2, or |F_m|^2 (Algorithms 3 and 4).  The N1 modes
//             k = -floor(N1/2) .. ceil(N1/2) - 1 of the transforms pair k with -k
//             (real series: F_{-k} = conj(F_k)), so fac = 2, except fac = 1 at
//             m = 0 and, for even N1, at the unpaired m = N1/2;
//   eval      the type-2 transform at the lags, as the direct sum
//             c_raw(tau) = sum_m Re(A_m exp(-2 pi i m tau / L)):
//             the raw Dirichlet-kernel correlation of the paper;
//   finish    S_h along the sorted lag array (Gaussian of width h or a box of
//             round(2h) entries, reflecting edges), division by the pair
//             counts, normalisation by the lag-0 entry (ACF) or by
//             sqrt(ACF_x(0) ACF_y(0)) from the interior of the symmetric lag
//             array (CCF, Algorithm 3), and unsorting.
#include "spectral.cuh"

namespace ncf {

namespace {

constexpr int kEvalWarps = 8;     // warps of an evaluation CTA
constexpr int kEvalModes = 256;   // modes summed by one warp (one lag per lane)

__global__ void paper_spectrum_kernel(const double2 *__restrict__ Fa, const double2 *__restrict__ Fb,
                                      int64_t Mh, int64_t N1, double2 *__restrict__ A) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m > Mh) return;
    const double fac = (m == 0 || (N1 % 2 == 0 && m == Mh)) ? 1.0 : 2.0;
    const double2 a = Fa[m], b = Fb[m];
    A[m] = make_double2(fac * (a.x * b.x + a.y * b.y), fac * (a.x * b.y - a.y * b.x));
}

// c[k] += sum over this warp's modes of Re(A_m exp(-2 pi i m tau_k / L)).
// phi[k] = frac(tau_k / L) 2^64: the phase of mode m is m phi[k] mod 2^64,
// exact in integer arithmetic, so each warp starts its run of modes from an
// exactly reduced angle and steps with the rotation exp(-2 pi i tau_k / L).
__global__ void __launch_bounds__(kEvalWarps * 32)
paper_eval_kernel(const double2 *__restrict__ A0, const double2 *__restrict__ A1, int64_t Mh,
                  const unsigned long long *__restrict__ phi, int64_t K, double *__restrict__ c0,
                  double *__restrict__ c1) {
    // blockIdx.z selects one of two spectra evaluated at the same lags
    const double2 *__restrict__ A = blockIdx.z ? A1 : A0;
    double *__restrict__ c = blockIdx.z ? c1 : c0;
    __shared__ double part[kEvalWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // With 16 lags or fewer (one lag tile), S = 32 / K lanes share a lag and take
    // every S-th mode of the warp's run, so that no lane idles; else S = 1.
    const int S = (K <= 16) ? (int)(32 / K) : 1;
    const int64_t k = (int64_t)blockIdx.y * 32 + lane / S;
    const int sub = lane % S;
    const int64_t m0 = ((int64_t)blockIdx.x * kEvalWarps + warp) * kEvalModes;
    double acc = 0.0;
    if (k < K && lane / S < 32 / S && m0 + sub <= Mh) {
        const unsigned long long ph = phi[k];
        const unsigned long long p0 = (unsigned long long)(m0 + sub) * ph;
        const unsigned long long pstep = (unsigned long long)S * ph;
        double zs, zc, rs, rc;
        sincospi(2.0 * ((double)(p0 >> 11) * 0x1.0p-53), &zs, &zc);
        sincospi(2.0 * ((double)(pstep >> 11) * 0x1.0p-53), &rs, &rc);
        const int64_t m1 = min(m0 + kEvalModes, Mh + 1);
        for (int64_t m = m0 + sub; m < m1; m += S) {
            const double2 a = A[m];
            acc = fma(a.x, zc, fma(a.y, zs, acc));  // Re[(a.x + i a.y)(cos - i sin)]
            const double c2 = fma(zc, rc, -zs * rs);
            zs = fma(zs, rc, zc * rs);
            zc = c2;
        }
    }
    part[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && lane < 32 / S) {
        const int64_t kk = (int64_t)blockIdx.y * 32 + lane;
        if (kk < K) {
            double s = 0.0;
            for (int w = 0; w < kEvalWarps; ++w)
                for (int j = 0; j < S; ++j) s += part[w][lane * S + j];
            atomicAdd(c + kk, s);
        }
    }
}

__device__ __forceinline__ int64_t reflect(int64_t q, int64_t n) {
    int64_t r = q % (2 * n);
    if (r < 0) r += 2 * n;
    return r < n ? r : 2 * n - 1 - r;
}

// S_h at position i of an array of n entries: weights w[0 .. nw) at offsets
// o0 .. o0 + nw - 1, half-sample reflection at both ends.
__device__ __forceinline__ double smooth_at(const double *__restrict__ a, int64_t n, int64_t i,
                                            const double *__restrict__ w, int nw, int o0) {
    double s = 0.0;
    for (int j = 0; j < nw; ++j) s = fma(w[j], a[reflect(i + o0 + j, n)], s);
    return s;
}

// One CTA.  craw, bsrt: raw correlation and pair counts at the sorted lags
// (K1 = K + 1 entries, the prepended lag 0 at sorted position pos0); perm[i]:
// index in (0, tau_1 .. tau_K) of sorted entry i.  CCF: craw_x, craw_y on the
// symmetric array of nsym entries and the lag-0 pair counts bx0, by0.
__global__ void paper_finish_kernel(const double *__restrict__ craw, const double *__restrict__ bsrt,
                                    int64_t K1, const int64_t *__restrict__ perm, int64_t pos0,
                                    const double *__restrict__ w, int nw, int o0, int acf,
                                    const double *__restrict__ craw_x, const double *__restrict__ craw_y,
                                    int64_t nsym, const double *__restrict__ bx0,
                                    const double *__restrict__ by0, double *__restrict__ tmp,
                                    double *__restrict__ c_out, double *__restrict__ b_out) {
    __shared__ double norm;
    for (int64_t i = threadIdx.x; i < K1; i += blockDim.x)
        tmp[i] = smooth_at(craw, K1, i, w, nw, o0) / fmax(bsrt[i], 1e-16);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (acf) {
            norm = tmp[pos0];
        } else {
            const int64_t ctr = nsym / 2;
            const double sx = smooth_at(craw_x, nsym, ctr, w, nw, o0) / fmax(*bx0, 1e-16);
            const double sy = smooth_at(craw_y, nsym, ctr, w, nw, o0) / fmax(*by0, 1e-16);
            norm = sqrt(sx * sy);
        }
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < K1; i += blockDim.x) {
        const int64_t o = perm[i];
        if (o < 1) continue;
        c_out[o - 1] = tmp[i] / norm;
        if (b_out) b_out[o - 1] = fmax(bsrt[i], 1e-16);
    }
}

}  // namespace

void paper_spectrum(const double2 *Fa, const double2 *Fb, int64_t Mh, int64_t N1, double2 *A, cudaStream_t st) {
    NCF_LAUNCH("paper_spectrum_kernel", st,
               paper_spectrum_kernel<<<(unsigned)((Mh + 256) / 256), 256, 0, st>>>(Fa, Fb, Mh, N1, A));
}

void paper_eval(const double2 *A, int64_t Mh, const unsigned long long *phi, int64_t K, double *c,
                cudaStream_t st, const double2 *A1, double *c1) {
    const int64_t per_cta = (int64_t)kEvalWarps * kEvalModes;
    dim3 grid((unsigned)((Mh + per_cta) / per_cta), (unsigned)((K + 31) / 32), A1 ? 2u : 1u);
    NCF_LAUNCH("paper_eval_kernel", st,
               paper_eval_kernel<<<grid, kEvalWarps * 32, 0, st>>>(A, A1, Mh, phi, K, c, c1));
}

void paper_finish(const double *craw, const double *bsrt, int64_t K1, const int64_t *perm, int64_t pos0,
                  const double *w, int nw, int o0, bool acf, const double *craw_x, const double *craw_y,
                  int64_t nsym, const double *bx0, const double *by0, double *tmp, double *c_out,
                  double *b_out, cudaStream_t st) {
    NCF_LAUNCH("paper_finish_kernel", st,
               paper_finish_kernel<<<1, 1024, 0, st>>>(craw, bsrt, K1, perm, pos0, w, nw, o0, acf ? 1 : 0, craw_x,
                                                       craw_y, nsym, bx0, by0, tmp, c_out, b_out));
}

}  // namespace ncf
