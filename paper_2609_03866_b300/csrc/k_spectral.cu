// k_spectral.cu -- the Wiener-Khinchin (NUFFT) path for the Gaussian kernel
// (Sec. 2.6; Algorithms 2 and 4 with the smoothing step replaced by the
// kernel's Fourier transform, see below).
//
// For lag tau and the Gaussian b, Poisson summation on a period L gives
//   N(tau) = (1/L) sum_m bhat(m/L) conj(X_m) Y_m exp(-2 pi i m tau / L),
//   X_m = sum_i x_i exp(+2 pi i m (t_i - t_c) / L)            (Eq. nufft_type1)
// exactly as long as every pair separation s_j - t_i - tau stays more than a
// few kernel widths away from +-L (the padded period of Algorithm 1, with a
// kernel-width margin added).  bhat(f) = exp(-2 pi^2 h^2 f^2) decays fast, so
// |m| <= m_max modes suffice.  The effective pair count B(tau) is the same sum
// with unit weights.  Both series' values x and unit weights ride one complex
// spreading pass (strength x_std + i); Hermitian unpacking separates them.
//
// Steps (all on the caller's stream):
//   spread   ES-kernel type-1 spreading onto an oversampled periodic grid of
//            n_f cells, SMEM tile per chunk of sorted points, one global add
//            per touched cell (sorted times make the chunks bin-sorted);
//   fft      Stockham radix-8/4/2 passes over the grids of all series;
//   spectrum Hermitian unpack, deconvolution by the ES kernel's transform,
//            cross (or power) spectrum times bhat: one row of modes per series;
//   contract rows of modes times the shared table of cos/sin(2 pi m tau_k / L)
//            (a dense [B x M] x [M x K] product), split over mode chunks with
//            FP64 accumulation of the partial sums;
//   finish   c = N / max(B, 1e-16), optional lag-0 (Pearson) scaling.
//
// The ES ("exponential of semicircle") kernel phi(z) = exp(beta (sqrt(1 - z^2) - 1))
// and its Fourier transform by Gauss-Legendre quadrature follow Barnett,
// Magland & af Klinteberg (SIAM J. Sci. Comput. 2019), the NUFFT the paper
// uses (Sec. 2.5).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "fft.cuh"
#include "spectral.cuh"

namespace ncf {

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

size_t al(size_t b) { return (b + 255) & ~size_t(255); }

// Gauss-Legendre nodes and weights on [-1, 1] by Newton's iteration on P_n.
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// ---------------------------------------------------------------------------
// tables
// ---------------------------------------------------------------------------

// Per-mode weight of the spectra, folding the deconvolution (1 / phihat_m^2),
// the Gaussian transform bhat(m/L), the 1/L of the Fourier series and the
// factor 2 of the +-m pair:  wgt_m = fac_m bhat(m/L) / (L phihat_m^2).
// phihat_m = (w/2) int_{-1}^{1} phi(z) cos(pi m w z / n_f) dz by quadrature.
__global__ void mode_weight_kernel(const double *__restrict__ gx, const double *__restrict__ gphi,
                                   int nq, int64_t M, int64_t Mp, int W, int nf, double L, double h,
                                   double *__restrict__ wgt64, float *__restrict__ wgt32) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= Mp) return;
    double out = 0.0;
    if (m < M) {
        const double a = (double)m * W / nf;  // cos(pi a z)
        double s = 0.0;
        for (int q = 0; q < nq; ++q) s += gphi[q] * cospi(a * gx[q]);
        const double ph = 0.5 * W * s;
        const double f = (double)m / L;
        const double bhat = exp(-2.0 * kPi * kPi * h * h * f * f);
        out = (m == 0 ? 1.0 : 2.0) * bhat / (L * ph * ph);
    }
    if (wgt64) wgt64[m] = out;
    if (wgt32) wgt32[m] = (float)out;
}

// tw[q] = exp(+2 pi i q / n), q in [0, n)
template <typename V>
__global__ void twiddle_kernel(V *__restrict__ tw, int n) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    double s, c;
    sincospi(2.0 * (double)q / n, &s, &c);
    tw[q].x = c;
    tw[q].y = s;
}

// Lag table E[m][k] = cos(2 pi m tau_k / L) for m < Mp, and for a CCF
// E[Mp + m][k] = sin(2 pi m tau_k / L).  The phase m tau_k / L mod 1 is
// formed exactly in 64-bit fixed point: Phi_k = frac(tau_k / L) 2^64, and
// m Phi_k mod 2^64 is an exact integer product.
template <typename R>
__global__ void lag_table_kernel(const unsigned long long *__restrict__ Phi, int64_t Mp, int64_t Kp,
                                 int64_t K1, bool with_sin, R *__restrict__ E) {
    const int64_t k = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    const int64_t m = blockIdx.x;
    if (k >= Kp) return;
    double c = 0.0, s = 0.0;
    if (k < K1) {
        const unsigned long long ph = (unsigned long long)m * Phi[k];
        const double p = (double)(ph >> 11) * 0x1.0p-53;  // [0, 1)
        sincospi(2.0 * p, &s, &c);
    }
    E[m * Kp + k] = (R)c;
    if (with_sin) E[(Mp + m) * Kp + k] = (R)s;
}

// ---------------------------------------------------------------------------
// spreading (global-memory grids)
// ---------------------------------------------------------------------------

__device__ __forceinline__ int64_t find_series(const int64_t *chunk_base, int64_t B, int64_t g) {
    int64_t lo = 0, hi = B;
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (chunk_base[mid] <= g) lo = mid; else hi = mid;
    }
    return lo;
}

template <typename R> __device__ __forceinline__ R es_kernel(R z, R beta);
template <> __device__ __forceinline__ float es_kernel<float>(float z, float beta) {
    const float u = fmaxf(0.0f, fmaf(-z, z, 1.0f));
    return __expf(beta * (sqrtf(u) - 1.0f));
}
template <> __device__ __forceinline__ double es_kernel<double>(double z, double beta) {
    const double u = fmax(0.0, fma(-z, z, 1.0));
    return exp(beta * (sqrt(u) - 1.0));
}

template <typename V> __device__ __forceinline__ void atomic_add_v(V *p, decltype(V{}.x) a, decltype(V{}.x) b) {
    atomicAdd(&p->x, a);
    atomicAdd(&p->y, b);
}

constexpr int kSpreadThreads = 256;

// One CTA per prep chunk (kPrepChunk consecutive points of one series).
// Grid coordinate of a point: g = (t - t_c) n_f / L; the kernel touches the W
// cells l0 .. l0+W-1 with l0 = ceil(g - W/2) (taken mod n_f).  gs = g - W/2 +
// n_f is formed with one FP64 FMA (positive, so ceil is a plain conversion).
template <typename R, int W, int TILE>
__global__ void __launch_bounds__(kSpreadThreads)
spread_kernel(const double *__restrict__ t, const double *__restrict__ x,
              const int64_t *__restrict__ offs, const int64_t *__restrict__ chunk_base, int64_t B,
              const SeriesStats *__restrict__ st, const double *__restrict__ tc, double a_scale,
              int nf, R beta, typename CT<R>::V *__restrict__ grids) {
    using V = typename CT<R>::V;
    __shared__ V tile[TILE];
    const int64_t g = blockIdx.x;
    const int64_t b = find_series(chunk_base, B, g);
    const int64_t a0 = offs[b], a1 = offs[b + 1];
    const int64_t start = a0 + (g - chunk_base[b]) * (int64_t)kPrepChunk;
    const int64_t end = min(start + (int64_t)kPrepChunk, a1);
    const double c_off = -tc[b] * a_scale - 0.5 * W + nf;
    const double mean = st[b].mean, inv = st[b].inv_std;
    V *grid = grids + b * (int64_t)nf;
    const int mask = nf - 1;
    const int l_first = (int)ceil(fma(t[start], a_scale, c_off));
    const int l_last = (int)ceil(fma(t[end - 1], a_scale, c_off)) + W - 1;
    const int span = l_last - l_first + 1;
    const bool use_tile = span <= TILE;
    if (use_tile) {
        for (int i = threadIdx.x; i < span; i += blockDim.x) { tile[i].x = 0; tile[i].y = 0; }
        __syncthreads();
    }
    const R half = (R)(0.5 * W), inv_half = (R)(2.0 / W);
    for (int64_t i = start + threadIdx.x; i < end; i += blockDim.x) {
        const double gs = fma(t[i], a_scale, c_off);
        const int l0 = (int)ceil(gs);
        const R f0 = (R)((double)l0 - gs);          // in [0, 1)
        const R xs = (R)((x[i] - mean) * inv);
#pragma unroll
        for (int k = 0; k < W; ++k) {
            const R z = (f0 + (R)k - half) * inv_half;
            const R phi = es_kernel<R>(z, beta);
            if (use_tile) {
                atomicAdd(&tile[l0 + k - l_first].x, phi * xs);
                atomicAdd(&tile[l0 + k - l_first].y, phi);
            } else {
                atomic_add_v(&grid[(l0 + k) & mask], phi * xs, phi);
            }
        }
    }
    if (use_tile) {
        __syncthreads();
        for (int i = threadIdx.x; i < span; i += blockDim.x) {
            const V v = tile[i];
            if (v.x != 0 || v.y != 0) atomic_add_v(&grid[(l_first + i) & mask], v.x, v.y);
        }
    }
}

// ---------------------------------------------------------------------------
// FFT: one Stockham pass over the grids of all series (out of place)
// ---------------------------------------------------------------------------
template <typename V, int RAD>
__global__ void fft_pass_kernel(const V *__restrict__ in, V *__restrict__ out, int lg, int Ns,
                                const V *__restrict__ tw, int64_t B) {
    const int n = 1 << lg;
    const int per = n / RAD;
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= B * per) return;
    const int64_t b = item / per;
    const int j = (int)(item - b * per);
    const V *src = in + b * n;
    V *dst = out + b * n;
    const int k = j % Ns;
    const int stride = n / (Ns * RAD);
    V v[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[r] = src[j + r * per];
#pragma unroll
    for (int r = 1; r < RAD; ++r) v[r] = cmul(v[r], tw[(r * k) * stride]);
    dft<RAD>(v);
    const int base = (j / Ns) * Ns * RAD + k;
#pragma unroll
    for (int r = 0; r < RAD; ++r) dst[base + r * Ns] = v[r];
}

// ---------------------------------------------------------------------------
// spectra
// ---------------------------------------------------------------------------

// Hermitian unpack of G = FFT(spread of x_std + i): X_m and W_m (unit weights),
// without the deconvolution (folded into wgt).
template <typename V>
__device__ __forceinline__ void unpack(const V *__restrict__ G, int nf, int64_t m, V &X, V &Wt) {
    const V a = G[m];
    const V c = G[(nf - m) & (nf - 1)];
    X.x = (a.x + c.x) * 0.5f; X.y = (a.y - c.y) * 0.5f;
    Wt.x = (a.y + c.y) * 0.5f; Wt.y = (c.x - a.x) * 0.5f;
}

// A rows: ACF  num[b][m] = wgt |X|^2,     den[b][m] = wgt |W|^2
//         CCF  num[b][m] = wgt Re(conj(X) Y), num[b][Mp + m] = wgt Im(conj(X) Y),
//              den likewise with the unit-weight spectra.
// With lag0 and a CCF, also the per-series lag-0 sums of both power spectra.
template <typename R>
__device__ __forceinline__ void spectrum_one(const typename CT<R>::V *__restrict__ Gx,
                                             const typename CT<R>::V *__restrict__ Gy, int nf,
                                             int64_t M, int64_t Mp, int64_t b, int64_t m,
                                             const R *__restrict__ wgt, R *__restrict__ Anum,
                                             R *__restrict__ Aden, double *__restrict__ lag0) {
    using V = typename CT<R>::V;
    const bool ccf = Gy != nullptr;
    const int64_t row = ccf ? 2 * Mp : Mp;
    R *an = Anum + b * row, *ad = Aden + b * row;
    if (m >= M) {
        an[m] = 0; ad[m] = 0;
        if (ccf) { an[Mp + m] = 0; ad[Mp + m] = 0; }
        return;
    }
    const R wm = wgt[m];
    V X, Wx;
    unpack(Gx + b * (int64_t)nf, nf, m, X, Wx);
    if (!ccf) {
        an[m] = wm * (X.x * X.x + X.y * X.y);
        ad[m] = wm * (Wx.x * Wx.x + Wx.y * Wx.y);
        return;
    }
    V Y, Wy;
    unpack(Gy + b * (int64_t)nf, nf, m, Y, Wy);
    an[m] = wm * (X.x * Y.x + X.y * Y.y);
    an[Mp + m] = wm * (X.x * Y.y - X.y * Y.x);
    ad[m] = wm * (Wx.x * Wy.x + Wx.y * Wy.y);
    ad[Mp + m] = wm * (Wx.x * Wy.y - Wx.y * Wy.x);
    if (lag0) {
        atomicAdd(lag0 + 4 * b + 0, (double)(wm * (X.x * X.x + X.y * X.y)));
        atomicAdd(lag0 + 4 * b + 1, (double)(wm * (Wx.x * Wx.x + Wx.y * Wx.y)));
        atomicAdd(lag0 + 4 * b + 2, (double)(wm * (Y.x * Y.x + Y.y * Y.y)));
        atomicAdd(lag0 + 4 * b + 3, (double)(wm * (Wy.x * Wy.x + Wy.y * Wy.y)));
    }
}

template <typename R>
__global__ void spectrum_kernel(const typename CT<R>::V *__restrict__ Gx,
                                const typename CT<R>::V *__restrict__ Gy, int nf, int64_t M,
                                int64_t Mp, int64_t B, const R *__restrict__ wgt,
                                R *__restrict__ Anum, R *__restrict__ Aden, double *__restrict__ lag0) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= Mp) return;
    for (int64_t b = blockIdx.y; b < B; b += gridDim.y)
        spectrum_one<R>(Gx, Gy, nf, M, Mp, b, m, wgt, Anum, Aden, lag0);
}


// ---------------------------------------------------------------------------
// contraction: acc[c][b][k] += sum_{m in chunk} A_c[b][m] E[m][k], c = num, den
// ---------------------------------------------------------------------------
constexpr int kBM = 32, kBN = 64, kBK = 32, kChunk = 512;

template <typename R>
__global__ void __launch_bounds__(256)
contract_kernel(const R *__restrict__ Anum, const R *__restrict__ Aden, const R *__restrict__ E,
                int64_t B, int64_t M2, int64_t Kp, double *__restrict__ acc_num,
                double *__restrict__ acc_den) {
    __shared__ R sA[2][kBK][kBM + 1];
    __shared__ R sE[kBK][kBN];
    const int tid = threadIdx.x;
    const int tb = tid / 16, tk = tid % 16;  // 16 x 16 threads, each 2 (b) x 4 (k)
    const int64_t b0 = (int64_t)blockIdx.y * kBM, k0 = (int64_t)blockIdx.x * kBN;
    const int64_t m_lo = (int64_t)blockIdx.z * kChunk, m_hi = min(m_lo + kChunk, M2);
    R an[2][4] = {}, ad[2][4] = {};
    for (int64_t m0 = m_lo; m0 < m_hi; m0 += kBK) {
        for (int i = tid; i < kBK * kBM; i += 256) {
            const int mm = i % kBK, bb = i / kBK;
            const int64_t gb = b0 + bb, gm = m0 + mm;
            const bool ok = gb < B && gm < m_hi;
            sA[0][mm][bb] = ok ? Anum[gb * M2 + gm] : (R)0;
            sA[1][mm][bb] = ok ? Aden[gb * M2 + gm] : (R)0;
        }
        for (int i = tid; i < kBK * kBN; i += 256) {
            const int kk = i % kBN, mm = i / kBN;
            const int64_t gk = k0 + kk, gm = m0 + mm;
            sE[mm][kk] = (gk < Kp && gm < m_hi) ? E[gm * Kp + gk] : (R)0;
        }
        __syncthreads();
#pragma unroll 8
        for (int mm = 0; mm < kBK; ++mm) {
            R e[4], xn[2], xd[2];
#pragma unroll
            for (int q = 0; q < 4; ++q) e[q] = sE[mm][tk + 16 * q];
#pragma unroll
            for (int p = 0; p < 2; ++p) { xn[p] = sA[0][mm][tb + 16 * p]; xd[p] = sA[1][mm][tb + 16 * p]; }
#pragma unroll
            for (int p = 0; p < 2; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    an[p][q] = fma(xn[p], e[q], an[p][q]);
                    ad[p][q] = fma(xd[p], e[q], ad[p][q]);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t gb = b0 + tb + 16 * p, gk = k0 + tk + 16 * q;
            if (gb < B && gk < Kp) {
                atomicAdd(acc_num + gb * Kp + gk, (double)an[p][q]);
                atomicAdd(acc_den + gb * Kp + gk, (double)ad[p][q]);
            }
        }
}

__global__ void finish_spectral_kernel(const double *__restrict__ acc_num,
                                       const double *__restrict__ acc_den, int64_t B, int64_t K,
                                       int64_t Kp, int lag0_mode, const double *__restrict__ lag0,
                                       double *__restrict__ c, double *__restrict__ bo,
                                       int64_t *__restrict__ cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * K) return;
    const int64_t b = i / K, k = i - b * K;
    const double N = acc_num[b * Kp + k], D = acc_den[b * Kp + k];
    double ci = N / fmax(D, 1e-16);
    if (lag0_mode == 1) {          // ACF: divide by c(0) from the appended zero lag
        ci /= acc_num[b * Kp + K] / fmax(acc_den[b * Kp + K], 1e-16);
    } else if (lag0_mode == 2) {   // CCF: divide by sqrt(ACF_x(0) ACF_y(0))
        const double sx = lag0[4 * b] / fmax(lag0[4 * b + 1], 1e-16);
        const double sy = lag0[4 * b + 2] / fmax(lag0[4 * b + 3], 1e-16);
        ci /= sqrt(sx * sy);
    }
    c[i] = ci;
    if (bo) bo[i] = D;
    if (cnt) cnt[i] = 0;
}

template <typename T>
T *take(char *base, size_t &used, size_t count) {
    T *p = reinterpret_cast<T *>(base + used);
    used += al(count * sizeof(T));
    return p;
}

struct Plan {
    double L = 0, beta = 0;
    int64_t M = 0, Mp = 0, K1 = 0, Kp = 0, M2 = 0;
    int nf = 0, lg = 0, W = 8, nq = 64;
};

Plan make_plan(const SpectralArgs &a, double max_span) {
    Plan p;
    const double tol = a.tol;
    const double R_alias = std::sqrt(2.0 * std::log(1.0 / (tol * 1e-2)));
    p.L = max_span + a.max_tau + R_alias * a.h;
    const double delta = tol * 1e-3;
    const double mscale = std::sqrt(std::log(1.0 / delta) / (2.0 * kPi * kPi));
    p.M = (int64_t)std::ceil(p.L * mscale / a.h) + 1;
    p.Mp = (p.M + 31) / 32 * 32;
    p.W = a.fp32 ? 8 : 16;
    p.beta = 2.30 * p.W;
    p.nq = a.fp32 ? 64 : 128;
    int64_t need = 2 * 2 * p.M + p.W;  // oversampling >= 2
    p.lg = 1;
    while ((int64_t(1) << p.lg) < need) ++p.lg;
    p.nf = 1 << p.lg;
    p.K1 = a.K + 1;                    // + an internal zero lag (lag-0 scale of the ACF)
    p.Kp = (p.K1 + 3) / 4 * 4;
    p.M2 = a.acf ? p.Mp : 2 * p.Mp;
    return p;
}

template <typename R>
ncf_status run_typed(const SpectralArgs &a, const Plan &p, char *ws, const double *h_tc,
                     const unsigned long long *h_phi, const std::vector<double> &gx,
                     const std::vector<double> &gphi, char *pinned, cudaStream_t st, std::string *msg) {
    using V = typename CT<R>::V;
    const int64_t B = a.B;
    const bool ccf = !a.acf;
    size_t used = 0;
    V *grid_x = take<V>(ws, used, B * (size_t)p.nf);
    V *grid_y = ccf ? take<V>(ws, used, B * (size_t)p.nf) : nullptr;
    V *scratch = take<V>(ws, used, B * (size_t)p.nf);
    V *tw = take<V>(ws, used, p.nf);
    double *wgt64 = take<double>(ws, used, p.Mp);
    R *wgt = take<R>(ws, used, p.Mp);
    R *Anum = take<R>(ws, used, B * p.M2);
    R *Aden = take<R>(ws, used, B * p.M2);
    R *E = take<R>(ws, used, p.M2 * p.Kp);
    double *acc_num = take<double>(ws, used, B * p.Kp);
    double *acc_den = take<double>(ws, used, B * p.Kp);
    double *lag0 = take<double>(ws, used, 4 * B);
    double *d_tc = take<double>(ws, used, B);
    unsigned long long *d_phi = take<unsigned long long>(ws, used, p.Kp);
    double *d_gx = take<double>(ws, used, p.nq);
    double *d_gphi = take<double>(ws, used, p.nq);

    // small host tables -> device (pinned staging)
    size_t off = 0;
    auto up = [&](void *dst, const void *src, size_t bytes) {
        std::memcpy(pinned + off, src, bytes);
        cudaMemcpyAsync(dst, pinned + off, bytes, cudaMemcpyHostToDevice, st);
        off += al(bytes);
    };
    up(d_tc, h_tc, B * 8);
    up(d_phi, h_phi, p.Kp * 8);
    up(d_gx, gx.data(), p.nq * 8);
    up(d_gphi, gphi.data(), p.nq * 8);

    NCF_LAUNCH("mode_weight_kernel", st,
    mode_weight_kernel<<<(unsigned)((p.Mp + 255) / 256), 256, 0, st>>>(
        d_gx, d_gphi, p.nq, p.M, p.Mp, p.W, p.nf, p.L, a.h, wgt64,
        std::is_same<R, float>::value ? reinterpret_cast<float *>(wgt) : nullptr));
    if (std::is_same<R, double>::value)
        cudaMemcpyAsync(wgt, wgt64, p.Mp * 8, cudaMemcpyDeviceToDevice, st);
    NCF_LAUNCH("twiddle_kernel", st,
    twiddle_kernel<V><<<(p.nf + 255) / 256, 256, 0, st>>>(tw, p.nf));
    {
        dim3 grid((unsigned)p.Mp, (unsigned)((p.Kp + 127) / 128));
        NCF_LAUNCH("lag_table_kernel", st,
        lag_table_kernel<R><<<grid, 128, 0, st>>>(d_phi, p.Mp, p.Kp, p.K1, ccf, E));
    }

    // spreading
    const double a_scale = (double)p.nf / p.L;
    auto spread = [&](const SpecSide &sd, V *grid, const int64_t *chunk_base, int64_t n_chunks) {
        cudaMemsetAsync(grid, 0, B * (size_t)p.nf * sizeof(V), st);
        constexpr int TILE = sizeof(R) == 4 ? 4096 : 2048;
        if (p.W == 8)
            NCF_LAUNCH("spread_kernel", st,
                       spread_kernel<R, 8, TILE><<<(unsigned)n_chunks, kSpreadThreads, 0, st>>>(
                           sd.t, sd.v, sd.d_offs, chunk_base, B, sd.d_stats, d_tc, a_scale, p.nf,
                           (R)p.beta, grid));
        else
            NCF_LAUNCH("spread_kernel", st,
                       spread_kernel<R, 16, TILE><<<(unsigned)n_chunks, kSpreadThreads, 0, st>>>(
                           sd.t, sd.v, sd.d_offs, chunk_base, B, sd.d_stats, d_tc, a_scale, p.nf,
                           (R)p.beta, grid));
    };
    spread(a.x, grid_x, a.x.d_chunk_base, a.x.n_chunks);
    if (ccf) spread(a.y, grid_y, a.y.d_chunk_base, a.y.n_chunks);

    // FFT passes (ping-pong with scratch); result returned in *res
    const RadixPlan rp = radix_plan(p.lg);
    auto fft = [&](V *grid) -> V * {
        V *in = grid, *out = scratch;
        int Ns = 1;
        for (int q = 0; q < rp.n_pass; ++q) {
            const int rad = rp.radix[q];
            const int64_t items = B * (int64_t)(p.nf / rad);
            const unsigned blocks = (unsigned)((items + 255) / 256);
            if (rad == 8)
                NCF_LAUNCH("fft_pass_kernel", st,
                           fft_pass_kernel<V, 8><<<blocks, 256, 0, st>>>(in, out, p.lg, Ns, tw, B));
            else if (rad == 4)
                NCF_LAUNCH("fft_pass_kernel", st,
                           fft_pass_kernel<V, 4><<<blocks, 256, 0, st>>>(in, out, p.lg, Ns, tw, B));
            else
                NCF_LAUNCH("fft_pass_kernel", st,
                           fft_pass_kernel<V, 2><<<blocks, 256, 0, st>>>(in, out, p.lg, Ns, tw, B));
            Ns *= rad;
            std::swap(in, out);
        }
        return in;
    };
    V *Gx = fft(grid_x);
    if (Gx == scratch && ccf) {
        // keep x's transform out of the scratch buffer before y's passes
        cudaMemcpyAsync(grid_x, scratch, B * (size_t)p.nf * sizeof(V), cudaMemcpyDeviceToDevice, st);
        Gx = grid_x;
    }
    V *Gy = ccf ? fft(grid_y) : nullptr;

    const bool lag0_ccf = a.lag0 && ccf;
    if (lag0_ccf) cudaMemsetAsync(lag0, 0, 4 * B * 8, st);
    {
        dim3 grid((unsigned)((p.Mp + 255) / 256), (unsigned)std::min<int64_t>(B, 65535));
        NCF_LAUNCH("spectrum_kernel", st,
        spectrum_kernel<R><<<grid, 256, 0, st>>>(Gx, Gy, p.nf, p.M, p.Mp, B, wgt, Anum, Aden,
                                                 lag0_ccf ? lag0 : nullptr));
    }
    cudaMemsetAsync(acc_num, 0, B * p.Kp * 8, st);
    cudaMemsetAsync(acc_den, 0, B * p.Kp * 8, st);
    {
        dim3 grid((unsigned)((p.Kp + kBN - 1) / kBN), (unsigned)((B + kBM - 1) / kBM),
                  (unsigned)((p.M2 + kChunk - 1) / kChunk));
        NCF_LAUNCH("contract_kernel", st,
        contract_kernel<R><<<grid, 256, 0, st>>>(Anum, Aden, E, B, p.M2, p.Kp, acc_num, acc_den));
    }
    {
        const int mode = a.lag0 ? (ccf ? 2 : 1) : 0;
        NCF_LAUNCH("finish_spectral_kernel", st,
        finish_spectral_kernel<<<(unsigned)((B * a.K + 255) / 256), 256, 0, st>>>(
            acc_num, acc_den, B, a.K, p.Kp, mode, lag0, a.c_out, a.b_out, a.count_out));
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        *msg = std::string("spectral path launch failed: ") + cudaGetErrorString(e);
        return NCF_ECUDA;
    }
    return NCF_OK;
}

template <typename R>
size_t workspace_bytes(const Plan &p, int64_t B, bool ccf) {
    using V = typename CT<R>::V;
    size_t s = 0;
    s += al(B * (size_t)p.nf * sizeof(V)) * (ccf ? 3 : 2);
    s += al(p.nf * sizeof(V));
    s += al(p.Mp * 8) + al(p.Mp * sizeof(R));
    s += al(B * p.M2 * sizeof(R)) * 2 + al(p.M2 * p.Kp * sizeof(R));
    s += al(B * p.Kp * 8) * 2 + al(4 * B * 8) + al(B * 8) + al(p.Kp * 8) + al(p.nq * 8) * 2;
    return s + 1024;
}

}  // namespace

ncf_status run_spectral(const SpectralArgs &a, char **ws, size_t *ws_cap, char **pinned,
                        size_t *pinned_cap, cudaStream_t st, std::string *msg,
                        SpectralGeometry *geom) {
    const int64_t B = a.B;
    const bool ccf = !a.acf;
    // per-series centre t_c and the common period L (Algorithm 1 with an
    // alias margin: L = max span + max|tau| + R h)
    std::vector<double> tc(B);
    double max_span = 0.0;
    for (int64_t b = 0; b < B; ++b) {
        double lo = a.x.h_stats[b].t_first, hi = a.x.h_stats[b].t_last;
        if (ccf) {
            lo = std::min(lo, a.y.h_stats[b].t_first);
            hi = std::max(hi, a.y.h_stats[b].t_last);
        }
        tc[b] = lo + 0.5 * (hi - lo);
        max_span = std::max(max_span, hi - lo);
    }
    const Plan p = make_plan(a, max_span);
    if (geom) *geom = SpectralGeometry{p.L, p.M, p.nf, p.W};
    if (p.lg > 28) {
        *msg = "spectral grid would exceed 2^28 cells (span / h too large); use the windowed path";
        return NCF_EUNSUPPORTED;
    }
    // lag phases in 64-bit fixed point; the appended lag K is zero
    std::vector<unsigned long long> phi(p.Kp, 0ull);
    for (int64_t k = 0; k < a.K; ++k) {
        double f = a.h_lags[k] / p.L;
        f -= std::floor(f);
        phi[k] = (unsigned long long)std::ldexp(f, 64 - 11) << 11;
    }
    std::vector<double> gx, gw, gphi;
    gauss_legendre(p.nq, gx, gw);
    gphi.resize(p.nq);
    for (int q = 0; q < p.nq; ++q)
        gphi[q] = gw[q] * std::exp(p.beta * (std::sqrt(std::max(0.0, 1.0 - gx[q] * gx[q])) - 1.0));

    const size_t need = a.fp32 ? workspace_bytes<float>(p, B, ccf) : workspace_bytes<double>(p, B, ccf);
    if (need > *ws_cap) {
        if (*ws) {
            cudaStreamSynchronize(st);
            cudaFree(*ws);
            *ws = nullptr;
            *ws_cap = 0;
        }
        if (cudaMalloc(ws, need) != cudaSuccess) {
            cudaGetLastError();
            *ws = nullptr;
            *msg = "cudaMalloc of the spectral workspace failed";
            return NCF_ENOMEM;
        }
        *ws_cap = need;
    }
    const size_t pin_need = al(B * 8) + al(p.Kp * 8) + 2 * al(p.nq * 8);
    if (pin_need > *pinned_cap) {
        cudaStreamSynchronize(st);
        if (*pinned) cudaFreeHost(*pinned);
        *pinned = nullptr;
        *pinned_cap = 0;
        if (cudaHostAlloc(pinned, pin_need, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            *msg = "cudaHostAlloc of the staging buffer failed";
            return NCF_ENOMEM;
        }
        *pinned_cap = pin_need;
    }
    if (a.fp32) return run_typed<float>(a, p, *ws, tc.data(), phi.data(), gx, gphi, *pinned, st, msg);
    return run_typed<double>(a, p, *ws, tc.data(), phi.data(), gx, gphi, *pinned, st, msg);
}

}  // namespace ncf
