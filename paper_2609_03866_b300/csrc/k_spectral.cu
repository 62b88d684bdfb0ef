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

// Per-tap polynomial form of the ES kernel for spreading: tap k of a point at
// fractional offset f0 in [0, 1) has weight phi((f0 + k - W/2) / (W/2)); on that
// interval phi is interpolated at D+1 Chebyshev nodes in u = 2 f0 - 1 and the
// interpolant is rewritten in powers of u (coefficient d of tap k at
// c[k * (D+1) + d]), so the kernel evaluates it with D fused multiply-adds and
// no special-function instructions.  Max error: 8e-8 (W = 8, D = 8, FP32) and
// 4e-15 (W = 16, D = 14, FP64) of the peak value 1.  The Chebyshev nodes are
// symmetric and phi is even, so tap W-1-k's interpolant is tap k's at -u; the
// kernel uses the first W/2 taps' coefficients only.
std::vector<double> es_poly(int W, double beta, int D) {
    std::vector<double> out((size_t)W * (D + 1));
    const int n = D + 1;
    std::vector<double> node(n), val(n), cheb(n), pw(n), tk(n), tkm1(n), tkp1(n);
    for (int i = 0; i < n; ++i) node[i] = std::cos(kPi * (i + 0.5) / n);
    for (int k = 0; k < W; ++k) {
        for (int i = 0; i < n; ++i) {
            const double f = 0.5 * (node[i] + 1.0);
            const double z = (f + k - 0.5 * W) / (0.5 * W);
            const double u = std::max(0.0, 1.0 - z * z);
            val[i] = std::exp(beta * (std::sqrt(u) - 1.0));
        }
        // Chebyshev coefficients of the interpolant
        for (int j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int i = 0; i < n; ++i) acc += val[i] * std::cos(kPi * j * (i + 0.5) / n);
            cheb[j] = acc * (j == 0 ? 1.0 : 2.0) / n;
        }
        // sum_j cheb_j T_j(u) in powers of u, with T_{j+1} = 2u T_j - T_{j-1}
        std::fill(pw.begin(), pw.end(), 0.0);
        std::fill(tkm1.begin(), tkm1.end(), 0.0);
        std::fill(tk.begin(), tk.end(), 0.0);
        tkm1[0] = 1.0;            // T_0
        if (n > 1) tk[1] = 1.0;   // T_1
        pw[0] += cheb[0];
        for (int j = 1; j < n; ++j) {
            for (int d = 0; d < n; ++d) pw[d] += cheb[j] * tk[d];
            std::fill(tkp1.begin(), tkp1.end(), 0.0);
            for (int d = 0; d + 1 < n; ++d) tkp1[d + 1] += 2.0 * tk[d];
            for (int d = 0; d < n; ++d) tkp1[d] -= tkm1[d];
            tkm1 = tk;
            tk = tkp1;
        }
        for (int d = 0; d < n; ++d) out[(size_t)k * n + d] = pw[d];
    }
    return out;
}

// Largest sum over the W taps of one point, max over u in [0, 1] of
// sum_k P_k(2u - 1) (sampled finely, with a margin far above the sampling's
// error for these smooth, bounded interpolants): a bound for fixed-point sums.
double es_tap_sum(const std::vector<double> &poly, int W, int D) {
    double best = 0.0;
    for (int i = 0; i <= 4096; ++i) {
        const double u = 2.0 * i / 4096.0 - 1.0;
        double s = 0.0;
        for (int k = 0; k < W; ++k) {
            double v = 0.0;
            for (int d = D; d >= 0; --d) v = v * u + poly[(size_t)k * (D + 1) + d];
            s += std::fabs(v);
        }
        best = std::max(best, s);
    }
    return best * 1.01 + 1e-3;
}

template <typename R, int W, int D> struct EsPoly { R c[W * (D + 1)]; };
template <int W> struct PolyDeg;
template <> struct PolyDeg<8> { static constexpr int D = 8; };
template <> struct PolyDeg<16> { static constexpr int D = 14; };

// ---------------------------------------------------------------------------
// tables
// ---------------------------------------------------------------------------

// Per-mode weight of the spectra, folding the deconvolution (1 / phihat_m^2),
// the kernel's transform bhat(m/L), the 1/L of the Fourier series and the
// factor 2 of the +-m pair:  wgt_m = fac_m bhat(m/L) / (L phihat_m^2).
// Gaussian (unit mass): bhat(f) = exp(-2 pi^2 h^2 f^2).  Rectangle (a pair
// counts 1 inside |d| <= h): bhat(f) = sin(2 pi f h) / (pi f), 2h at f = 0; its
// 1/f tail makes the truncated sum an approximation (the spectral-sinc variant).
// phihat_m = (w/2) int_{-1}^{1} phi(z) cos(pi m w z / n_f) dz by quadrature.
__global__ void mode_weight_kernel(const double *__restrict__ gx, const double *__restrict__ gphi,
                                   int nq, int64_t M, int64_t Mp, int W, int nf, double L, double h, int rect,
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
        const double bhat = rect ? (m == 0 ? 2.0 * h : sinpi(2.0 * f * h) / (kPi * f))
                                 : exp(-2.0 * kPi * kPi * h * h * f * f);
        out = (m == 0 ? 1.0 : 2.0) * bhat / (L * ph * ph);
    }
    if (wgt64) wgt64[m] = out;
    if (wgt32) wgt32[m] = (float)out;
}

// tw[q] = exp(+2 pi i q / n), q in [0, n): each thread starts a run of kTwRun
// entries from sincospi and steps along it by the rotation exp(2 pi i / n)
// (error below 3e-15 after the run's 7 steps).
constexpr int kTwRun = 8;
template <typename V>
__global__ void twiddle_kernel(V *__restrict__ tw, int n) {
    const int q0 = (blockIdx.x * blockDim.x + threadIdx.x) * kTwRun;
    if (q0 >= n) return;
    double s, c, rs, rc;
    sincospi(2.0 * (double)q0 / n, &s, &c);
    sincospi(2.0 / n, &rs, &rc);
#pragma unroll
    for (int j = 0; j < kTwRun; ++j) {
        if (q0 + j >= n) break;
        tw[q0 + j].x = c;
        tw[q0 + j].y = s;
        const double c2 = fma(c, rc, -s * rs);
        s = fma(s, rc, c * rs);
        c = c2;
    }
}
inline unsigned twiddle_blocks(int n) { return (unsigned)((n / kTwRun + 255) / 256 + 1); }

// Lag table E[m][k] = cos(2 pi m tau_k / L) for m < Mp, and for a CCF
// E[Mp + m][k] = sin(2 pi m tau_k / L).  The phase m tau_k / L mod 1 is
// formed exactly in 64-bit fixed point: Phi_k = frac(tau_k / L) 2^64, and
// m Phi_k mod 2^64 is an exact integer product.
template <typename R>
__device__ __forceinline__ void lag_sincos(unsigned long long ph, R &c, R &s);
// FP64 table: sin and cos of 2 pi ph 2^-64 from the 53 leading bits
template <>
__device__ __forceinline__ void lag_sincos<double>(unsigned long long ph, double &c, double &s) {
    const double p = (double)(ph >> 11) * 0x1.0p-53;  // [0, 1)
    sincospi(2.0 * p, &s, &c);
}
// FP32 table, FP32 arithmetic only: the phase splits exactly into a = the leading
// 24 bits and b < 2^-24 (the next 24 bits); sin and cos of 2 pi a by the FP32
// function, then one first-order step to a + b (the dropped term is below
// (2 pi 2^-24)^2 / 2 < 1e-13).  Within a few FP32 ulps, which is what the table is
// stored in (an FP64 sincospi per entry cost 13 ms for 2.8e8 entries).
template <>
__device__ __forceinline__ void lag_sincos<float>(unsigned long long ph, float &c, float &s) {
    const float a = (float)(unsigned)(ph >> 40) * 0x1.0p-24f;                          // exact
    const float b = (float)(unsigned)((ph >> 16) & 0xFFFFFFu) * 0x1.0p-48f;            // exact, < 2^-24
    float sa, ca;
    sincospif(2.0f * a, &sa, &ca);
    const float d = 6.28318530717958647692f * b;
    c = fmaf(-d, sa, ca);
    s = fmaf(d, ca, sa);
}

template <typename R>
__global__ void lag_table_kernel(const unsigned long long *__restrict__ Phi, int64_t Mp, int64_t Kp,
                                 int64_t K1, bool with_sin, R *__restrict__ E) {
    const int64_t k = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    const int64_t m = blockIdx.x;
    if (k >= Kp) return;
    R c = (R)0, s = (R)0;
    if (k < K1) lag_sincos<R>((unsigned long long)m * Phi[k], c, s);
    E[m * Kp + k] = c;
    if (with_sin) E[(Mp + m) * Kp + k] = s;
}

// ---------------------------------------------------------------------------
// spreading (global-memory grids)
// ---------------------------------------------------------------------------

template <typename V> __device__ __forceinline__ void atomic_add_v(V *p, decltype(V{}.x) a, decltype(V{}.x) b) {
    atomicAdd(&p->x, a);
    atomicAdd(&p->y, b);
}

constexpr int kSpreadThreads = 256;
constexpr int kSpreadTile = 2048;                          // grid cells of the SMEM tile
// staged points of a CTA of kPts points: one pad slot per kPts / 32 (a lane's run)
template <int kPts> __host__ __device__ constexpr int stage_pad() { return kPts + 32; }

// ceil(g) and ceil(g) - g for 1 <= g < 2^52 from the bit pattern of g: on this
// GPU FP64 conversion instructions run at about half the FP64 add rate, while
// integer shifts and masks run at the full integer rate.
__device__ __forceinline__ void split_ceil(double g, int &l0, float &f0) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(g);
    const int E = (int)((u >> 52) & 0x7FF) - 1023;             // g in [2^E, 2^(E+1))
    if (E < 0 || E > 40 || (u >> 63)) {  // outside any periodic domain (NaN, negative, huge):
        l0 = 0;                          // a plan's device guard reports it; keep indexing sane
        f0 = 0.0f;
        return;
    }
    const unsigned long long m = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const unsigned long long fr = m << (12 + E);               // fraction * 2^64
    l0 = (int)(m >> (52 - E)) + (fr != 0ull);
    // 1 - fraction (0 when g is an integer), 23 bits, built as a float in [1, 2) minus 1
    f0 = __uint_as_float(0x3F800000u | (unsigned)((0ull - fr) >> 41)) - 1.0f;
}


template <typename R> struct PointPhase;
template <> struct PointPhase<float> {
    // FP32 form: one FP64 FMA for the phase, everything else in integer/FP32
    __device__ static void eval(double t, double x, double a_scale, double c_off, float mhi, float mlo,
                                float inv, int &l0, float &f0, float &xs) {
        split_ceil(fma(t, a_scale, c_off), l0, f0);
        float xh, xl;
        split_df(x, xh, xl);
        xs = ((xh - mhi) + (xl - mlo)) * inv;
    }
};
template <> struct PointPhase<double> {
    __device__ static void eval(double t, double x, double a_scale, double c_off, double mean, double,
                                double inv, int &l0, double &f0, double &xs) {
        const double gs = fma(t, a_scale, c_off);
        l0 = (int)ceil(gs);
        f0 = (double)l0 - gs;
        xs = (x - mean) * inv;
    }
};

// One CTA per prep chunk (kPrepChunk consecutive points of one series).
// Grid coordinate of a point: g = (t - t_c) n_f / L; the kernel touches the W
// cells l0 .. l0+W-1 with l0 = ceil(g - W/2) (taken mod n_f), gs = g - W/2 + n_f
// formed with one FP64 FMA.
//   phase 1  coalesced loads of (t, x); per point (l0, f0, x_std) staged in SMEM;
//   phase 2  spreading: lane l of warp w takes points l*128 + w*16 + q, so the
//            32 lanes of an atomic instruction sit 128 points (several cells)
//            apart -- sorted points would otherwise hit the same cell 32 times;
//            the staging pad (one slot per 128 points) keeps these reads free of
//            bank conflicts;
//   phase 3  the chunk's tile of cells goes to the series' grid in HBM: plain
//            stores for the interior, atomic adds for the W-cell edges shared
//            with the neighbouring chunks.
// A chunk spanning more cells than the tile (a sparse series) adds straight to HBM.
//
// kFix (FP32): the tile holds fixed-point integers and a departing window cell
// is added with native 32-bit integer shared-memory atomics, instead of the
// compare-and-swap loop an FP32 add to shared memory takes.  A cell value v
// becomes round(v q); q is set per CTA so that no cell's sum can reach 2^31 (a
// cell sums at most the chunk's |x_std| for the values and its points' tap sums
// for the unit weights; each rounding adds at most 1/2), so the integer sums are
// exact and each flush is off by at most 1/(2q): about 8e-7 for the values and
// 3e-6 for the weights of a dense 4096-point chunk, the size of the FP32
// rounding of the same tile sums.
template <typename R, int W, int kPts, bool kFix = false>
__global__ void __launch_bounds__(kSpreadThreads)
spread_kernel(const double *__restrict__ t, const double *__restrict__ x,
              const int64_t *__restrict__ offs, const int64_t *__restrict__ offs_end,
              const int64_t *__restrict__ chunk_base,
              const int32_t *__restrict__ cs,
              const SeriesStats *__restrict__ st, const double *__restrict__ tc, double a_scale,
              int nf, const EsPoly<R, W, PolyDeg<W>::D> poly, float tap_sum,
              typename CT<R>::V *__restrict__ grids) {
    static_assert(!kFix || sizeof(R) == 4, "fixed-point tiles for the FP32 form");
    using V = typename CT<R>::V;
    constexpr int D = PolyDeg<W>::D;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int kSub = kPrepChunk / kPts;         // CTAs per statistics chunk
    constexpr int kRunLen = kPts / 32;              // a lane's run of points
    constexpr int kPer = kPts / kSpreadThreads;     // points per thread
    static_assert(kSub * kPts == kPrepChunk && kPer * kSpreadThreads == kPts, "whole chunks");
    auto pad = [](int p) { return p + p / kRunLen; };
    V *tile = reinterpret_cast<V *>(smem_raw);
    R *sf = reinterpret_cast<R *>(tile + kSpreadTile);
    R *sx = sf + stage_pad<kPts>();
    int *sl = reinterpret_cast<int *>(sx + stage_pad<kPts>());
    const int64_t g = blockIdx.x / kSub;
    const int64_t b = cs[g];
    const int64_t a0 = offs[b], a1 = offs_end[b];
    const int64_t start = a0 + (g - chunk_base[b]) * (int64_t)kPrepChunk + (int64_t)(blockIdx.x % kSub) * kPts;
    const int n = (int)(min(start + (int64_t)kPts, a1) - start);
    if (n <= 0) return;  // the part of a series' last chunk past its end
    const double c_off = -tc[b] * a_scale - 0.5 * W + nf;
    const double mean = st[b].mean;
    R mhi, mlo;
    if constexpr (sizeof(R) == 4) {
        float h, l;
        split_df(mean, h, l);
        mhi = h;
        mlo = l;
    } else {
        mhi = mean;
        mlo = 0;
    }
    const R inv = (R)st[b].inv_std;
    V *grid = grids + b * (int64_t)nf;
    const int mask = nf - 1;
    float asum = 0.0f;
#pragma unroll 4
    for (int r = 0; r < kPer; ++r) {
        const int p = threadIdx.x + r * kSpreadThreads;
        if (p < n) {
            int l0;
            R f0, xs;
            PointPhase<R>::eval(t[start + p], x[start + p], a_scale, c_off, mhi, mlo, inv, l0, f0, xs);
            const int pi = pad(p);
            sl[pi] = l0;
            sf[pi] = f0;
            sx[pi] = xs;
            if constexpr (kFix) asum += fabsf(xs);
        }
    }
    __shared__ float fix_q[2 + kSpreadThreads / 32];
    if constexpr (kFix) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) asum += __shfl_xor_sync(0xffffffffu, asum, o);
        if ((threadIdx.x & 31) == 0) fix_q[2 + (threadIdx.x >> 5)] = asum;
    }
    __syncthreads();
    if constexpr (kFix) {
        if (threadIdx.x == 0) {
            float s = 0.0f;
            for (int w = 0; w < kSpreadThreads / 32; ++w) s += fix_q[2 + w];
            const float room = 2147483648.0f - 8.0f * (float)n;  // below 2^31 after the roundings
            fix_q[0] = room / fmaxf(1.01f * s, 1e-20f);
            fix_q[1] = room / (1.01f * tap_sum * (float)n);
        }
    }
    const int l_first = sl[0];
    const int l_last = sl[pad(n - 1)] + W - 1;
    const int span = l_last - l_first + 1;
    const bool use_tile = span <= kSpreadTile;
    if (use_tile) {
        for (int i = threadIdx.x; i < span; i += blockDim.x) { tile[i].x = 0; tile[i].y = 0; }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // Each lane walks 16 consecutive sorted points and accumulates their taps in
    // a register window of W cells that slides with the points; a cell is added
    // to the tile (or the grid) only when the window leaves it.  Dense series put
    // many points in one cell, so most taps never touch shared memory.
    R wre[W], wim[W];
#pragma unroll
    for (int k = 0; k < W; ++k) { wre[k] = 0; wim[k] = 0; }
    int wbase = 0;
    bool started = false;
    float qr = 0.0f, qi = 0.0f;
    if constexpr (kFix) {
        qr = fix_q[0];
        qi = fix_q[1];
    }
    // A cell that got nothing is still added to the shared tile (a shared atomic
    // costs less than the branch that would skip it: 1.212 -> 1.159 ms on the bench
    // batch); only the grid's global atomics skip it.
    auto flush_cell = [&](int cell, R re, R im) {
        // inside the tile for sorted, in-domain points; anything else goes to the grid
        if (use_tile && (unsigned)(cell - l_first) < (unsigned)span) {
            if constexpr (kFix) {
                int2 *ic = reinterpret_cast<int2 *>(tile) + (cell - l_first);
                atomicAdd(&ic->x, __float2int_rn(re * qr));
                atomicAdd(&ic->y, __float2int_rn(im * qi));
            } else {
                atomicAdd(&tile[cell - l_first].x, re);
                atomicAdd(&tile[cell - l_first].y, im);
            }
        } else if (re != (R)0 || im != (R)0) {
            atomic_add_v(&grid[cell & mask], re, im);
        }
    };
    // FP32 taps (W = 8): the 36 polynomial coefficients are copied into a local
    // array before the point loop.  The compiler still reads them from the
    // parameter bank where they are used, but the FP32 instances came down from 48-78
    // to 39-63 registers and the spreading on the bench batch from 1.389 to 1.212 ms.
    // The FP64 form (W = 16, 120 coefficients) reads poly.c directly.
    constexpr bool kHoist = sizeof(R) == 4;
    constexpr int kNc = W / 2 * (D + 1);
    R cf[kHoist ? kNc : 1];
    if constexpr (kHoist) {
#pragma unroll
        for (int i = 0; i < kNc; ++i) cf[i] = poly.c[i];
    }
#pragma unroll 1
    for (int q = 0; q < kPer; ++q) {
        const int p = lane * kRunLen + warp * kPer + q;
        if (p >= n) break;
        const int pi = pad(p);
        const int l0 = sl[pi];
        const R f0 = sf[pi], xs = sx[pi];
        if (!started) {
            wbase = l0;
            started = true;
        }
        // A move of two cells or more flushes the whole window and restarts it at
        // l0 (cells that got nothing cost one test each); a move of one cell slides
        // it.  Sliding one cell at a time for every move below W ran the slide as
        // often as the warp's farthest-moving lane needed (a lane's points crossing
        // the gap between two nights): spreading on the bench batch 1.517 -> 1.348 ms
        // (a flush from 3 cells: 1.361 ms, from 4: 1.429 ms); the FP32 form's largest
        // error against FP64 on that batch is unchanged (4.509e-6).
        const int dd = l0 - wbase;
        if (dd >= 2) {
#pragma unroll
            for (int k = 0; k < W; ++k) {
                flush_cell(wbase + k, wre[k], wim[k]);
                wre[k] = 0;
                wim[k] = 0;
            }
            wbase = l0;
        } else if (dd == 1) {  // slide by one cell
            flush_cell(wbase, wre[0], wim[0]);
#pragma unroll
            for (int k = 0; k < W - 1; ++k) { wre[k] = wre[k + 1]; wim[k] = wim[k + 1]; }
            wre[W - 1] = 0;
            wim[W - 1] = 0;
            ++wbase;
        }
        // taps k and W-1-k are one polynomial at u and -u (phi is even): its even
        // and odd parts in v = u^2 give both with about half the multiply-adds
        const R u = (R)2 * f0 - (R)1;
        const R v = u * u;
#pragma unroll
        for (int k = 0; k < W / 2; ++k) {
            const R *c;
            if constexpr (kHoist) c = cf + k * (D + 1); else c = poly.c + k * (D + 1);
            constexpr int De = D & ~1, Do = (D - 1) | 1;  // highest even / odd power
            R e = c[De], o = c[Do];
#pragma unroll
            for (int d = De - 2; d >= 0; d -= 2) e = fma(e, v, c[d]);
#pragma unroll
            for (int d = Do - 2; d >= 1; d -= 2) o = fma(o, v, c[d]);
            const R pk = fma(u, o, e), pm = fma(-u, o, e);
            wre[k] = fma(pk, xs, wre[k]);
            wim[k] += pk;
            wre[W - 1 - k] = fma(pm, xs, wre[W - 1 - k]);
            wim[W - 1 - k] += pm;
        }
    }
    if (started) {
#pragma unroll
        for (int k = 0; k < W; ++k) flush_cell(wbase + k, wre[k], wim[k]);
    }
    if (use_tile) {
        __syncthreads();
        // Sorted points: a neighbouring chunk's cells overlap this tile only in its
        // first and last W cells, so the interior is this chunk's alone and goes to
        // the (zeroed) grid with plain stores; the edges are added atomically.
        for (int i = threadIdx.x; i < span; i += blockDim.x) {
            V v = tile[i];
            if constexpr (kFix) {
                const int2 c = reinterpret_cast<const int2 *>(tile)[i];
                v.x = (float)c.x / qr;
                v.y = (float)c.y / qi;
            }
            if (v.x == 0 && v.y == 0) continue;
            V *dst = &grid[(l_first + i) & mask];
            if (i >= W && i < span - W) {
                *dst = v;
            } else if constexpr (sizeof(R) == 4) {
                atomicAdd(reinterpret_cast<float2 *>(dst), make_float2(v.x, v.y));
            } else {
                atomic_add_v(dst, v.x, v.y);
            }
        }
    }
}

template <typename R, int kPts>
constexpr size_t spread_smem_bytes() {
    return kSpreadTile * sizeof(typename CT<R>::V) + (size_t)stage_pad<kPts>() * (2 * sizeof(R) + sizeof(int));
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
// FFT and spectrum of one series' grid in shared memory (FP32 ACFs on grids of
// up to 2^14 cells): one CTA per series reads its spread grid from HBM once,
// transforms it in place in shared memory and writes only the weighted power
// spectra -- instead of lg / 3 global Stockham passes that each read and write
// the whole batch, and a spectrum pass that reads it once more.
//   load      the grid into shared memory, padded by one cell per 32 so that the
//             late passes, whose lanes step across blocks, fall on distinct bank
//             pairs;
//   fft       in-place decimation-in-frequency passes of radix 8 (then 4 or 2):
//             for a block of length Lb, butterfly j takes the R cells at stride
//             Lb / R, applies the R-point DFT and the twiddles w_Lb^(j r), read
//             as the product of two 128-entry tables in shared memory; the
//             transform ends at digit-reversed positions;
//   spectrum  modes m and n_f - m read from their digit-reversed positions,
//             Hermitian unpack, wgt_m |X_m|^2 and wgt_m |W_m|^2 into the A rows
//             (zero beyond the kept modes), as spectrum_kernel.
// ---------------------------------------------------------------------------
constexpr int kSmemFftThreads = 512;
constexpr int kSmemFftMaxLg = 14;
constexpr int kSmemFftTw = 128;  // entries of each twiddle table

__host__ __device__ __forceinline__ int sfft_pad(int i) { return i + (i >> 5); }
inline size_t sfft_smem_bytes(int lg) {
    return (size_t)sfft_pad(1 << lg) * sizeof(float2) + 2 * kSmemFftTw * sizeof(float2);
}

// position of frequency k after the in-place passes (radix 8 while >= 3 bits
// remain, then 4 or 2): its mixed-radix digits, first pass's digit least
// significant, placed at the passes' strides
__device__ __forceinline__ int sfft_pos(int k, int lg) {
    int pos = 0;
    for (int Llg = lg; Llg > 0;) {
        const int rlg = Llg >= 3 ? 3 : Llg;
        pos += (k & ((1 << rlg) - 1)) << (Llg - rlg);
        k >>= rlg;
        Llg -= rlg;
    }
    return pos;
}

// exp(+2 pi i q / n_f) = T1[q >> 7] T2[q & 127]
__device__ __forceinline__ float2 sfft_tw(const float2 *T1, const float2 *T2, int q) {
    return cmul(T1[q >> 7], T2[q & (kSmemFftTw - 1)]);
}

template <int R>
__device__ __forceinline__ void sfft_pass(float2 *g, int lg, int Llg, const float2 *T1, const float2 *T2) {
    constexpr int rlg = R == 8 ? 3 : (R == 4 ? 2 : 1);
    const int slg = Llg - rlg;   // log2 of the butterfly stride Lb / R
    const int blg = lg - Llg;    // log2 of the number of blocks (= n_f / Lb)
    const int nbf = 1 << (lg - rlg);
    for (int t = threadIdx.x; t < nbf; t += kSmemFftThreads) {
        int j, blk;
        if (slg >= 5) {          // lanes along j: consecutive cells
            j = t & ((1 << slg) - 1);
            blk = t >> slg;
        } else {                 // lanes along blocks: padded cells on distinct bank pairs
            blk = t & ((1 << blg) - 1);
            j = t >> blg;
        }
        const int base = (blk << Llg) + j;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = g[sfft_pad(base + (r << slg))];
        dft<R>(v);
        // twiddles w^(q r), q = j 2^blg: w^q, w^2q and w^4q from the tables, the
        // others as their products (about 3 ulp), so that a butterfly reads 3
        // table pairs instead of R - 1
        const int q = j << blg;
        const float2 w1 = sfft_tw(T1, T2, q);
        v[1] = cmul(v[1], w1);
        if constexpr (R >= 4) {
            const float2 w2 = sfft_tw(T1, T2, 2 * q);
            v[2] = cmul(v[2], w2);
            const float2 w3 = cmul(w2, w1);
            v[3] = cmul(v[3], w3);
            if constexpr (R == 8) {
                const float2 w4 = sfft_tw(T1, T2, 4 * q);
                v[4] = cmul(v[4], w4);
                v[5] = cmul(v[5], cmul(w4, w1));
                v[6] = cmul(v[6], cmul(w4, w2));
                v[7] = cmul(v[7], cmul(w4, w3));
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) g[sfft_pad(base + (r << slg))] = v[r];
    }
}

__global__ void __launch_bounds__(kSmemFftThreads)
fft_spectrum_smem_kernel(const float2 *__restrict__ grids, int lg, int64_t M, int64_t Mp,
                         const float2 *__restrict__ tw, const float *__restrict__ wgt, float *__restrict__ Anum,
                         float *__restrict__ Aden) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nf = 1 << lg, nfm = nf - 1;
    float2 *g = reinterpret_cast<float2 *>(smem_raw);
    float2 *T1 = g + sfft_pad(nf), *T2 = T1 + kSmemFftTw;
    const int64_t b = blockIdx.x;
    const float4 *src = reinterpret_cast<const float4 *>(grids + b * (int64_t)nf);  // two cells per load
#pragma unroll 8
    for (int i = threadIdx.x; i < nf / 2; i += kSmemFftThreads) {
        const float4 v = src[i];
        g[sfft_pad(2 * i)] = make_float2(v.x, v.y);
        g[sfft_pad(2 * i + 1)] = make_float2(v.z, v.w);
    }
    for (int i = threadIdx.x; i < kSmemFftTw; i += kSmemFftThreads) {
        T1[i] = (i << 7) < nf ? tw[i << 7] : make_float2(1.0f, 0.0f);
        T2[i] = i < nf ? tw[i] : make_float2(1.0f, 0.0f);
    }
    for (int Llg = lg; Llg > 0;) {
        const int rlg = Llg >= 3 ? 3 : Llg;
        __syncthreads();
        if (rlg == 3) sfft_pass<8>(g, lg, Llg, T1, T2);
        else if (rlg == 2) sfft_pass<4>(g, lg, Llg, T1, T2);
        else sfft_pass<2>(g, lg, Llg, T1, T2);
        Llg -= rlg;
    }
    __syncthreads();
    float *an = Anum + b * Mp, *ad = Aden + b * Mp;
    for (int m = threadIdx.x; m < Mp; m += kSmemFftThreads) {
        float vn = 0.0f, vd = 0.0f;
        if (m < M) {
            const float2 a = g[sfft_pad(sfft_pos(m, lg))];
            const float2 c = g[sfft_pad(sfft_pos((nf - m) & nfm, lg))];
            const float Xr = (a.x + c.x) * 0.5f, Xi = (a.y - c.y) * 0.5f;
            const float Wr = (a.y + c.y) * 0.5f, Wi = (c.x - a.x) * 0.5f;
            vn = wgt[m] * (Xr * Xr + Xi * Xi);
            vd = wgt[m] * (Wr * Wr + Wi * Wi);
        }
        an[m] = vn;
        ad[m] = vd;
    }
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
                                       const int *__restrict__ status, const float *__restrict__ dc_num,
                                       const float *__restrict__ dc_den, int64_t row,
                                       const int64_t *__restrict__ row_map, double *__restrict__ c,
                                       double *__restrict__ bo, int64_t *__restrict__ cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * K) return;
    const int64_t b = i / K, k = i - b * K;
    const int64_t o = (row_map ? row_map[b] : b) * K + k;  // output element (a bucket's series keep their rows)
    if (*status != 0) {  // a bounded device wait gave up: no valid result
        c[o] = __longlong_as_double(0x7ff8000000000000ll);
        if (bo) bo[o] = c[o];
        if (cnt) cnt[o] = -1;
        return;
    }
    // m = 0 terms kept out of the tensor-core sums (cos 0 = 1, sin 0 = 0)
    const double n0 = dc_num ? (double)dc_num[b * row] : 0.0, d0 = dc_den ? (double)dc_den[b * row] : 0.0;
    const double N = acc_num[b * Kp + k] + n0, D = acc_den[b * Kp + k] + d0;
    double ci = N / fmax(D, 1e-16);
    if (lag0_mode == 1) {          // ACF: divide by c(0) from the appended zero lag
        ci /= (acc_num[b * Kp + K] + n0) / fmax(acc_den[b * Kp + K] + d0, 1e-16);
    } else if (lag0_mode == 2) {   // CCF: divide by sqrt(ACF_x(0) ACF_y(0))
        const double sx = lag0[4 * b] / fmax(lag0[4 * b + 1], 1e-16);
        const double sy = lag0[4 * b + 2] / fmax(lag0[4 * b + 3], 1e-16);
        ci /= sqrt(sx * sy);
    }
    c[o] = ci;
    if (bo) bo[o] = D;
    if (cnt) cnt[o] = 0;
}

template <typename T>
T *take(char *base, size_t &used, size_t count) {
    T *p = reinterpret_cast<T *>(base + used);
    used += al(count * sizeof(T));
    return p;
}

void make_plan(const SpectralArgs &a, double max_span, SpectralPrepared &p) {
    const double tol = a.tol;
    if (a.kernel == 1) {
        // spectral-sinc rectangle: compact support (alias margin 2h); the sum
        // keeps |m| <= L / (h tol), so the truncated kernel's error near a
        // window edge is of order L / (M h) = tol of a pair's weight
        p.R_alias = 2.0;
        p.L = max_span + a.max_tau + p.R_alias * a.h;
        p.M = (int64_t)std::ceil(p.L / (a.h * tol)) + 1;
    } else {
        p.R_alias = std::sqrt(2.0 * std::log(1.0 / (tol * 1e-2)));
        p.L = max_span + a.max_tau + p.R_alias * a.h;
        const double delta = tol * 1e-3;
        const double mscale = std::sqrt(std::log(1.0 / delta) / (2.0 * kPi * kPi));
        p.M = (int64_t)std::ceil(p.L * mscale / a.h) + 1;
    }
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
    p.fp32 = a.fp32;
    // One series: the mode sums at the lags directly (runs of modes from exactly
    // reduced 64-bit phases, stepped by rotations) instead of a [modes x lags]
    // table whose entries would each be computed, packed and read once.  A batch
    // shares the table across its series and keeps it.
    p.direct = a.B == 1;
    p.kernel = a.kernel;
    p.acf = a.acf;
    p.lag0 = a.lag0;
    p.B = a.B;
    p.K = a.K;
    p.h = a.h;
    p.max_tau = a.max_tau;
}

template <typename R>
struct Bufs {
    typename CT<R>::V *grid_x, *grid_y, *scratch, *tw;
    double *wgt64;
    R *wgt, *Anum, *Aden, *E;
    double2 *Apk;  // direct mode sums: the rows as complex spectra
    unsigned char *At, *Et;  // FP32 form: operand tiles of the tensor-core contraction
    double *acc_num, *acc_den, *lag0, *d_tc;
    unsigned long long *d_phi;
    double *d_gx, *d_gphi;
    size_t used;
};

// The one layout of the spectral workspace, used by prepare, launch and sizing.
template <typename R>
Bufs<R> carve(const SpectralPrepared &p, char *ws) {
    using V = typename CT<R>::V;
    const int64_t B = p.B;
    const bool ccf = !p.acf;
    Bufs<R> b{};
    size_t used = 0;
    b.grid_x = take<V>(ws, used, B * (size_t)p.nf);
    b.grid_y = ccf ? take<V>(ws, used, B * (size_t)p.nf) : nullptr;
    b.scratch = take<V>(ws, used, B * (size_t)p.nf);
    b.tw = take<V>(ws, used, p.nf);
    b.wgt64 = take<double>(ws, used, p.Mp);
    b.wgt = take<R>(ws, used, p.Mp);
    b.Anum = take<R>(ws, used, B * p.M2);
    b.Aden = take<R>(ws, used, B * p.M2);
    b.E = take<R>(ws, used, p.direct ? 0 : p.M2 * p.Kp);
    b.Apk = take<double2>(ws, used, (p.direct && !std::is_same<R, float>::value) ? 2 * p.Mp : 0);
    const bool tc = std::is_same<R, float>::value && !p.direct;
    b.At = take<unsigned char>(ws, used, tc ? tc_a_tiles_bytes(B, p.M2) : 0);
    b.Et = take<unsigned char>(ws, used, tc ? tc_e_tiles_bytes(p.M2, p.Kp) : 0);
    b.acc_num = take<double>(ws, used, B * p.Kp);
    b.acc_den = take<double>(ws, used, B * p.Kp);
    b.lag0 = take<double>(ws, used, 4 * B);
    b.d_tc = take<double>(ws, used, B);
    b.d_phi = take<unsigned long long>(ws, used, p.Kp);
    b.d_gx = take<double>(ws, used, p.nq);
    b.d_gphi = take<double>(ws, used, p.nq);
    b.used = used + 256;
    return b;
}

template <typename R>
void prepare_typed(const SpectralPrepared &p, char *ws, const double *h_tc,
                   const unsigned long long *h_phi, const std::vector<double> &gx,
                   const std::vector<double> &gphi, char *pinned, cudaStream_t st) {
    using V = typename CT<R>::V;
    const int64_t B = p.B;
    const bool ccf = !p.acf;
    Bufs<R> bf = carve<R>(p, ws);
    size_t off = 0;
    auto up = [&](void *dst, const void *src, size_t bytes) {
        std::memcpy(pinned + off, src, bytes);
        copy_pinned(dst, pinned + off, bytes, st);
        off += al(bytes);
    };
    up(bf.d_tc, h_tc, B * 8);
    up(bf.d_phi, h_phi, p.Kp * 8);
    up(bf.d_gx, gx.data(), p.nq * 8);
    up(bf.d_gphi, gphi.data(), p.nq * 8);
    NCF_LAUNCH("mode_weight_kernel", st,
               mode_weight_kernel<<<(unsigned)((p.Mp + 255) / 256), 256, 0, st>>>(
                   bf.d_gx, bf.d_gphi, p.nq, p.M, p.Mp, p.W, p.nf, p.L, p.h, p.kernel == 1, bf.wgt64,
                   std::is_same<R, float>::value ? reinterpret_cast<float *>(bf.wgt) : nullptr));
    if (std::is_same<R, double>::value)
        cudaMemcpyAsync(bf.wgt, bf.wgt64, p.Mp * 8, cudaMemcpyDeviceToDevice, st);
    NCF_LAUNCH("twiddle_kernel", st, twiddle_kernel<V><<<twiddle_blocks(p.nf), 256, 0, st>>>(bf.tw, p.nf));
    if (!p.direct) {
        dim3 grid((unsigned)p.Mp, (unsigned)((p.Kp + 127) / 128));
        NCF_LAUNCH("lag_table_kernel", st,
                   lag_table_kernel<R><<<grid, 128, 0, st>>>(bf.d_phi, p.Mp, p.Kp, p.K1, ccf, bf.E));
        if constexpr (std::is_same<R, float>::value)
            launch_tc_pack_e(reinterpret_cast<const float *>(bf.E), p.M2, p.Kp, bf.Et, st);
    }
}

// Direct mode sums of one FP32 series at the lags: for channel z (numerator,
// denominator) and lag k, acc_z[k] += sum_m (A_z[m] cos(2 pi m tau_k / L) +
// A_z[Mp + m] sin(2 pi m tau_k / L)) (the sin block for a CCF only).  A warp
// takes kDirRuns runs of kDirRun modes, one lag per lane (with few lags, S lanes
// share a lag and take every S-th mode); each run starts from its exactly
// reduced 64-bit phase m phi[k] (split-phase FP32 sincos, as the lag table)
// and steps by the rotation S phi[k], so FP32 rounding drifts over at most
// kDirRun / S steps.  Runs are summed in FP32, the warp's runs and lanes in FP64.
constexpr int kDirWarps = 8, kDirRun = 32, kDirRuns = 8;
__global__ void __launch_bounds__(kDirWarps * 32)
direct_modes_f32_kernel(const float *__restrict__ An, const float *__restrict__ Ad, int64_t Mp, bool ccf,
                        const unsigned long long *__restrict__ phi, int64_t K, double *__restrict__ acc_n,
                        double *__restrict__ acc_d) {
    __shared__ double part_n[kDirWarps][32], part_d[kDirWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int S = (K <= 16) ? (int)(32 / K) : 1;
    const int64_t k = (int64_t)blockIdx.y * 32 + lane / S;
    const int sub = lane % S;
    const int64_t m0 = ((int64_t)blockIdx.x * kDirWarps + warp) * (kDirRun * kDirRuns);
    double sn = 0.0, sd = 0.0;
    if (k < K && lane / S < 32 / S) {
        const unsigned long long ph = phi[k];
        float rc, rs;
        lag_sincos<float>((unsigned long long)S * ph, rc, rs);
        for (int r = 0; r < kDirRuns; ++r) {
            const int64_t ma = m0 + (int64_t)r * kDirRun, mb = min(ma + kDirRun, Mp);
            if (ma + sub >= mb) break;
            float zc, zs;
            lag_sincos<float>((unsigned long long)(ma + sub) * ph, zc, zs);
            float fn = 0.0f, fd = 0.0f;
            for (int64_t m = ma + sub; m < mb; m += S) {
                if (ccf) {
                    fn = fmaf(An[m], zc, fmaf(An[Mp + m], zs, fn));
                    fd = fmaf(Ad[m], zc, fmaf(Ad[Mp + m], zs, fd));
                } else {
                    fn = fmaf(An[m], zc, fn);
                    fd = fmaf(Ad[m], zc, fd);
                }
                const float c2 = fmaf(zc, rc, -zs * rs);
                zs = fmaf(zs, rc, zc * rs);
                zc = c2;
            }
            sn += (double)fn;
            sd += (double)fd;
        }
    }
    part_n[warp][lane] = sn;
    part_d[warp][lane] = sd;
    __syncthreads();
    if (warp == 0 && lane < 32 / S) {
        const int64_t kk = (int64_t)blockIdx.y * 32 + lane;
        if (kk < K) {
            double a = 0.0, b = 0.0;
            for (int w = 0; w < kDirWarps; ++w)
                for (int j = 0; j < S; ++j) {
                    a += part_n[w][lane * S + j];
                    b += part_d[w][lane * S + j];
                }
            atomicAdd(acc_n + kk, a);
            atomicAdd(acc_d + kk, b);
        }
    }
}

// The FP64 spectra rows of one series as complex values (cos row, sin row; an
// ACF's sin row is zero) for the direct mode sums.
__global__ void pack_rows_kernel(const double *__restrict__ num, const double *__restrict__ den, int64_t Mp,
                                 bool ccf, double2 *__restrict__ out) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= Mp) return;
    out[m] = make_double2(num[m], ccf ? num[Mp + m] : 0.0);
    out[Mp + m] = make_double2(den[m], ccf ? den[Mp + m] : 0.0);
}

// Contraction of the A rows with the lag table, then the normalisation.
template <typename R>
ncf_status contract_and_finish(const SpectralArgs &a, const SpectralPrepared &p, const Bufs<R> &bf, int *status,
                               cudaStream_t st, std::string *msg) {
    const int64_t B = p.B;
    const bool ccf = !p.acf;
    cudaMemsetAsync(bf.acc_num, 0, B * p.Kp * 8, st);
    cudaMemsetAsync(bf.acc_den, 0, B * p.Kp * 8, st);
    if (std::is_same<R, float>::value && !p.direct && p.contract_variant == 0) {
        // FP32 form: tensor cores (TF32 split products, FP64 chunk sums)
        launch_tc_pack_a(reinterpret_cast<const float *>(bf.Anum), reinterpret_cast<const float *>(bf.Aden), B,
                         p.M2, bf.At, st);
        launch_contract_tc(bf.At, bf.Et, B, p.M2, p.Kp, a.sm_count, bf.acc_num, bf.acc_den, status, st);
    } else if (p.direct && std::is_same<R, float>::value) {
        const int64_t per = (int64_t)kDirWarps * kDirRun * kDirRuns;
        dim3 grid((unsigned)((p.Mp + per - 1) / per), (unsigned)((p.K1 + 31) / 32));
        NCF_LAUNCH("direct_modes_f32_kernel", st,
                   direct_modes_f32_kernel<<<grid, kDirWarps * 32, 0, st>>>(
                       reinterpret_cast<const float *>(bf.Anum), reinterpret_cast<const float *>(bf.Aden), p.Mp,
                       ccf, bf.d_phi, p.K1, bf.acc_num, bf.acc_den));
    } else if (p.direct) {
        // N_k = sum_m Re(A_m exp(-2 pi i m tau_k / L)), A_m = (cos row, sin row) of
        // the spectra, at the K + 1 lags (with the appended zero lag)
        NCF_LAUNCH("pack_rows_kernel", st,
                   pack_rows_kernel<<<(unsigned)((p.Mp + 255) / 256), 256, 0, st>>>(
                       reinterpret_cast<const double *>(bf.Anum), reinterpret_cast<const double *>(bf.Aden), p.Mp,
                       ccf, bf.Apk));
        paper_eval(bf.Apk, p.Mp - 1, bf.d_phi, p.K1, bf.acc_num, st, bf.Apk + p.Mp, bf.acc_den);
    } else {
        dim3 grid((unsigned)((p.Kp + kBN - 1) / kBN), (unsigned)((B + kBM - 1) / kBM),
                  (unsigned)((p.M2 + kChunk - 1) / kChunk));
        NCF_LAUNCH("contract_kernel", st,
                   contract_kernel<R><<<grid, 256, 0, st>>>(bf.Anum, bf.Aden, bf.E, B, p.M2, p.Kp, bf.acc_num,
                                                            bf.acc_den));
    }
    const int mode = p.lag0 ? (ccf ? 2 : 1) : 0;
    // the tensor-core contraction leaves out the m = 0 term, which the finish adds in FP64
    const bool m0_apart = std::is_same<R, float>::value && !p.direct && p.contract_variant == 0;
    NCF_LAUNCH("finish_spectral_kernel", st,
               finish_spectral_kernel<<<(unsigned)((B * p.K + 255) / 256), 256, 0, st>>>(
                   bf.acc_num, bf.acc_den, B, p.K, p.Kp, mode, bf.lag0, status,
                   m0_apart ? reinterpret_cast<const float *>(bf.Anum) : nullptr,
                   m0_apart ? reinterpret_cast<const float *>(bf.Aden) : nullptr, p.M2, a.row_map,
                   a.c_out, a.b_out, a.count_out));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        *msg = std::string("spectral path launch failed: ") + cudaGetErrorString(e);
        return NCF_ECUDA;
    }
    return NCF_OK;
}


template <typename R>
ncf_status launch_typed(const SpectralArgs &a, const SpectralPrepared &p, char *ws, int *status,
                        cudaStream_t st, std::string *msg) {
    using V = typename CT<R>::V;
    const int64_t B = p.B;
    const bool ccf = !p.acf;
    Bufs<R> bf = carve<R>(p, ws);
    // spreading
    const double a_scale = (double)p.nf / p.L;
    constexpr size_t smem = spread_smem_bytes<R, kPrepChunk>();
    constexpr size_t smem_half = spread_smem_bytes<R, kPrepChunk / 2>();
    static std::atomic<unsigned long long> attr_done{0};
    once_per_device(attr_done, [&] {
        return set_smem_limit(spread_kernel<R, 8, kPrepChunk>, smem) &
               set_smem_limit(spread_kernel<R, 8, kPrepChunk / 2>, smem_half) &
               set_smem_limit(spread_kernel<R, 16, kPrepChunk>, smem) &
               (sizeof(R) != 4 || (set_smem_limit(spread_kernel<float, 8, kPrepChunk, true>, smem) &
                                   set_smem_limit(spread_kernel<float, 8, kPrepChunk / 2, true>, smem_half)));
    });
    EsPoly<R, 8, PolyDeg<8>::D> poly8{};
    EsPoly<R, 16, PolyDeg<16>::D> poly16{};
    for (size_t i = 0; i < p.poly.size(); ++i) {
        if (p.W == 8) poly8.c[i] = (R)p.poly[i];
        else poly16.c[i] = (R)p.poly[i];
    }
    const float tap_sum = (float)p.tap_sum;
    // FP32 spreading shapes (the tuner's choice): bit 0 = CTAs of half a statistics
    // chunk, bit 1 = fixed-point tile sums
    auto spread = [&](const SpecSide &sd, V *grid) {
        cudaMemsetAsync(grid, 0, B * (size_t)p.nf * sizeof(V), st);
        const int64_t *offs_end = sd.d_offs_end ? sd.d_offs_end : sd.d_offs + 1;
        auto go = [&](auto kern, unsigned grid_dim, size_t sm, const auto &poly) {
            NCF_LAUNCH("spread_kernel", st,
                       kern<<<grid_dim, kSpreadThreads, sm, st>>>(sd.t, sd.v, sd.d_offs, offs_end, sd.d_chunk_base,
                                                                   sd.d_cs, sd.d_stats, bf.d_tc, a_scale, p.nf, poly,
                                                                   tap_sum, grid));
            return NCF_OK;
        };
        const unsigned full = (unsigned)sd.n_chunks, half = (unsigned)(2 * sd.n_chunks);
        if (p.W != 8) return go(spread_kernel<R, 16, kPrepChunk>, full, smem, poly16);
        if constexpr (sizeof(R) == 4) {
            if (p.spread_variant == 2) return go(spread_kernel<float, 8, kPrepChunk, true>, full, smem, poly8);
            if (p.spread_variant == 3) return go(spread_kernel<float, 8, kPrepChunk / 2, true>, half, smem_half, poly8);
        }
        if (p.spread_variant & 1) return go(spread_kernel<R, 8, kPrepChunk / 2>, half, smem_half, poly8);
        return go(spread_kernel<R, 8, kPrepChunk>, full, smem, poly8);
    };
    spread(a.x, bf.grid_x);
    if (ccf) spread(a.y, bf.grid_y);

    // FFT passes (ping-pong with the scratch grid); returns the buffer holding the result
    const RadixPlan rp = radix_plan(p.lg);
    auto fft = [&](V *grid) -> V * {
        V *in = grid, *out = bf.scratch;
        int Ns = 1;
        for (int q = 0; q < rp.n_pass; ++q) {
            const int rad = rp.radix[q];
            const int64_t items = B * (int64_t)(p.nf / rad);
            const unsigned blocks = (unsigned)((items + 255) / 256);
            if (rad == 8)
                NCF_LAUNCH("fft_pass_kernel", st,
                           fft_pass_kernel<V, 8><<<blocks, 256, 0, st>>>(in, out, p.lg, Ns, bf.tw, B));
            else if (rad == 4)
                NCF_LAUNCH("fft_pass_kernel", st,
                           fft_pass_kernel<V, 4><<<blocks, 256, 0, st>>>(in, out, p.lg, Ns, bf.tw, B));
            else
                NCF_LAUNCH("fft_pass_kernel", st,
                           fft_pass_kernel<V, 2><<<blocks, 256, 0, st>>>(in, out, p.lg, Ns, bf.tw, B));
            Ns *= rad;
            std::swap(in, out);
        }
        return in;
    };
    if constexpr (std::is_same<R, float>::value) {
        if (!ccf && p.lg <= kSmemFftMaxLg && p.lg >= 7 && p.fft_variant == 0) {
            // ACF on a grid that fits shared memory: FFT and spectrum per series there
            const size_t smem = sfft_smem_bytes(p.lg);
            static std::atomic<unsigned long long> sfft_done{0};
            once_per_device(sfft_done,
                            [&] { return set_smem_limit(fft_spectrum_smem_kernel, sfft_smem_bytes(kSmemFftMaxLg)); });
            NCF_LAUNCH("fft_spectrum_smem_kernel", st,
                       fft_spectrum_smem_kernel<<<(unsigned)B, kSmemFftThreads, smem, st>>>(
                           reinterpret_cast<const float2 *>(bf.grid_x), p.lg, p.M, p.Mp,
                           reinterpret_cast<const float2 *>(bf.tw), reinterpret_cast<const float *>(bf.wgt),
                           reinterpret_cast<float *>(bf.Anum), reinterpret_cast<float *>(bf.Aden)));
            return contract_and_finish(a, p, bf, status, st, msg);
        }
    }
    V *Gx = fft(bf.grid_x);
    if (Gx == bf.scratch && ccf) {
        // keep x's transform out of the scratch buffer before y's passes
        cudaMemcpyAsync(bf.grid_x, bf.scratch, B * (size_t)p.nf * sizeof(V), cudaMemcpyDeviceToDevice, st);
        Gx = bf.grid_x;
    }
    V *Gy = ccf ? fft(bf.grid_y) : nullptr;

    const bool lag0_ccf = p.lag0 && ccf;
    if (lag0_ccf) cudaMemsetAsync(bf.lag0, 0, 4 * B * 8, st);
    {
        dim3 grid((unsigned)((p.Mp + 255) / 256), (unsigned)std::min<int64_t>(B, 65535));
        NCF_LAUNCH("spectrum_kernel", st,
                   spectrum_kernel<R><<<grid, 256, 0, st>>>(Gx, Gy, p.nf, p.M, p.Mp, B, bf.wgt, bf.Anum,
                                                            bf.Aden, lag0_ccf ? bf.lag0 : nullptr));
    }
    return contract_and_finish(a, p, bf, status, st, msg);
}

// Checks, on the device, that every series of an executed plan still fits the
// plan's periodic domain: its span leaves every pair separation at least
// R_alias h away from +-L (span <= L - max|tau| - R_alias h; the result does not
// depend on where the series sits), and its points stay within 0.9 L of the
// plan's centre so that grid coordinates stay positive.
__global__ void spectral_guard_kernel(const SeriesStats *__restrict__ sx, const SeriesStats *__restrict__ sy,
                                      const double *__restrict__ tc, int64_t B, double max_span, double reach,
                                      int *__restrict__ status) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    double lo = sx[b].t_first, hi = sx[b].t_last;
    if (sy) {
        lo = fmin(lo, sy[b].t_first);
        hi = fmax(hi, sy[b].t_last);
    }
    if (!(hi - lo <= max_span) || !(lo >= tc[b] - reach) || !(hi <= tc[b] + reach))
        atomicOr(status, STATUS_DOMAIN);
}

// ---------------------------------------------------------------------------
// The paper's own NUFFT estimators (Algorithms 2-4, smoothing step included):
// deconvolved type-1 coefficients on the padded period of Algorithm 1.
// ---------------------------------------------------------------------------
// phihat_m = (W/2) int_{-1}^{1} phi(z) cos(pi m W z / n_f) dz varies on a scale of
// about n_f / W modes (its value falls by a factor of about 4 from m = 0 to the
// band edge), so Gauss-Legendre quadrature runs only at every kPhiStep-th mode and
// the modes between come from 8-point Lagrange interpolation (nodes -3 .. 4 around
// them): the interpolation error, (pi W kPhiStep / n_f)^8 / 8! relative, is far
// below the quadrature's own rounding (about 3e-15).
constexpr int kPhiStep = 64;
constexpr int kPhiTaps = 8;

// coarse[i] = the positive-node half of the quadrature at mode (i - 3) kPhiStep
// (phihat is even in m, so the three leading negative modes are valid too)
__global__ void paper_phihat_kernel(int nf, int W, const double *__restrict__ gx, const double *__restrict__ gphi,
                                    int nq_half, int64_t n_coarse, double *__restrict__ coarse) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_coarse) return;
    const double k = (double)((i - 3) * kPhiStep);
    double acc = 0.0;
    for (int q = 0; q < nq_half; ++q) acc = fma(gphi[q], cospi(k * ((double)W / nf * gx[q])), acc);
    coarse[i] = acc;
}

// F_m = X_m / phihat_m for m = 0 .. Mh, X_m from the Hermitian unpack of the grid
// transform, phihat_m interpolated from the coarse quadrature (lagw[r][j]: the
// Lagrange weight of node j - 3 at offset r / kPhiStep).
// G: the FFT of the spread grid.  packed = 0: one series, its values in the real
// part (the imaginary part holds the unit weights, unused here); packed = 1: the
// CCF's two series, x in the real and y in the imaginary part, so that one FFT
// serves both transforms and Hermitian symmetry separates them.
__global__ void paper_coef_kernel(const double2 *__restrict__ G, int packed, int nf, int64_t Mh, int W,
                                  const double *__restrict__ coarse, const double *__restrict__ lagw,
                                  double2 *__restrict__ Fx, double2 *__restrict__ Fy, double *__restrict__ invph) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m > Mh) return;
    const int64_t c = m / kPhiStep;
    const double *wr = lagw + (m - c * kPhiStep) * kPhiTaps;
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < kPhiTaps; ++j) acc = fma(wr[j], coarse[c + j], acc);
    const double inv = 1.0 / (W * acc);  // (W/2) x 2 x (sum over the positive nodes)
    invph[m] = inv;
    double2 X, Wt;
    unpack(G, nf, m, X, Wt);
    Fx[m] = make_double2(X.x * inv, X.y * inv);
    if (packed) Fy[m] = make_double2(Wt.x * inv, Wt.y * inv);
}

// the CCF's second series into the imaginary part of the first one's grid
__global__ void paper_pack_kernel(double2 *__restrict__ gx, const double2 *__restrict__ gy, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) gx[i].y = gy[i].x;
}

struct PaperBufs {
    double2 *grid_x, *grid_y, *scratch, *tw, *Fx, *Fy;
    double *d_tc, *d_gx, *d_gphi, *invph, *coarse, *lagw;
    size_t used;
};

// coarse quadrature samples: modes -3 kPhiStep .. (Mh / kPhiStep + 4) kPhiStep
int64_t paper_coarse_count(const PaperModes &pm) { return pm.Mh / kPhiStep + 8; }

// Lagrange weights of the nodes -3 .. 4 at t = r / kPhiStep, r = 0 .. kPhiStep - 1
const std::vector<double> &paper_lagrange_weights() {
    static const std::vector<double> w = [] {
        std::vector<double> v((size_t)kPhiStep * kPhiTaps);
        for (int r = 0; r < kPhiStep; ++r) {
            const long double t = (long double)r / kPhiStep;
            for (int j = 0; j < kPhiTaps; ++j) {
                long double l = 1.0L;
                for (int i = 0; i < kPhiTaps; ++i)
                    if (i != j) l *= (t - (i - 3)) / (long double)(j - i);
                v[(size_t)r * kPhiTaps + j] = (double)l;
            }
        }
        return v;
    }();
    return w;
}

PaperBufs carve_paper(const PaperModes &pm, bool ccf, char *ws) {
    PaperBufs b{};
    size_t used = 0;
    b.grid_x = take<double2>(ws, used, pm.nf);
    b.grid_y = ccf ? take<double2>(ws, used, pm.nf) : nullptr;
    b.scratch = take<double2>(ws, used, pm.nf);
    b.tw = take<double2>(ws, used, pm.nf);
    b.Fx = take<double2>(ws, used, pm.Mh + 1);
    b.Fy = ccf ? take<double2>(ws, used, pm.Mh + 1) : nullptr;
    b.d_tc = take<double>(ws, used, 1);
    b.d_gx = take<double>(ws, used, pm.nq / 2);
    b.d_gphi = take<double>(ws, used, pm.nq / 2);
    b.invph = take<double>(ws, used, pm.Mh + 1);
    b.coarse = take<double>(ws, used, paper_coarse_count(pm));
    b.lagw = take<double>(ws, used, kPhiStep * kPhiTaps);
    b.used = used + 256;
    return b;
}

// Type-2 evaluation (modes -> lags) of S(tau) = sum_{m=0}^{Mh} A_m exp(-2 pi i m tau / L)
// by the ES kernel: b_m = A_m / phihat_m on the n_f grid, one FFT, and at each lag a
// W-tap interpolation at grid coordinate u = frac(tau / L) n_f, taken from the lag's
// 64-bit phase.  The +i FFT of conj(b) is the conjugate of the -i transform, so its
// real part is Re S directly.  Cost: one FFT plus W taps per lag, whatever K.
__global__ void paper_place_kernel(const double2 *__restrict__ A, const double *__restrict__ invph, int64_t Mh,
                                   int nf, double2 *__restrict__ grid) {
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nf) return;
    double2 v = make_double2(0.0, 0.0);
    if (l <= Mh) {
        const double s = invph[l];
        const double2 a = A[l];
        v = make_double2(a.x * s, -a.y * s);
    }
    grid[l] = v;
}

template <int W, int D>
__global__ void paper_interp_kernel(const double2 *__restrict__ G, int lg, const unsigned long long *__restrict__ phi,
                                    int64_t K, const EsPoly<double, W, D> poly, double *__restrict__ c) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const long long mask = (1ll << lg) - 1;
    const unsigned long long ph = phi[k];
    const long long ui = (long long)(ph >> (64 - lg));                  // integer part of u
    const double uf = (double)((ph << lg) >> 11) * 0x1.0p-53;           // fraction of u
    const int up = uf > 0.0;
    const long long l0 = ui - W / 2 + up;                               // ceil(u - W/2)
    const double v = 2.0 * (up ? 1.0 - uf : 0.0) - 1.0;                 // 2 f0 - 1
    double acc = 0.0;
#pragma unroll
    for (int t = 0; t < W; ++t) {
        const double *cf = poly.c + t * (D + 1);
        double w = cf[D];
#pragma unroll
        for (int d = D - 1; d >= 0; --d) w = fma(w, v, cf[d]);
        acc = fma(G[(l0 + t) & mask].x, w, acc);
    }
    c[k] = acc;
}

}  // namespace

ncf_status paper_modes_plan(double L, double tc, int64_t N1, PaperModes *pm, std::string *msg) {
    PaperModes p;
    p.L = L;
    p.tc = tc;
    p.N1 = N1;
    p.Mh = N1 / 2;
    p.W = 16;
    p.beta = 2.30 * p.W;
    p.nq = 128;
    const int64_t need = 4 * (p.Mh + 1) + p.W;  // oversampling >= 2, as the Gaussian path
    p.lg = 1;
    while ((int64_t(1) << p.lg) < need) ++p.lg;
    if (p.lg > 27) {
        *msg = "N1 = " + std::to_string(N1) + " needs a grid above 2^27 cells";
        return NCF_EUNSUPPORTED;
    }
    p.nf = 1 << p.lg;
    std::vector<double> gw;
    gauss_legendre(p.nq, p.gx, gw);  // nodes in decreasing order: the first nq/2 are positive
    p.gphi.resize(p.nq);
    for (int q = 0; q < p.nq; ++q)
        p.gphi[q] = gw[q] * std::exp(p.beta * (std::sqrt(std::max(0.0, 1.0 - p.gx[q] * p.gx[q])) - 1.0));
    p.poly = es_poly(p.W, p.beta, PolyDeg<16>::D);
    *pm = std::move(p);
    return NCF_OK;
}

size_t paper_modes_bytes(const PaperModes &pm, bool ccf) { return carve_paper(pm, ccf, nullptr).used; }

size_t paper_modes_pinned_bytes(const PaperModes &pm) {
    return al(8) + 2 * al(pm.nq / 2 * 8) + al((size_t)kPhiStep * kPhiTaps * 8);
}

void paper_modes_run(const PaperModes &pm, const SpecSide &x, const SpecSide *y, char *ws, char *pinned,
                     double2 **Fx, double2 **Fy, cudaStream_t st) {
    const bool ccf = y != nullptr;
    PaperBufs bf = carve_paper(pm, ccf, ws);
    size_t off = 0;
    auto up = [&](void *dst, const void *src, size_t bytes) {
        std::memcpy(pinned + off, src, bytes);
        copy_pinned(dst, pinned + off, bytes, st);
        off += al(bytes);
    };
    up(bf.d_tc, &pm.tc, 8);
    up(bf.d_gx, pm.gx.data(), pm.nq / 2 * 8);
    up(bf.d_gphi, pm.gphi.data(), pm.nq / 2 * 8);
    up(bf.lagw, paper_lagrange_weights().data(), (size_t)kPhiStep * kPhiTaps * 8);
    constexpr size_t smem = spread_smem_bytes<double, kPrepChunk>();
    static std::atomic<unsigned long long> attr_done{0};
    once_per_device(attr_done, [&] { return set_smem_limit(spread_kernel<double, 16, kPrepChunk>, smem); });
    EsPoly<double, 16, PolyDeg<16>::D> poly{};
    for (size_t i = 0; i < pm.poly.size(); ++i) poly.c[i] = pm.poly[i];
    const double a_scale = (double)pm.nf / pm.L;
    auto spread = [&](const SpecSide &sd, double2 *grid) {
        cudaMemsetAsync(grid, 0, (size_t)pm.nf * sizeof(double2), st);
        NCF_LAUNCH("spread_kernel", st,
                   spread_kernel<double, 16, kPrepChunk><<<(unsigned)sd.n_chunks, kSpreadThreads, smem, st>>>(
                       sd.t, sd.v, sd.d_offs, sd.d_offs + 1, sd.d_chunk_base, sd.d_cs, sd.d_stats, bf.d_tc,
                       a_scale, pm.nf,
                       poly, 0.0f, grid));
    };
    spread(x, bf.grid_x);
    if (ccf) {
        spread(*y, bf.grid_y);
        NCF_LAUNCH("paper_pack_kernel", st,
                   paper_pack_kernel<<<(unsigned)((pm.nf + 255) / 256), 256, 0, st>>>(bf.grid_x, bf.grid_y,
                                                                                     pm.nf));
    }
    NCF_LAUNCH("twiddle_kernel", st,
               twiddle_kernel<double2><<<twiddle_blocks(pm.nf), 256, 0, st>>>(bf.tw, pm.nf));
    const double2 *G = fft_forward_f64(bf.grid_x, bf.scratch, bf.tw, pm.lg, 1, st);
    const int64_t n_coarse = paper_coarse_count(pm);
    NCF_LAUNCH("paper_phihat_kernel", st,
               paper_phihat_kernel<<<(unsigned)((n_coarse + 127) / 128), 128, 0, st>>>(
                   pm.nf, pm.W, bf.d_gx, bf.d_gphi, pm.nq / 2, n_coarse, bf.coarse));
    NCF_LAUNCH("paper_coef_kernel", st,
               paper_coef_kernel<<<(unsigned)((pm.Mh + 256) / 256), 256, 0, st>>>(
                   G, ccf ? 1 : 0, pm.nf, pm.Mh, pm.W, bf.coarse, bf.lagw, bf.Fx, bf.Fy, bf.invph));
    *Fx = bf.Fx;
    *Fy = bf.Fy;
}

void paper_type2(const PaperModes &pm, bool ccf, char *ws, const double2 *A, const unsigned long long *phi,
                 int64_t K, double *c, cudaStream_t st) {
    PaperBufs bf = carve_paper(pm, ccf, ws);
    NCF_LAUNCH("paper_place_kernel", st,
               paper_place_kernel<<<(unsigned)((pm.nf + 255) / 256), 256, 0, st>>>(A, bf.invph, pm.Mh, pm.nf,
                                                                                 bf.grid_x));
    const double2 *G = fft_forward_f64(bf.grid_x, bf.scratch, bf.tw, pm.lg, 1, st);
    EsPoly<double, 16, PolyDeg<16>::D> poly{};
    for (size_t i = 0; i < pm.poly.size(); ++i) poly.c[i] = pm.poly[i];
    NCF_LAUNCH("paper_interp_kernel", st,
               (paper_interp_kernel<16, PolyDeg<16>::D><<<(unsigned)((K + 127) / 128), 128, 0, st>>>(
                   G, pm.lg, phi, K, poly, c)));
}

// ---------------------------------------------------------------------------
// Per-series grid sizing: a batch whose series need grids of very different
// sizes (spans) is split into buckets of series needing the same grid size;
// each bucket runs the whole path on its own period, grid and lag table.  A
// bucket names its series by index (their points stay where they are: the
// spreading reads each series' own [start, end) range), its statistics are
// gathered from the batch's at every launch, and its results go to the series'
// own output rows.
// ---------------------------------------------------------------------------
struct SpectralBucket {
    std::vector<int64_t> idx;             // series of the batch, ascending
    std::vector<SeriesStats> hsx, hsy;    // their host statistics (planning)
    SpectralPrepared p;                   // the bucket's own plan
    size_t ws_off = 0, pin_off = 0;       // its workspace and staging
    size_t tab_off = 0, tab_pin_off = 0;  // its index tables (device, staging)
    std::vector<char> tab_img;            // host image of the index tables
    int64_t nx_total = 0, nx_max = 0, nx_chunks = 0, ny_total = 0, ny_max = 0, ny_chunks = 0;
};

struct BucketTabs {
    size_t row, xlo, xend, xcb, csx, sx, ylo, yend, ycb, csy, sy, bytes;
};
BucketTabs bucket_tabs(const SpectralBucket &bk, bool ccf) {
    BucketTabs t{};
    size_t u = 0;
    const size_t Bk = bk.idx.size();
    auto take = [&](size_t n) {
        const size_t o = u;
        u += al(n);
        return o;
    };
    t.row = take(Bk * 8);
    t.xlo = take(Bk * 8);
    t.xend = take(Bk * 8);
    t.xcb = take((Bk + 1) * 8);
    t.csx = take((size_t)bk.nx_chunks * 4);
    t.sx = take(Bk * sizeof(SeriesStats));
    if (ccf) {
        t.ylo = take(Bk * 8);
        t.yend = take(Bk * 8);
        t.ycb = take((Bk + 1) * 8);
        t.csy = take((size_t)bk.ny_chunks * 4);
        t.sy = take(Bk * sizeof(SeriesStats));
    }
    t.bytes = u;
    return t;
}

__global__ void gather_stats_kernel(const SeriesStats *__restrict__ src, const int64_t *__restrict__ idx, int64_t n,
                                    SeriesStats *__restrict__ dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[idx[i]];
}

// The bucket's arguments: the batch's points, the bucket's index tables and
// gathered statistics, output rows through the row map.
SpectralArgs bucket_args(const SpectralArgs &a, const SpectralBucket &bk, char *ws, cudaStream_t st) {
    const bool ccf = !a.acf;
    const BucketTabs t = bucket_tabs(bk, ccf);
    char *tb = ws + bk.tab_off;
    const int64_t Bk = (int64_t)bk.idx.size();
    const int64_t *row = reinterpret_cast<const int64_t *>(tb + t.row);
    SeriesStats *sx = reinterpret_cast<SeriesStats *>(tb + t.sx);
    NCF_LAUNCH("gather_stats_kernel", st,
               gather_stats_kernel<<<(unsigned)((Bk + 255) / 256), 256, 0, st>>>(a.x.d_stats, row, Bk, sx));
    SpectralArgs ab = a;
    ab.B = Bk;
    ab.row_map = row;
    ab.no_buckets = true;
    ab.x = {a.x.t, a.x.v, reinterpret_cast<const int64_t *>(tb + t.xlo), sx, nullptr, bk.hsx.data(), bk.nx_total,
            bk.nx_max, reinterpret_cast<const int64_t *>(tb + t.xcb), bk.nx_chunks,
            reinterpret_cast<const int32_t *>(tb + t.csx), reinterpret_cast<const int64_t *>(tb + t.xend)};
    if (ccf) {
        SeriesStats *sy = reinterpret_cast<SeriesStats *>(tb + t.sy);
        NCF_LAUNCH("gather_stats_kernel", st,
                   gather_stats_kernel<<<(unsigned)((Bk + 255) / 256), 256, 0, st>>>(a.y.d_stats, row, Bk, sy));
        ab.y = {a.y.t, a.y.v, reinterpret_cast<const int64_t *>(tb + t.ylo), sy, nullptr, bk.hsy.data(),
                bk.ny_total, bk.ny_max, reinterpret_cast<const int64_t *>(tb + t.ycb), bk.ny_chunks,
                reinterpret_cast<const int32_t *>(tb + t.csy), reinterpret_cast<const int64_t *>(tb + t.yend)};
    }
    return ab;
}

// Buckets by grid size when the per-series grids would hold at most 3/4 of the
// cells of one common grid and the buckets' device memory is no more than one
// grid's (NCF_SPEC_BUCKETS=0 keeps one grid).  Their host staging (each
// bucket's tables) is bounded by spectral_bucket_pinned_allowance.  Returns
// false when the batch keeps one grid.
bool plan_buckets(const SpectralArgs &a, SpectralPrepared &out, size_t *ws_bytes, size_t *pinned_bytes,
                  std::string *msg, ncf_status *rc) {
    *rc = NCF_OK;
    const int64_t B = a.B;
    const bool ccf = !a.acf;
    if (a.no_buckets || B < 2 || !a.x.h_offs || (ccf && !a.y.h_offs)) return false;
    if (const char *e = std::getenv("NCF_SPEC_BUCKETS"))
        if (std::atoi(e) == 0) return false;
    std::vector<int> lgs(B);
    int lg_max = 0;
    for (int64_t b = 0; b < B; ++b) {
        double lo = a.x.h_stats[b].t_first, hi = a.x.h_stats[b].t_last;
        if (ccf) {
            lo = std::min(lo, a.y.h_stats[b].t_first);
            hi = std::max(hi, a.y.h_stats[b].t_last);
        }
        SpectralPrepared q;
        make_plan(a, hi - lo, q);
        lgs[b] = q.lg;
        lg_max = std::max(lg_max, q.lg);
    }
    double cells_sum = 0.0;
    std::vector<int> levels;
    for (int64_t b = 0; b < B; ++b) {
        cells_sum += std::ldexp(1.0, lgs[b]);
        if (std::find(levels.begin(), levels.end(), lgs[b]) == levels.end()) levels.push_back(lgs[b]);
    }
    if (levels.size() < 2 || cells_sum > 0.75 * (double)B * std::ldexp(1.0, lg_max)) return false;
    std::sort(levels.begin(), levels.end());
    size_t ws = 0, pin = 0;
    out.buckets.clear();
    for (int lv : levels) {
        auto bk = std::make_shared<SpectralBucket>();
        for (int64_t b = 0; b < B; ++b)
            if (lgs[b] == lv) bk->idx.push_back(b);
        const int64_t Bk = (int64_t)bk->idx.size();
        for (int64_t j = 0; j < Bk; ++j) {
            bk->hsx.push_back(a.x.h_stats[bk->idx[j]]);
            if (ccf) bk->hsy.push_back(a.y.h_stats[bk->idx[j]]);
        }
        SpectralArgs ak = a;
        ak.B = Bk;
        ak.no_buckets = true;
        ak.x.h_stats = bk->hsx.data();
        if (ccf) ak.y.h_stats = bk->hsy.data();
        size_t wk = 0, pk = 0;
        if ((*rc = spectral_plan(ak, &bk->p, &wk, &pk, msg))) return true;
        bk->ws_off = ws;
        ws += al(wk);
        bk->pin_off = pin;
        pin += al(pk);
        // index tables: row map, [start, end) of each series, chunk tables
        auto side = [&](const int64_t *offs, int64_t &total, int64_t &nmax, int64_t &nchunks,
                        std::vector<int64_t> &lo, std::vector<int64_t> &end, std::vector<int64_t> &cb,
                        std::vector<int32_t> &cs) {
            cb.push_back(0);
            for (int64_t j = 0; j < Bk; ++j) {
                const int64_t b = bk->idx[j], n = offs[b + 1] - offs[b];
                lo.push_back(offs[b]);
                end.push_back(offs[b + 1]);
                total += n;
                nmax = std::max(nmax, n);
                const int64_t c = (n + kPrepChunk - 1) / kPrepChunk;
                for (int64_t q = 0; q < c; ++q) cs.push_back((int32_t)j);
                cb.push_back(cb.back() + c);
            }
            nchunks = cb.back();
        };
        std::vector<int64_t> xlo, xend, xcb, ylo, yend, ycb;
        std::vector<int32_t> csx, csy;
        side(a.x.h_offs, bk->nx_total, bk->nx_max, bk->nx_chunks, xlo, xend, xcb, csx);
        if (ccf) side(a.y.h_offs, bk->ny_total, bk->ny_max, bk->ny_chunks, ylo, yend, ycb, csy);
        const BucketTabs t = bucket_tabs(*bk, ccf);
        bk->tab_img.assign(t.bytes, 0);
        auto put = [&](size_t off, const void *src, size_t bytes) {
            if (bytes) std::memcpy(bk->tab_img.data() + off, src, bytes);
        };
        put(t.row, bk->idx.data(), Bk * 8);
        put(t.xlo, xlo.data(), Bk * 8);
        put(t.xend, xend.data(), Bk * 8);
        put(t.xcb, xcb.data(), (Bk + 1) * 8);
        put(t.csx, csx.data(), csx.size() * 4);
        if (ccf) {
            put(t.ylo, ylo.data(), Bk * 8);
            put(t.yend, yend.data(), Bk * 8);
            put(t.ycb, ycb.data(), (Bk + 1) * 8);
            put(t.csy, csy.data(), csy.size() * 4);
        }
        bk->tab_off = ws;
        ws += al(t.bytes);
        bk->tab_pin_off = pin;
        pin += al(t.bytes);
        out.buckets.push_back(bk);
    }
    // split only where it also needs no more memory than one grid, so that a
    // size-only bound (ncf_workspace_bytes) holds for either plan
    {
        SpectralArgs a1 = a;
        a1.no_buckets = true;
        SpectralPrepared one;
        size_t w1 = 0, p1 = 0;
        if ((*rc = spectral_plan(a1, &one, &w1, &p1, msg))) return true;
        if (ws + 256 > w1) {
            out.buckets.clear();
            return false;
        }
    }
    // the evaluation's geometry fields describe its largest grid
    const SpectralPrepared &big = out.buckets.back()->p;
    auto buckets = std::move(out.buckets);
    out = big;
    out.tc.clear();
    out.phi.clear();
    out.B = B;
    out.direct = false;
    out.buckets = std::move(buckets);
    *ws_bytes = ws + 256;
    *pinned_bytes = pin;
    return true;
}

ncf_status spectral_plan(const SpectralArgs &a, SpectralPrepared *sp, size_t *ws_bytes,
                         size_t *pinned_bytes, std::string *msg) {
    {
        SpectralPrepared bp;
        ncf_status rc = NCF_OK;
        if (plan_buckets(a, bp, ws_bytes, pinned_bytes, msg, &rc)) {
            if (rc) return rc;
            *sp = std::move(bp);
            return NCF_OK;
        }
    }
    const int64_t B = a.B;
    const bool ccf = !a.acf;
    // per-series centre t_c and the common period L (Algorithm 1 with an
    // alias margin: L = max span + max|tau| + R h)
    SpectralPrepared p;
    p.tc.resize(B);
    double max_span = 0.0;
    for (int64_t b = 0; b < B; ++b) {
        double lo = a.x.h_stats[b].t_first, hi = a.x.h_stats[b].t_last;
        if (ccf) {
            lo = std::min(lo, a.y.h_stats[b].t_first);
            hi = std::max(hi, a.y.h_stats[b].t_last);
        }
        p.tc[b] = lo + 0.5 * (hi - lo);
        max_span = std::max(max_span, hi - lo);
    }
    make_plan(a, max_span, p);
    if (p.lg > 28) {
        *msg = "spectral grid would exceed 2^28 cells (span / h too large); use the windowed path";
        return NCF_EUNSUPPORTED;
    }
    // lag phases in 64-bit fixed point; the appended lag K is zero
    p.phi.assign(p.Kp, 0ull);
    for (int64_t k = 0; k < a.K; ++k) {
        double f = a.h_lags[k] / p.L;
        f -= std::floor(f);
        p.phi[k] = (unsigned long long)std::ldexp(f, 64 - 11) << 11;
    }
    std::vector<double> gw;
    gauss_legendre(p.nq, p.gx, gw);
    p.gphi.resize(p.nq);
    for (int q = 0; q < p.nq; ++q)
        p.gphi[q] = gw[q] * std::exp(p.beta * (std::sqrt(std::max(0.0, 1.0 - p.gx[q] * p.gx[q])) - 1.0));
    p.poly = es_poly(p.W, p.beta, p.W == 8 ? PolyDeg<8>::D : PolyDeg<16>::D);
    p.tap_sum = es_tap_sum(p.poly, p.W, p.W == 8 ? PolyDeg<8>::D : PolyDeg<16>::D);
    *ws_bytes = p.fp32 ? carve<float>(p, nullptr).used : carve<double>(p, nullptr).used;
    *pinned_bytes = al(B * 8) + al(p.Kp * 8) + 2 * al(p.nq * 8);
    *sp = std::move(p);
    return NCF_OK;
}

// Host staging a split plan may need beyond one grid's: per bucket (at most
// one per grid size, 2^1 .. 2^28 cells) its lag phases, quadrature tables and
// index tables, each region aligned.
size_t spectral_bucket_pinned_allowance(int64_t B, int64_t K, int64_t n_x, int64_t n_y, bool ccf) {
    const size_t levels = 28;
    const size_t per = al((size_t)(K + 4) * 8) + 2 * al(128 * 8) + 12 * 256;
    auto side = [&](int64_t n) {
        return 3 * al((size_t)B * 8) + al((size_t)(B + 1) * 8) + al((size_t)(n / kPrepChunk + B) * 4) +
               al((size_t)B * sizeof(SeriesStats));
    };
    return levels * per + al((size_t)B * 8) + side(n_x) + (ccf ? side(n_y) : 0);
}

void spectral_prepare(const SpectralPrepared &p, char *ws, char *pinned, cudaStream_t st) {
    if (!p.buckets.empty()) {
        for (const auto &bk : p.buckets) {
            spectral_prepare(bk->p, ws + bk->ws_off, pinned + bk->pin_off, st);
            std::memcpy(pinned + bk->tab_pin_off, bk->tab_img.data(), bk->tab_img.size());
            copy_pinned(ws + bk->tab_off, pinned + bk->tab_pin_off, bk->tab_img.size(), st);
        }
        return;
    }
    if (p.fp32) prepare_typed<float>(p, ws, p.tc.data(), p.phi.data(), p.gx, p.gphi, pinned, st);
    else prepare_typed<double>(p, ws, p.tc.data(), p.phi.data(), p.gx, p.gphi, pinned, st);
}

ncf_status spectral_launch(const SpectralArgs &a, const SpectralPrepared &p, char *ws, int *status,
                           cudaStream_t st, std::string *msg) {
    if (!p.buckets.empty()) {
        for (const auto &bk : p.buckets) {
            const SpectralArgs ab = bucket_args(a, *bk, ws, st);
            bk->p.fft_variant = p.fft_variant;  // the shapes tuned for the evaluation
            bk->p.contract_variant = p.contract_variant;
            bk->p.spread_variant = p.spread_variant;
            ncf_status rc = bk->p.fp32 ? launch_typed<float>(ab, bk->p, ws + bk->ws_off, status, st, msg)
                                       : launch_typed<double>(ab, bk->p, ws + bk->ws_off, status, st, msg);
            if (rc) return rc;
        }
        return NCF_OK;
    }
    if (p.fp32) return launch_typed<float>(a, p, ws, status, st, msg);
    return launch_typed<double>(a, p, ws, status, st, msg);
}

void spectral_guard(const SpectralArgs &a, const SpectralPrepared &p, char *ws, int *status,
                    cudaStream_t st) {
    if (!p.buckets.empty()) {
        for (const auto &bk : p.buckets) spectral_guard(bucket_args(a, *bk, ws, st), bk->p, ws + bk->ws_off, status, st);
        return;
    }
    const double *d_tc = p.fp32 ? carve<float>(p, ws).d_tc : carve<double>(p, ws).d_tc;
    const double max_span = (p.L - p.max_tau - p.R_alias * p.h) * (1.0 + 1e-12);
    NCF_LAUNCH("spectral_guard_kernel", st,
               spectral_guard_kernel<<<(unsigned)((p.B + 127) / 128), 128, 0, st>>>(
                   a.x.d_stats, p.acf ? nullptr : a.y.d_stats, d_tc, p.B, max_span, 0.9 * p.L, status));
}

// FP64 forward transforms (+i sign, unnormalised) of B contiguous grids of
// 2^lg complex values, by the same Stockham passes as the spectral path; the
// result lands in `grid` or `scratch` (returned).  tw must hold
// exp(+2 pi i q / 2^lg), q < 2^lg (fft_twiddles_f64).
void fft_twiddles_f64(double2 *tw, int lg, cudaStream_t st) {
    const int n = 1 << lg;
    NCF_LAUNCH("twiddle_kernel", st, twiddle_kernel<double2><<<twiddle_blocks(n), 256, 0, st>>>(tw, n));
}

double2 *fft_forward_f64(double2 *grid, double2 *scratch, const double2 *tw, int lg, int64_t B, cudaStream_t st) {
    const RadixPlan rp = radix_plan(lg);
    const int n = 1 << lg;
    double2 *in = grid, *out = scratch;
    int Ns = 1;
    for (int q = 0; q < rp.n_pass; ++q) {
        const int rad = rp.radix[q];
        const int64_t items = B * (int64_t)(n / rad);
        const unsigned blocks = (unsigned)((items + 255) / 256);
        if (rad == 8)
            NCF_LAUNCH("fft_pass_kernel", st, fft_pass_kernel<double2, 8><<<blocks, 256, 0, st>>>(in, out, lg, Ns, tw, B));
        else if (rad == 4)
            NCF_LAUNCH("fft_pass_kernel", st, fft_pass_kernel<double2, 4><<<blocks, 256, 0, st>>>(in, out, lg, Ns, tw, B));
        else
            NCF_LAUNCH("fft_pass_kernel", st, fft_pass_kernel<double2, 2><<<blocks, 256, 0, st>>>(in, out, lg, Ns, tw, B));
        Ns *= rad;
        std::swap(in, out);
    }
    return in;
}

}  // namespace ncf
