// k_scan.cu -- the Gaussian windowed real-space scan (Algorithms 5 and 7)
// and the normalisation kernels shared with the rectangle scan (k_rect.cu).
//
// Work decomposition: the outer points s_j of each series are cut into tiles
// of kTileJ consecutive points; a CTA owns one tile and kWarps lags, one lag
// per warp.  Lane l of a warp runs the paper's two-pointer scan over kRunJ
// consecutive outer points: one binary search at the start of the run, then
// the window pointers only advance (the window centre s_j + e*tau grows with
// j).  Each warp reduces its lane sums and adds them to the per-(series, lag)
// accumulators with FP64 atomics.  This is the plain FP64 path for the
// Gaussian kernel: one FP64 exponential per pair inside the window
// [c - R h, c + R h), by a table-driven method for non-positive arguments.
#include <cmath>
#include <cstdint>

#include "common.cuh"

namespace ncf {

namespace {

constexpr int kWarps = 8;               // lags per CTA
constexpr int kRunJ = 16;               // consecutive outer points per lane
constexpr int kTileJ = 32 * kRunJ;      // outer points per tile

__device__ __forceinline__ double centre(double s, double tau, int eps) {
    return __dadd_rn(s, eps > 0 ? tau : -tau);
}

constexpr double kInvSqrt2Pi = 0.398942280401432677939946059934381868;

// cos(x) for |x| <= pi/2 (the Hann window's range, x = pi d / 2h) as a polynomial of
// degree 8 in w = x^2: the interpolant of cos(sqrt(w)) at the 9 Chebyshev nodes of
// [0, pi^2/4], coefficients rounded to FP64.  Within 5.4e-17 of cos(x) in exact
// arithmetic, within 2e-16 in FP64 (against the 12 terms of its Taylor series in w).
__device__ __forceinline__ double cos_half_range(double x) {
    const double w = x * x;
    double a = 0x1.9f23c6262c74bp-45;
    a = fma(a, w, -0x1.9350a43729003p-37);
    a = fma(a, w, 0x1.1eecdf3980b2ap-29);
    a = fma(a, w, -0x1.27e4f97932bbcp-22);
    a = fma(a, w, 0x1.a01a01994c340p-16);
    a = fma(a, w, -0x1.6c16c16c09b4ep-10);
    a = fma(a, w, 0x1.55555555553c4p-5);
    a = fma(a, w, -0x1.ffffffffffffbp-2);
    return fma(a, w, 1.0);
}

// exp(z) for z <= 0 by Tang's table-driven method (P. T. P. Tang, ACM TOMS 15(2),
// 1989): z = (256 m + j) ln2/256 + r with |r| <= ln2/512, so exp(z) = 2^m 2^(j/256) e^r.
// r = z - N C in one FMA with C = fl(ln2/256), 9.1e-20 below ln2/256: with
// |N| <= |z| 256/ln2 + 1/2 this shifts r by at most 3.4e-17 |z|, an error of
// e^z |z| 3.4e-17 <= 1.3e-17 in absolute terms, whatever z (the weights only
// enter sums, whose scale is the peak weight 1).  e^r - 1 by its Taylor
// polynomial of degree 4 (remainder below 4e-17); the table 2^(j/256) is filled
// per CTA from exp2, and 2^m is added to the exponent field as an integer.
// 8 FP64 operations; within 1.5 ulp for -1 < z <= 0 and 1.3e-16 absolute for all
// z <= 0 (for a correctly rounded table).
constexpr double kExpInvL = 369.3299304675746;         // 256 / ln 2
constexpr double kExpC = 0x1.62e42fefa39efp-9;        // fl(ln2 / 256)
constexpr int kExpTable = 256;
// Below N = -1021 * 256 (z < -707.7) the weight is returned as 0: above it the
// result and every intermediate stay normal numbers.  The test reads all 64 bits
// of nd: while N >= -2^51, nd = 1.5 2^52 + N exactly and its bit pattern, read as
// an integer, is 0x4338000000000000 + N; any smaller nd (more negative z, down to
// -inf) has a smaller pattern (or a negative one), so the guard holds for every
// z <= 0.  A test on the low word alone would wrap once |N| >= 2^31
// (|z| > 5.8e6, a pair 3400 h from the centre under a wide window).
constexpr long long kExpFloor = 0x4338000000000000ll - 1021ll * kExpTable;
__device__ __forceinline__ double exp_neg(double z, const double *__restrict__ T) {
    const double nd = fma(z, kExpInvL, 0x1.8p52);       // N in the low bits
    if (__double_as_longlong(nd) < kExpFloor) return 0.0;
    const int n = (int)__double2loint(nd);
    const double N = nd - 0x1.8p52;
    const double r = fma(-N, kExpC, z);
    const double p = r * fma(r, fma(r, fma(r, 1.0 / 24.0, 1.0 / 6.0), 0.5), 1.0);
    const double t = T[n & (kExpTable - 1)];
    const double v = fma(t, p, t);                      // in [0.99, 2): a normal number
    return __longlong_as_double((long long)((unsigned long long)__double_as_longlong(v) +
                                            ((unsigned long long)(long long)(n >> 8) << 52)));
}

// kNum = false: the pair sums B alone (PairCount); x, y and num are not read
template <bool kNum>
__global__ void __launch_bounds__(kWarps * 32)
gauss_window_kernel(const double *__restrict__ tx, const double *__restrict__ x,
                    const int64_t *__restrict__ offs_x, const SeriesStats *__restrict__ stx,
                    const double *__restrict__ sy, const double *__restrict__ y,
                    const SeriesStats *__restrict__ sty, const ScanTile *__restrict__ tiles,
                    const double *__restrict__ lags, int64_t K, int eps, double h, double Rh, int hann,
                    double *__restrict__ num, double *__restrict__ den,
                    unsigned long long *__restrict__ cnt) {
    __shared__ double T2[kExpTable];  // 2^(j/256) for exp_neg
    for (int i = threadIdx.x; i < kExpTable; i += blockDim.x) T2[i] = exp2((double)i / kExpTable);
    __syncthreads();
    const ScanTile tile = tiles[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t k = (int64_t)blockIdx.y * kWarps + warp;
    if (k >= K) return;
    const double tau = lags[k];
    const int64_t xa = offs_x[tile.b], xb = offs_x[tile.b + 1];
    const double mx = stx[tile.b].mean, ix = stx[tile.b].inv_std;
    const double my = sty[tile.b].mean, iy = sty[tile.b].inv_std;
    const double inv2h2 = 1.0 / (2.0 * h * h);
    const double pi2h = 3.141592653589793 * (0.5 / h);  // Hann: the argument pi d / 2h in one product
    const double norm = hann ? 1.0 / h : kInvSqrt2Pi / h;
    const int64_t j0 = tile.j0 + (int64_t)lane * kRunJ;
    const int64_t j1 = min(j0 + kRunJ, tile.j1);
    double N = 0.0, Bw = 0.0;
    unsigned long long c = 0;
    if (j0 < j1) {
        // first index with t >= v, by bisection on the FP64 times
        auto lb = [&](int64_t lo, int64_t hi, double v) {
            while (lo < hi) {
                int64_t mid = lo + ((hi - lo) >> 1);
                if (tx[mid] < v) lo = mid + 1; else hi = mid;
            }
            return lo;
        };
        // first index with t > v
        auto ub = [&](int64_t lo, int64_t hi, double v) {
            while (lo < hi) {
                int64_t mid = lo + ((hi - lo) >> 1);
                if (tx[mid] <= v) lo = mid + 1; else hi = mid;
            }
            return lo;
        };
        // Gaussian: half-open [c - Rh, c + Rh); Hann: the rectangle's closed [c - h, c + h]
        const double c0 = centre(sy[j0], tau, eps);
        int64_t lo = lb(xa, xb, __dsub_rn(c0, Rh));
        int64_t hi = hann ? ub(lo, xb, __dadd_rn(c0, Rh)) : lb(lo, xb, __dadd_rn(c0, Rh));
        for (int64_t j = j0; j < j1; ++j) {
            const double cj = centre(sy[j], tau, eps);
            const double wl = __dsub_rn(cj, Rh), wu = __dadd_rn(cj, Rh);
            while (lo < xb && tx[lo] < wl) ++lo;
            if (hann)
                while (hi < xb && tx[hi] <= wu) ++hi;
            else
                while (hi < xb && tx[hi] < wu) ++hi;
            // sum_i w_i (x_i - m_x); the factor 1 / sigma_x is applied once per outer point
            double nj = 0.0, bj = 0.0;
            for (int64_t i = lo; i < hi; ++i) {
                const double d = tx[i] - cj;
                double w;
                if (hann) {
                    const double cw = cos_half_range(d * pi2h);
                    w = cw * cw;
                } else {
                    w = exp_neg(-d * d * inv2h2, T2);
                }
                bj += w;
                if constexpr (kNum) nj = fma(w, x[i] - mx, nj);
            }
            Bw += bj;
            if constexpr (kNum) N = fma(nj * ix, (y[j] - my) * iy, N);
            c += (unsigned long long)(hi > lo ? hi - lo : 0);
        }
    }
    for (int o = 16; o; o >>= 1) {
        N += __shfl_down_sync(0xffffffffu, N, o);
        Bw += __shfl_down_sync(0xffffffffu, Bw, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    if (lane == 0) {
        const int64_t slot = (int64_t)tile.b * K + k;
        if constexpr (kNum) atomicAdd(num + slot, N * norm);
        atomicAdd(den + slot, Bw * norm);
        atomicAdd(cnt + slot, c);
    }
}

__device__ __forceinline__ bool failed_write(const int *status, int64_t i, double *c, double *b,
                                             int64_t *count) {
    if (!status || *status == 0) return false;  // a device check failed: no valid result
    c[i] = __longlong_as_double(0x7ff8000000000000ll);
    if (b) b[i] = c[i];
    if (count) count[i] = -1;
    return true;
}

__global__ void finish_rect_kernel(const unsigned long long *__restrict__ cnt,
                                   const unsigned long long *__restrict__ num128, int64_t B,
                                   int64_t K, ValueBits vb, const double *__restrict__ scale,
                                   const int *__restrict__ status, double *__restrict__ c,
                                   double *__restrict__ b, int64_t *__restrict__ count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * K) return;
    if (failed_write(status, i, c, b, count)) return;
    const int64_t sb = i / K;
    const double inv_v2 = ldexp(1.0, -(vb.px(sb) + vb.py(sb)));
    const unsigned long long n = cnt[i];
    const double N = ((double)(long long)num128[2 * i + 1] * 18446744073709551616.0 +
                      (double)num128[2 * i]) * inv_v2;
    const double Bd = (double)n;
    double ci = N / fmax(Bd, 1e-16);
    if (scale) ci /= scale[i / K];
    c[i] = ci;
    if (b) b[i] = Bd;
    if (count) count[i] = (int64_t)n;
}

__global__ void finish_gauss_kernel(const double *__restrict__ num, const double *__restrict__ den,
                                    const unsigned long long *__restrict__ cnt, int64_t B,
                                    int64_t K, const double *__restrict__ scale,
                                    const int *__restrict__ status, double *__restrict__ c,
                                    double *__restrict__ b, int64_t *__restrict__ count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * K) return;
    if (failed_write(status, i, c, b, count)) return;
    double ci = num[i] / fmax(den[i], 1e-16);
    if (scale) ci /= scale[i / K];
    c[i] = ci;
    if (b) b[i] = den[i];
    if (count) count[i] = cnt ? (int64_t)cnt[i] : 0;
}

__global__ void lag0_scale_rect_kernel(const unsigned long long *__restrict__ cx,
                                       const unsigned long long *__restrict__ nx,
                                       const unsigned long long *__restrict__ cy,
                                       const unsigned long long *__restrict__ ny, int64_t B,
                                       ValueBits vb, double *__restrict__ scale) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    // the lag-0 ACF of side x is in units of 2^(2 px), of side y in 2^(2 py)
    auto val = [&](const unsigned long long *c, const unsigned long long *n, int p) {
        const double N = ((double)(long long)n[2 * b + 1] * 18446744073709551616.0 + (double)n[2 * b]) *
                         ldexp(1.0, -2 * p);
        return N / fmax((double)c[b], 1e-16);
    };
    const double sx = val(cx, nx, vb.px(b));
    scale[b] = cy ? sqrt(sx * val(cy, ny, vb.py(b))) : sx;
}

__global__ void lag0_scale_gauss_kernel(const double *__restrict__ nx, const double *__restrict__ dx,
                                        const double *__restrict__ ny, const double *__restrict__ dy,
                                        int64_t B, double *__restrict__ scale) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const double sx = nx[b] / fmax(dx[b], 1e-16);
    scale[b] = ny ? sqrt(sx * (ny[b] / fmax(dy[b], 1e-16))) : sx;
}

}  // namespace

int scan_tile_points() { return kTileJ; }

void launch_lag0_scale_rect(const unsigned long long *cnt_x, const unsigned long long *num_x,
                            const unsigned long long *cnt_y, const unsigned long long *num_y,
                            int64_t B, ValueBits vb, double *scale, cudaStream_t st) {
    NCF_LAUNCH("lag0_scale_rect_kernel", st,
    lag0_scale_rect_kernel<<<(unsigned)((B + 127) / 128), 128, 0, st>>>(cnt_x, num_x, cnt_y, num_y, B,
                                                                         vb, scale));
}

void launch_lag0_scale_gauss(const double *num_x, const double *den_x, const double *num_y,
                             const double *den_y, int64_t B, double *scale, cudaStream_t st) {
    NCF_LAUNCH("lag0_scale_gauss_kernel", st,
    lag0_scale_gauss_kernel<<<(unsigned)((B + 127) / 128), 128, 0, st>>>(num_x, den_x, num_y, den_y, B,
                                                                          scale));
}

void launch_gauss_window(const double *tx, const double *x, const int64_t *offs_x,
                         const SeriesStats *stx, const double *sy, const double *y,
                         const SeriesStats *sty, const ScanTile *tiles, int64_t n_tiles,
                         const double *lags, int64_t K, int eps, double h, double Rh, int hann,
                         double *num, double *den, unsigned long long *cnt, cudaStream_t st) {
    dim3 grid((unsigned)n_tiles, (unsigned)((K + kWarps - 1) / kWarps));
    if (x)
        NCF_LAUNCH("gauss_window_kernel", st,
        gauss_window_kernel<true><<<grid, kWarps * 32, 0, st>>>(tx, x, offs_x, stx, sy, y, sty, tiles, lags, K,
                                                                eps, h, Rh, hann, num, den, cnt));
    else
        NCF_LAUNCH("gauss_window_kernel", st,
        gauss_window_kernel<false><<<grid, kWarps * 32, 0, st>>>(tx, x, offs_x, stx, sy, y, sty, tiles, lags, K,
                                                                 eps, h, Rh, hann, num, den, cnt));
}

void launch_finish_rect(const unsigned long long *cnt, const unsigned long long *num128,
                        int64_t B, int64_t K, ValueBits vb, const double *scale, const int *status,
                        double *c, double *b, int64_t *count, cudaStream_t st) {
    const int64_t n = B * K;
    NCF_LAUNCH("finish_rect_kernel", st,
    finish_rect_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(cnt, num128, B, K, vb, scale, status,
                                                                     c, b, count));
}

void launch_finish_gauss(const double *num, const double *den, const unsigned long long *cnt,
                         int64_t B, int64_t K, const double *scale, const int *status, double *c,
                         double *b, int64_t *count, cudaStream_t st) {
    const int64_t n = B * K;
    NCF_LAUNCH("finish_gauss_kernel", st,
    finish_gauss_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(num, den, cnt, B, K, scale, status, c,
                                                                      b, count));
}

}  // namespace ncf
