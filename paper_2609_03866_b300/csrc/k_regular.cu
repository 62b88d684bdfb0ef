// k_regular.cu -- the classic-FFT estimator for data on a regular grid.
//
// When every time is a whole multiple of one step, t_i = m_i dt (m_i integer,
// non-decreasing), a pair's separation is a whole number d of steps, so the
// kernel-weighted sums of Eq. kernel_estimator collapse onto the lattice:
//     N(tau) = sum_d R(d) b(d dt - tau),   B(tau) = sum_d C(d) b(d dt - tau),
// with R(d) = sum over pairs at separation d of x_std,i y_std,j (the raw
// correlation) and C(d) = the number of such pairs (the correlation of the
// sampling masks -- the "raw-pair ramp" n - |d| when there are no gaps).  The
// paper's dedicated FFT path (Table 1, Sec. 5.2) obtains both with plain FFTs,
// at a cost independent of K; here:
//   1. statistics and validation of each series (one CTA per series);
//   2. x_std + i * mask (ACF), or x_std + i * y_std and mask_x + i * mask_y
//      (CCF), added onto zero-padded grids of 2^lg >= span + reach + 1 cells
//      (no circular wrap reaches a lag that is read);
//   3. forward FFTs; Hermitian unpack to the spectrum
//      W_m = conj(A_m) B_m + i conj(MA_m) MB_m, whose transform is
//      2^lg (R(-d) + i C(-d)) with both parts real;
//   4. one more forward FFT, then per lag the weighted sum over the lattice
//      separations within the kernel's reach (h for the rectangle and the Hann
//      window, 8 h for the Gaussian, whose tail beyond is 1.3e-14 of the peak).
// Pair counts C(d) come out of FP64 FFTs within far less than 1/2 of an
// integer and are rounded, so rectangle counts are exact.  A rectangle pair
// counts when |fl(d dt - tau)| <= h in FP64 (the lattice separation itself,
// not the difference of two rounded times).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "spectral.cuh"

namespace ncf {
namespace {

constexpr int kRegThreads = 256;
constexpr double kRegPi = 3.141592653589793238462643383279502884;

struct RegStats {
    int64_t m_first, m_last;
    double mean, inv_std;
    int32_t flags, pad;
};

// One CTA: FP64 mean and variance (two passes, ddof 0), the lattice range, and
// the validation flags (indices non-decreasing, values finite, spread > 0).
__global__ void __launch_bounds__(kRegThreads)
reg_stats_kernel(const int64_t *__restrict__ m, const double *__restrict__ v, int64_t n, RegStats *__restrict__ out) {
    __shared__ double red[kRegThreads];
    __shared__ int flg[kRegThreads];
    const int tid = threadIdx.x;
    double s = 0.0;
    int f = 0;
    for (int64_t i = tid; i < n; i += blockDim.x) {
        const double x = v[i];
        if (!isfinite(x)) f |= STAT_NONFINITE;
        if (i > 0 && m[i] < m[i - 1]) f |= STAT_UNSORTED;
        s += x;
    }
    red[tid] = s;
    flg[tid] = f;
    __syncthreads();
    for (int o = kRegThreads / 2; o > 0; o >>= 1) {
        if (tid < o) {
            red[tid] += red[tid + o];
            flg[tid] |= flg[tid + o];
        }
        __syncthreads();
    }
    const double mean = red[0] / (double)n;
    const int flags = flg[0];
    __syncthreads();
    double q = 0.0;
    for (int64_t i = tid; i < n; i += blockDim.x) {
        const double d = v[i] - mean;
        q += d * d;
    }
    red[tid] = q;
    __syncthreads();
    for (int o = kRegThreads / 2; o > 0; o >>= 1) {
        if (tid < o) red[tid] += red[tid + o];
        __syncthreads();
    }
    if (tid == 0) {
        const double var = red[0] / (double)n;
        RegStats r;
        r.m_first = m[0];
        r.m_last = m[n - 1];
        r.mean = mean;
        r.inv_std = var > 0.0 ? 1.0 / sqrt(var) : 0.0;
        r.flags = flags | ((var > 0.0 && isfinite(var)) ? 0 : STAT_DEGENERATE);
        r.pad = 0;
        *out = r;
    }
}

// Adds the standardised value of point i to vals[2 (m_i - m0)] and 1 to
// mask[2 (m_i - m0)] (each optional): pointers to the real or the imaginary
// parts of interleaved complex grids.
__global__ void reg_scatter_kernel(const int64_t *__restrict__ m, const double *__restrict__ v, int64_t n,
                                   const RegStats *__restrict__ st, int64_t m0, double *__restrict__ vals,
                                   double *__restrict__ mask) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t l = m[i] - m0;
    if (vals) atomicAdd(vals + 2 * l, (v[i] - st->mean) * st->inv_std);
    if (mask) atomicAdd(mask + 2 * l, 1.0);
}

// split the transform Z of a + i b (a, b real) into A_m and B_m
__device__ __forceinline__ void reg_unpack(const double2 *Z, int64_t m, int64_t N, double2 &A, double2 &B) {
    const double2 p = Z[m], q = Z[(N - m) & (N - 1)];
    A = make_double2(0.5 * (p.x + q.x), 0.5 * (p.y - q.y));
    B = make_double2(0.5 * (p.y + q.y), 0.5 * (q.x - p.x));
}

// ACF: W = |X|^2 + i |M|^2 from Z = FFT(x_std + i mask).
// CCF: W = conj(X) Y + i conj(MX) MY from Z1 = FFT(x_std + i y_std), Z2 = FFT(mask_x + i mask_y).
__global__ void reg_spectrum_kernel(const double2 *__restrict__ Z1, const double2 *__restrict__ Z2, int64_t N,
                                    double2 *__restrict__ W) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    double2 a, b;
    reg_unpack(Z1, m, N, a, b);
    if (!Z2) {  // a = X, b = mask spectrum
        W[m] = make_double2(a.x * a.x + a.y * a.y, b.x * b.x + b.y * b.y);
        return;
    }
    double2 ma, mb;
    reg_unpack(Z2, m, N, ma, mb);
    // conj(a) b and conj(ma) mb are Hermitian in m: their transforms are real
    const double2 num = make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
    const double2 den = make_double2(ma.x * mb.x + ma.y * mb.y, ma.x * mb.y - ma.y * mb.x);
    W[m] = make_double2(num.x - den.y, num.y + den.x);
}

// Per lag: N = sum_d R(d) b(d dt - tau), B = sum_d C(d) b(d dt - tau) over the
// separations within the kernel's reach.  T = FFT(W) holds N_grid (R(-d) + i C(-d)).
// kern: 0 Gaussian (reach 8 h), 1 rectangle, 2 Hann window (reach h, closed).
__global__ void reg_lag_kernel(const double2 *__restrict__ T, int64_t N, const double *__restrict__ lags, int64_t K,
                               double dt, int kern, double h, double reach, double *__restrict__ num,
                               double *__restrict__ den, int64_t *__restrict__ cnt) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const double tau = lags[k];
    const int64_t d0 = (int64_t)ceil((tau - reach) / dt) - 1, d1 = (int64_t)floor((tau + reach) / dt) + 1;
    const double invN = 1.0 / (double)N;
    const double gnorm = 1.0 / (sqrt(2.0 * kRegPi) * h);
    double sn = 0.0, sd = 0.0;
    long long sc = 0;
    for (int64_t d = d0; d <= d1; ++d) {
        const double u = __dsub_rn(__dmul_rn((double)d, dt), tau);
        double wgt;
        if (kern == 1) {
            if (!(fabs(u) <= h)) continue;
            wgt = 1.0;
        } else if (kern == 2) {
            if (!(fabs(u) <= h)) continue;
            const double cw = cospi(0.5 * u / h);
            wgt = cw * cw / h;
        } else {
            if (!(fabs(u) <= reach)) continue;
            wgt = gnorm * exp(-0.5 * (u / h) * (u / h));
        }
        const double2 v = T[(-d) & (N - 1)];
        const double R = v.x * invN;
        const long long C = llrint(v.y * invN);
        sn += R * wgt;
        sd += (double)C * wgt;
        sc += C;
    }
    num[k] = sn;
    den[k] = sd;
    if (cnt) cnt[k] = kern != 0 ? sc : 0;
}

__global__ void reg_finish_kernel(const double *__restrict__ num, const double *__restrict__ den, int64_t K,
                                  const double *__restrict__ scale, double *__restrict__ c, double *__restrict__ b) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    double ci = num[k] / fmax(den[k], 1e-16);
    if (scale) ci /= *scale;
    c[k] = ci;
    if (b) b[k] = den[k];
}

// scale = c_xx(0) (one pipeline), or sqrt(c_xx(0) c_yy(0)) from two lag-0 results
__global__ void reg_scale_kernel(const double *__restrict__ n0, const double *__restrict__ d0, int two,
                                 double *__restrict__ scale) {
    const double sx = n0[0] / fmax(d0[0], 1e-16);
    if (!two) {
        *scale = sx;
        return;
    }
    const double sy = n0[1] / fmax(d0[1], 1e-16);
    *scale = sqrt(sx * sy);
}

size_t al(size_t b) { return (b + 255) & ~size_t(255); }

struct RegLayout {
    size_t grid, tw, num, den, misc, total;
};
RegLayout reg_layout(int lg, bool ccf, int64_t K) {
    RegLayout L;
    const size_t g = al(((size_t)1 << lg) * sizeof(double2));
    L.grid = 0;
    L.tw = g * (ccf ? 3 : 2);
    L.num = L.tw + g;
    L.den = L.num + al((K + 2) * 8);
    L.misc = L.den + al((K + 2) * 8);
    L.total = L.misc + 256;
    return L;
}

}  // namespace

size_t regular_stats_bytes() { return 2 * sizeof(RegStats); }

// The lattice size 2^lg for a span of cells and the lags' reach (0 if over 2^29).
int regular_lg(int64_t span, double max_tau, double reach, double dt) {
    const double cells = (double)span + std::ceil((max_tau + reach) / dt) + 3.0;
    int lg = 3;
    while ((double)((int64_t)1 << lg) < cells && lg < 29) ++lg;
    return (double)((int64_t)1 << lg) < cells ? 0 : lg;
}

size_t regular_workspace_bytes(int lg, bool ccf, int64_t K) { return reg_layout(lg, ccf, K).total; }

// Statistics and validation of one ACF (my == nullptr) or CCF into stat_buf
// (device, regular_stats_bytes()), read back through `pinned` (one host
// synchronisation); returns the lattice range.
ncf_status regular_stats(const int64_t *mx, const double *x, int64_t nx, const int64_t *my, const double *y,
                         int64_t ny, char *stat_buf, char *pinned, int64_t *m0, int64_t *m1, cudaStream_t st,
                         std::string *msg) {
    const bool ccf = my != nullptr;
    RegStats *dst = reinterpret_cast<RegStats *>(stat_buf);
    NCF_LAUNCH("reg_stats_kernel", st, reg_stats_kernel<<<1, kRegThreads, 0, st>>>(mx, x, nx, dst));
    if (ccf) NCF_LAUNCH("reg_stats_kernel", st, reg_stats_kernel<<<1, kRegThreads, 0, st>>>(my, y, ny, dst + 1));
    if (cudaMemcpyAsync(pinned, dst, sizeof(RegStats) * (ccf ? 2 : 1), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        *msg = "regular path: statistics read-back failed";
        return NCF_ECUDA;
    }
    RegStats hs[2];
    std::memcpy(hs, pinned, sizeof(RegStats) * (ccf ? 2 : 1));
    for (int q = 0; q < (ccf ? 2 : 1); ++q) {
        if (hs[q].flags & STAT_NONFINITE) { *msg = "non-finite value"; return NCF_ENONFINITE; }
        if (hs[q].flags & STAT_UNSORTED) { *msg = "lattice indices must be non-decreasing"; return NCF_ENOTSORTED; }
        if (hs[q].flags & STAT_DEGENERATE) { *msg = "zero variance"; return NCF_EDEGENERATE; }
    }
    *m0 = ccf ? std::min(hs[0].m_first, hs[1].m_first) : hs[0].m_first;
    *m1 = ccf ? std::max(hs[0].m_last, hs[1].m_last) : hs[0].m_last;
    return NCF_OK;
}

// The FFT pipeline and the lag sums, on a workspace of regular_workspace_bytes(lg, ccf, K).
ncf_status regular_launch(const int64_t *mx, const double *x, int64_t nx, const int64_t *my, const double *y,
                          int64_t ny, const char *stat_buf, int64_t m0, int lg, double dt, const double *lags,
                          int64_t K, int kernel, double h, int lag0, char *ws, double *c_out, double *b_out,
                          int64_t *count_out, cudaStream_t st, std::string *msg) {
    const bool ccf = my != nullptr;
    const int kern = kernel == NCF_RECTANGLE ? 1 : (kernel == NCF_HANNING ? 2 : 0);
    const double reach = kern == 0 ? 8.0 * h : h;
    const RegStats *dst = reinterpret_cast<const RegStats *>(stat_buf);
    const RegLayout Lo = reg_layout(lg, ccf, K);
    const int64_t N = (int64_t)1 << lg;
    const size_t gb = al((size_t)N * sizeof(double2));
    double2 *G[3] = {reinterpret_cast<double2 *>(ws), reinterpret_cast<double2 *>(ws + gb),
                     ccf ? reinterpret_cast<double2 *>(ws + 2 * gb) : nullptr};
    double2 *tw = reinterpret_cast<double2 *>(ws + Lo.tw);
    double *num = reinterpret_cast<double *>(ws + Lo.num);
    double *den = reinterpret_cast<double *>(ws + Lo.den);
    double *misc = reinterpret_cast<double *>(ws + Lo.misc);  // [0] zero lag, [1] Pearson scale
    fft_twiddles_f64(tw, lg, st);
    const unsigned nbk = (unsigned)((N + 255) / 256);
    auto blocks = [](int64_t n) { return (unsigned)((n + 255) / 256); };
    auto re = [](double2 *g) { return reinterpret_cast<double *>(g); };
    auto im = [](double2 *g) { return reinterpret_cast<double *>(g) + 1; };

    // grids -> spectrum -> T = FFT(W); an ACF of one series when mb == nullptr
    auto pipeline = [&](const int64_t *ma, const double *va, int64_t na, const RegStats *sa, const int64_t *mb,
                        const double *vb, int64_t nb, const RegStats *sb) -> double2 * {
        if (!mb) {
            cudaMemsetAsync(G[0], 0, (size_t)N * sizeof(double2), st);
            NCF_LAUNCH("reg_scatter_kernel", st,
                       reg_scatter_kernel<<<blocks(na), 256, 0, st>>>(ma, va, na, sa, m0, re(G[0]), im(G[0])));
            double2 *Z = fft_forward_f64(G[0], G[1], tw, lg, 1, st);
            double2 *Wb = Z == G[0] ? G[1] : G[0];
            NCF_LAUNCH("reg_spectrum_kernel", st, reg_spectrum_kernel<<<nbk, 256, 0, st>>>(Z, nullptr, N, Wb));
            return fft_forward_f64(Wb, Z, tw, lg, 1, st);
        }
        cudaMemsetAsync(G[0], 0, (size_t)N * sizeof(double2), st);
        cudaMemsetAsync(G[1], 0, (size_t)N * sizeof(double2), st);
        NCF_LAUNCH("reg_scatter_kernel", st,
                   reg_scatter_kernel<<<blocks(na), 256, 0, st>>>(ma, va, na, sa, m0, re(G[0]), re(G[1])));
        NCF_LAUNCH("reg_scatter_kernel", st,
                   reg_scatter_kernel<<<blocks(nb), 256, 0, st>>>(mb, vb, nb, sb, m0, im(G[0]), im(G[1])));
        double2 *Z1 = fft_forward_f64(G[0], G[2], tw, lg, 1, st);
        double2 *free1 = Z1 == G[0] ? G[2] : G[0];
        double2 *Z2 = fft_forward_f64(G[1], free1, tw, lg, 1, st);
        double2 *Wb = Z2 == G[1] ? free1 : G[1];
        NCF_LAUNCH("reg_spectrum_kernel", st, reg_spectrum_kernel<<<nbk, 256, 0, st>>>(Z1, Z2, N, Wb));
        return fft_forward_f64(Wb, Z1, tw, lg, 1, st);
    };
    double *scale = nullptr;
    if (lag0) {
        // Pearson scale from the lag-0 auto-correlations (Algorithms 4 and 10)
        cudaMemsetAsync(misc, 0, 8, st);
        double2 *Tx = pipeline(mx, x, nx, dst, nullptr, nullptr, 0, nullptr);
        NCF_LAUNCH("reg_lag_kernel", st,
                   reg_lag_kernel<<<1, 32, 0, st>>>(Tx, N, misc, 1, dt, kern, h, reach, num + K, den + K, nullptr));
        if (ccf) {
            double2 *Ty = pipeline(my, y, ny, dst + 1, nullptr, nullptr, 0, nullptr);
            NCF_LAUNCH("reg_lag_kernel", st, reg_lag_kernel<<<1, 32, 0, st>>>(Ty, N, misc, 1, dt, kern, h, reach,
                                                                              num + K + 1, den + K + 1, nullptr));
        }
        scale = misc + 1;
        NCF_LAUNCH("reg_scale_kernel", st, reg_scale_kernel<<<1, 1, 0, st>>>(num + K, den + K, ccf ? 1 : 0, scale));
    }
    double2 *T = pipeline(mx, x, nx, dst, my, y, ny, ccf ? dst + 1 : nullptr);
    const unsigned kb = blocks(K);
    NCF_LAUNCH("reg_lag_kernel", st,
               reg_lag_kernel<<<kb, 256, 0, st>>>(T, N, lags, K, dt, kern, h, reach, num, den, count_out));
    NCF_LAUNCH("reg_finish_kernel", st, reg_finish_kernel<<<kb, 256, 0, st>>>(num, den, K, scale, c_out, b_out));
    if (cudaGetLastError() != cudaSuccess) {
        *msg = "regular path: kernel launch failed";
        return NCF_ECUDA;
    }
    return NCF_OK;
}

}  // namespace ncf
