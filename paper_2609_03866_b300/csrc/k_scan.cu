// k_scan.cu -- real-space scans over sorted times (Appendix "Effective pair
// count algorithms" and "Real-space ACF/CCF algorithms", Algorithms 5-8).
//
// Work decomposition: the outer points s_j of each series are cut into tiles
// of kTileJ consecutive points; a CTA owns one tile and kWarps lags, one lag
// per warp.  Lane l of a warp runs the paper's two-pointer scan over kRunJ
// consecutive outer points: one binary search at the start of the run, then
// the window pointers only advance (the window centre s_j + e*tau grows with
// j).  Each warp reduces its lane sums and adds them to the per-(series, lag)
// accumulators with integer atomics (rectangle: exact and order-independent)
// or FP64 atomics (Gaussian windowed path).
//
// Rectangle (Algorithms 6 and 8).  The predicate fl(c - h) <= t_i <= fl(c + h),
// c = fl(s_j + e*tau), is decided on fixed-point keys T = floor(t * 2^q):
// integer bounds L^ = S_j + e*Tau_k - H and U^ = S_j + e*Tau_k + H differ from
// the scaled FP64 bounds by less than eta key units, so a key more than eta
// away from a bound decides the comparison exactly; keys inside the band are
// re-tested with the FP64 predicate itself.  Counts are therefore bit-exact,
// and the numerator sum_j Y_j (P[hi] - P[lo]) is accumulated exactly in
// 128-bit integers from the quantised standardised values.
#include <cmath>
#include <cstdint>

#include "common.cuh"

namespace ncf {

namespace {

constexpr int kWarps = 8;               // lags per CTA
constexpr int kRunJ = 32;               // consecutive outer points per lane
constexpr int kTileJ = 32 * kRunJ;      // outer points per tile

__device__ __forceinline__ int64_t lower_bound_key(const int64_t *__restrict__ T, int64_t lo,
                                                   int64_t hi, int64_t v) {
    // first index in [lo, hi) with T[i] >= v
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (T[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ double centre(double s, double tau, int eps) {
    return __dadd_rn(s, eps > 0 ? tau : -tau);
}

struct U128 { unsigned long long lo, hi; };

__device__ __forceinline__ void add128(U128 &a, unsigned long long lo, unsigned long long hi) {
    unsigned long long n = a.lo + lo;
    a.hi += hi + (n < a.lo ? 1ull : 0ull);
    a.lo = n;
}

constexpr int kStageCap = 6144;  // staged window keys per CTA (T and P: 96 KB)

// Advance p while key(p) < bound; reads only indices < end, and the caller
// guarantees the answer is <= end.  Sorted keys make the count of
// true predicates among the next four equal to the advance, so the common
// small step needs no data-dependent branch; a long jump (an outer point
// that crosses an observing gap moves its window by hundreds of points)
// gallops: doubling steps, then bisection, O(log jump) loads.
__device__ __forceinline__ int64_t advance(const int64_t *__restrict__ T, int64_t p, int64_t end,
                                           int64_t bound) {
    if (p + 4 <= end) {
        const int s = (T[p] < bound) + (T[p + 1] < bound) + (T[p + 2] < bound) + (T[p + 3] < bound);
        p += s;
        if (s < 4) return p;
        // T[p - 1] < bound: gallop
        int64_t step = 4;
        int64_t lo = p;          // invariant: T[lo - 1] < bound
        int64_t hi = p + step;   // candidate upper end
        while (hi < end && T[hi] < bound) {
            lo = hi + 1;
            step <<= 1;
            hi = lo + step;
        }
        return lower_bound_key(T, lo, min(hi, end), bound);
    }
    while (p < end && T[p] < bound) ++p;
    return p;
}

__global__ void __launch_bounds__(kWarps * 32, 2)
rect_scan_kernel(const int64_t *__restrict__ Tx, const int64_t *__restrict__ P,
                 const double *__restrict__ tx, const int64_t *__restrict__ offs_x,
                 const int64_t *__restrict__ Sy, const int64_t *__restrict__ Yq,
                 const double *__restrict__ sy, const ScanTile *__restrict__ tiles,
                 const double *__restrict__ lags, int64_t K, int eps, double h, int64_t H,
                 double tscale, int64_t eta, unsigned long long *__restrict__ cnt,
                 unsigned long long *__restrict__ num128) {
    extern __shared__ int64_t smem[];
    int64_t *sT = smem, *sP = smem + kStageCap;
    __shared__ int64_t s_lo[kWarps], s_hi[kWarps];
    __shared__ int64_t s_range[2];
    const ScanTile tile = tiles[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t k = (int64_t)blockIdx.y * kWarps + warp;
    const bool active = k < K;
    const double tau = active ? lags[k] : 0.0;
    const int64_t Tau = __double2ll_rd(tau * tscale);
    const int64_t dl = (eps > 0 ? Tau : -Tau) - H;
    const int64_t du = (eps > 0 ? Tau : -Tau) + H;
    const int64_t xa = offs_x[tile.b], xb = offs_x[tile.b + 1];
    // union of the windows of this CTA's lags over its outer points
    if (lane == 0) {
        s_lo[warp] = active ? Sy[tile.j0] + dl - eta : INT64_MAX;
        s_hi[warp] = active ? Sy[tile.j1 - 1] + du + eta : INT64_MIN;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t lo_b = INT64_MAX, hi_b = INT64_MIN;
        for (int w = 0; w < kWarps; ++w) { lo_b = min(lo_b, s_lo[w]); hi_b = max(hi_b, s_hi[w]); }
        const int64_t ia = lower_bound_key(Tx, xa, xb, lo_b);
        const int64_t ib = lower_bound_key(Tx, ia, xb, hi_b);  // last index a pointer can read
        s_range[0] = ia;
        s_range[1] = ib;
    }
    __syncthreads();
    // Every pointer stays <= ib (the first key >= the largest band edge), and
    // the four-wide look-ahead of advance() reads at most three keys past it.
    const int64_t ia = s_range[0], ib = min(s_range[1], xb);
    const int64_t t_last = min(ib + 3, xb - 1);
    const bool staged = (t_last - ia + 1 <= kStageCap) && (ib - ia + 1 <= kStageCap + 1);
    if (staged) {
        for (int64_t i = threadIdx.x; i <= t_last - ia; i += blockDim.x) sT[i] = Tx[ia + i];
        for (int64_t i = threadIdx.x; i <= ib - ia; i += blockDim.x) sP[i] = P[ia + i];
    }
    __syncthreads();
    if (!active) return;
    // every search answer is <= ib, so no read needs an index >= lim
    const int64_t lim = min(ib + 1, xb);
    const int64_t *T = staged ? sT - ia : Tx;
    const int64_t *PP = staged ? sP - ia : P;
    const int64_t j0 = tile.j0 + (int64_t)lane * kRunJ;
    const int64_t j1 = min(j0 + kRunJ, tile.j1);
    unsigned long long c = 0;
    U128 acc{0ull, 0ull};
    if (j0 < j1) {
        int64_t lo = lower_bound_key(T, ia, ib, Sy[j0] + dl - eta);
        int64_t hi = lower_bound_key(T, lo, ib, Sy[j0] + du - eta);
        for (int64_t j = j0; j < j1; ++j) {
            const int64_t S = Sy[j];
            const int64_t Lh = S + dl, Uh = S + du;
            lo = advance(T, lo, lim, Lh - eta);
            if (lo < xb && T[lo] < Lh + eta) {  // inside the band: decide in FP64
                const double lb = __dsub_rn(centre(sy[j], tau, eps), h);
                while (lo < xb && T[lo] < Lh + eta && tx[lo] < lb) ++lo;
            }
            hi = advance(T, max(hi, lo), lim, Uh - eta);
            if (hi < xb && T[hi] < Uh + eta) {
                const double ub = __dadd_rn(centre(sy[j], tau, eps), h);
                while (hi < xb && T[hi] < Uh + eta && tx[hi] <= ub) ++hi;
            }
            c += (unsigned long long)(hi - lo);
            const long long w = (long long)((unsigned long long)PP[hi] - (unsigned long long)PP[lo]);
            const __int128 prod = (__int128)w * (__int128)Yq[j];
            add128(acc, (unsigned long long)prod, (unsigned long long)(prod >> 64));
        }
    }
    for (int o = 16; o; o >>= 1) {
        c += __shfl_down_sync(0xffffffffu, c, o);
        const unsigned long long ol = __shfl_down_sync(0xffffffffu, acc.lo, o);
        const unsigned long long oh = __shfl_down_sync(0xffffffffu, acc.hi, o);
        add128(acc, ol, oh);
    }
    if (lane == 0) {
        const int64_t slot = (int64_t)tile.b * K + k;
        atomicAdd(cnt + slot, c);
        const unsigned long long old = atomicAdd(num128 + 2 * slot, acc.lo);
        const unsigned long long carry = (old + acc.lo < old) ? 1ull : 0ull;
        atomicAdd(num128 + 2 * slot + 1, acc.hi + carry);
    }
}

constexpr double kInvSqrt2Pi = 0.398942280401432677939946059934381868;

__global__ void __launch_bounds__(kWarps * 32)
gauss_window_kernel(const double *__restrict__ tx, const double *__restrict__ x,
                    const int64_t *__restrict__ offs_x, const SeriesStats *__restrict__ stx,
                    const double *__restrict__ sy, const double *__restrict__ y,
                    const SeriesStats *__restrict__ sty, const ScanTile *__restrict__ tiles,
                    const double *__restrict__ lags, int64_t K, int eps, double h, double Rh,
                    double *__restrict__ num, double *__restrict__ den,
                    unsigned long long *__restrict__ cnt) {
    const ScanTile tile = tiles[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t k = (int64_t)blockIdx.y * kWarps + warp;
    if (k >= K) return;
    const double tau = lags[k];
    const int64_t xa = offs_x[tile.b], xb = offs_x[tile.b + 1];
    const double mx = stx[tile.b].mean, ix = stx[tile.b].inv_std;
    const double my = sty[tile.b].mean, iy = sty[tile.b].inv_std;
    const double inv2h2 = 1.0 / (2.0 * h * h);
    const double norm = kInvSqrt2Pi / h;
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
        const double c0 = centre(sy[j0], tau, eps);
        int64_t lo = lb(xa, xb, __dsub_rn(c0, Rh));
        int64_t hi = lb(lo, xb, __dadd_rn(c0, Rh));
        for (int64_t j = j0; j < j1; ++j) {
            const double cj = centre(sy[j], tau, eps);
            const double wl = __dsub_rn(cj, Rh), wu = __dadd_rn(cj, Rh);
            while (lo < xb && tx[lo] < wl) ++lo;
            while (hi < xb && tx[hi] < wu) ++hi;
            const double yj = (y[j] - my) * iy;
            double nj = 0.0, bj = 0.0;
            for (int64_t i = lo; i < hi; ++i) {
                const double d = tx[i] - cj;
                const double w = exp(-d * d * inv2h2);
                bj += w;
                nj = fma(w, (x[i] - mx) * ix, nj);
            }
            Bw += bj;
            N = fma(nj, yj, N);
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
        atomicAdd(num + slot, N * norm);
        atomicAdd(den + slot, Bw * norm);
        atomicAdd(cnt + slot, c);
    }
}

__global__ void finish_rect_kernel(const unsigned long long *__restrict__ cnt,
                                   const unsigned long long *__restrict__ num128, int64_t B,
                                   int64_t K, double inv_v2, const double *__restrict__ scale,
                                   double *__restrict__ c, double *__restrict__ b,
                                   int64_t *__restrict__ count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * K) return;
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
                                    double *__restrict__ c, double *__restrict__ b,
                                    int64_t *__restrict__ count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * K) return;
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
                                       double inv_v2, double *__restrict__ scale) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    auto val = [&](const unsigned long long *c, const unsigned long long *n) {
        const double N = ((double)(long long)n[2 * b + 1] * 18446744073709551616.0 + (double)n[2 * b]) * inv_v2;
        return N / fmax((double)c[b], 1e-16);
    };
    const double sx = val(cx, nx);
    scale[b] = cy ? sqrt(sx * val(cy, ny)) : sx;
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
                            int64_t B, double inv_v2, double *scale, cudaStream_t st) {
    NCF_LAUNCH("lag0_scale_rect_kernel", st,
    lag0_scale_rect_kernel<<<(unsigned)((B + 127) / 128), 128, 0, st>>>(cnt_x, num_x, cnt_y, num_y, B,
                                                                         inv_v2, scale));
}

void launch_lag0_scale_gauss(const double *num_x, const double *den_x, const double *num_y,
                             const double *den_y, int64_t B, double *scale, cudaStream_t st) {
    NCF_LAUNCH("lag0_scale_gauss_kernel", st,
    lag0_scale_gauss_kernel<<<(unsigned)((B + 127) / 128), 128, 0, st>>>(num_x, den_x, num_y, den_y, B,
                                                                          scale));
}

void launch_rect_scan(const int64_t *Tx, const int64_t *P, const double *tx, const int64_t *offs_x,
                      const int64_t *Sy, const int64_t *Yq, const double *sy,
                      const ScanTile *tiles, int64_t n_tiles, const double *lags, int64_t K,
                      int eps, double h, FixedScales fs,
                      unsigned long long *cnt, unsigned long long *num128, cudaStream_t st) {
    const int64_t H = (int64_t)std::floor(h * fs.tscale);
    dim3 grid((unsigned)n_tiles, (unsigned)((K + kWarps - 1) / kWarps));
    const size_t smem = (2 * kStageCap + 1) * sizeof(int64_t);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(rect_scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr_set = true;
    }
    NCF_LAUNCH("rect_scan_kernel", st,
    rect_scan_kernel<<<grid, kWarps * 32, smem, st>>>(Tx, P, tx, offs_x, Sy, Yq, sy, tiles, lags, K, eps,
                                                   h, H, fs.tscale, fs.eta, cnt, num128));
}

void launch_gauss_window(const double *tx, const double *x, const int64_t *offs_x,
                         const SeriesStats *stx, const double *sy, const double *y,
                         const SeriesStats *sty, const ScanTile *tiles, int64_t n_tiles,
                         const double *lags, int64_t K, int eps, double h, double Rh,
                         double *num, double *den, unsigned long long *cnt, cudaStream_t st) {
    dim3 grid((unsigned)n_tiles, (unsigned)((K + kWarps - 1) / kWarps));
    NCF_LAUNCH("gauss_window_kernel", st,
    gauss_window_kernel<<<grid, kWarps * 32, 0, st>>>(tx, x, offs_x, stx, sy, y, sty, tiles, lags, K,
                                                      eps, h, Rh, num, den, cnt));
}

void launch_finish_rect(const unsigned long long *cnt, const unsigned long long *num128,
                        int64_t B, int64_t K, double inv_v2, const double *scale,
                        double *c, double *b, int64_t *count, cudaStream_t st) {
    const int64_t n = B * K;
    NCF_LAUNCH("finish_rect_kernel", st,
    finish_rect_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(cnt, num128, B, K, inv_v2, scale,
                                                                     c, b, count));
}

void launch_finish_gauss(const double *num, const double *den, const unsigned long long *cnt,
                         int64_t B, int64_t K, const double *scale, double *c, double *b,
                         int64_t *count, cudaStream_t st) {
    const int64_t n = B * K;
    NCF_LAUNCH("finish_gauss_kernel", st,
    finish_gauss_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(num, den, cnt, B, K, scale, c,
                                                                      b, count));
}

}  // namespace ncf
