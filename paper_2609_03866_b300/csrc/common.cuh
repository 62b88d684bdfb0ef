// common.cuh -- internal declarations shared by the libncf translation units.
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>

#include "ncf.h"

namespace ncf {

// Points per CTA of the chunked statistics / keys / prefix passes.
constexpr int kPrepChunk = 4096;

// Per-series statistics read back by the host after the statistics pass.
struct SeriesStats {
    double mean;      // mean of the values
    double inv_std;   // 1 / population std (ddof 0); 0 when the variance is not positive
    double t_first;   // first (smallest) time
    double t_last;    // last (largest) time
    int64_t n;        // number of points
    int32_t flags;    // STAT_* bits
    int32_t pad;
};
enum : int32_t { STAT_UNSORTED = 1, STAT_NONFINITE = 2, STAT_DEGENERATE = 4 };

// Bits of the device status word of an evaluation (reported by ncf_plan_status).
enum : int32_t {
    STATUS_TIMEOUT = 1,  // a bounded device-side wait gave up
    STATUS_DOMAIN = 2,   // a series no longer fits the plan's periodic domain
    STATUS_RANGE = 4,    // times beyond the plan's fixed-point key range
    STATUS_INPUT = 8     // unsorted, non-finite or zero-variance input
};

// Partial sums of one chunk of one series (statistics pass).
struct ChunkPartial {
    double s1, s2;    // sum of (x - x_ref), sum of (x - x_ref)^2
    int32_t flags;
    int32_t pad;
};

// Fixed-point scales of the exact rectangle scan.
//   time keys:  T = floor(t * 2^q)               (monotone in t; one q per call)
//   values:     X = round(x_std * 2^p)           (exact integer prefix sums; p per
//                                                  series side, value_bits below)
struct FixedScales {
    double tscale;    // 2^q
    int64_t eta;      // half-width of the ambiguity band of a window bound, key units
    int32_t q, pad;
};

// Value bits p of a series side of n points: p = 61 - ceil(1.5 ceil(log2 n)),
// clamped to [8, 40], so that p <= 61 - 1.5 log2 n bounds the quantised values
// (|x_std| <= sqrt(n)) and their window sums as the scan's 128-bit sums assume.
// Integer arithmetic only: host and device agree, and a series' quantisation
// depends on its own length alone, not on the other series of its batch.
__host__ __device__ inline int value_bits(int64_t n) {
    const unsigned long long m = (unsigned long long)(n > 2 ? n - 1 : 1);
#ifdef __CUDA_ARCH__
    const int L = 64 - __clzll((long long)m);
#else
    const int L = 64 - __builtin_clzll(m);
#endif
    const int p = 61 - (3 * L + 1) / 2;
    return p < 8 ? 8 : (p > 40 ? 40 : p);
}
// The value bits of side x (and y) of series b: its own point count, or n_force
// (> 0) for a shard standardised with a whole series' pooled statistics.
struct ValueBits {
    const int64_t *offs_x = nullptr, *offs_y = nullptr;  // offs_y NULL: an ACF (y = x)
    int64_t nfx = 0, nfy = 0;
#ifdef __CUDACC__
    __device__ int px(int64_t b) const { return value_bits(nfx > 0 ? nfx : offs_x[b + 1] - offs_x[b]); }
    __device__ int py(int64_t b) const {
        return offs_y ? value_bits(nfy > 0 ? nfy : offs_y[b + 1] - offs_y[b]) : px(b);
    }
#endif
};

// Stream-ordered bump allocator over the context workspace.
struct Arena {
    char *base = nullptr;
    size_t cap = 0, used = 0;
    template <class T> T *take(size_t count) {
        size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
        if (used + bytes > cap) return nullptr;
        T *p = reinterpret_cast<T *>(base + used);
        used += bytes;
        return p;
    }
};

// ---- statistics and keys (k_prep.cu) ----
// Chunked statistics: one CTA per chunk of `chunk` points; chunk_base[b] is
// the first chunk of series b (host-computed, B+1 entries on the device) and
// cs[g] the series of chunk g (launch_chunk_series fills it).
void launch_chunk_series(const int64_t *chunk_base, int64_t B, int32_t *cs, cudaStream_t st);
void launch_stats_chunks(const double *t, const double *x, const int64_t *offs,
                         const int64_t *chunk_base, const int32_t *cs, int64_t n_chunks, int chunk,
                         ChunkPartial *part, cudaStream_t st);
void launch_stats_finish(const double *t, const double *x, const int64_t *offs,
                         const int64_t *chunk_base, int64_t B, const ChunkPartial *part,
                         SeriesStats *stats, cudaStream_t st);
// Plan guards: set STATUS_INPUT if any series' statistics carry a flag, and
// STATUS_RANGE if a time magnitude exceeds t_abs (the key scale's bound).
void launch_stats_guard(const SeriesStats *sx, const SeriesStats *sy, int64_t B, int *status,
                        cudaStream_t st);
void launch_keys_guard(const SeriesStats *sx, const SeriesStats *sy, int64_t B, double t_abs, int *status,
                       cudaStream_t st);
// Fixed-point keys and the exclusive prefix sum of the quantised standardised values.
// Writes Tk[total], Xq[total] and P[total + 1].
// Side values quantised with value_bits of their series (n_force > 0: of n_force points).
void launch_keys_prefix(const double *t, const double *x, const int64_t *offs,
                        const int64_t *chunk_base, const int32_t *cs, int64_t n_chunks, int chunk,
                        const SeriesStats *stats, FixedScales fs, int64_t n_force, int64_t *Tk, int64_t *Xq,
                        int64_t *P, int64_t *chunk_sums, int64_t n_total, cudaStream_t st);

// ---- real-space scans (k_scan.cu) ----
struct ScanTile { int32_t b; int32_t pad; int64_t j0, j1; };
// Exact rectangle pair counts and fixed-point numerators (Algorithms 6 and 8),
// k_rect.cu.  Window side x (keys Tx, prefix sums P, times tx), outer side
// (keys Sy, quantised values Yq, times sy); cnt / num128 are indexed
// [series][lag] in the caller's lag order and must be zeroed.
struct RectArgs {
    const int64_t *Tx, *P;
    const double *tx;
    const int64_t *offs_x;
    const int64_t *Sy, *Yq;
    const double *sy;
    const std::vector<int64_t> *outer_offs;  // host CSR offsets of the outer side
    int64_t B, K;
    const double *h_lags;                    // host copy of the lags
    int eps;
    double h;
    FixedScales fs;
    unsigned long long *cnt, *num128;
};
// Device tables of one rectangle scan (tiles, sorted lags, lag groups).
struct RectPrepared {
    int variant = 1;  // lags on lanes with runs of 16 / 32 / 64 outer points (0-2), points on lanes (3); autotuned
    int64_t n_tiles = 0, G = 0;
    void *tiles = nullptr, *ranges = nullptr;
    double *slags = nullptr;
    int64_t *dls = nullptr, *dus = nullptr, *gmin = nullptr, *gmax = nullptr;
    int32_t *perm = nullptr;
};
constexpr int kRectVariants = 4;
int rect_tile_points();
int64_t rect_tiles_of(const std::vector<int64_t> &offs, int64_t B);
size_t rect_workspace_bytes(int64_t n_tiles, int64_t K);
size_t rect_staging_bytes(int64_t n_tiles, int64_t K);
ncf_status rect_prepare(const RectArgs &a, char *ws, size_t ws_cap, char *pinned, size_t pinned_cap,
                        cudaStream_t st, RectPrepared *out, std::string *msg);
ncf_status rect_launch(const RectArgs &a, const RectPrepared &r, cudaStream_t st, std::string *msg);
// Windowed FP64 scan (Algorithms 5 and 7): Gaussian over [c - Rh, c + Rh), or
// (hann) the Hann window cos^2(pi d / 2h) / h over the closed [c - h, c + h].
// x == nullptr: the pair sums (den, cnt) alone, PairCount of Algorithm 5; num untouched.
void launch_gauss_window(const double *tx, const double *x, const int64_t *offs_x,
                         const SeriesStats *stx, const double *sy, const double *y,
                         const SeriesStats *sty, const ScanTile *tiles, int64_t n_tiles,
                         const double *lags, int64_t K, int eps, double h, double Rh, int hann,
                         double *num, double *den, unsigned long long *cnt, cudaStream_t st);
// Bootstrap replicates (k_boot.cu): n_boot resamples with replacement of the n
// points (t, x), each in time order, written to bt, bx [n_boot][n]; cnt is
// scratch of n * n_boot int32.  Draw j of replicate r is SplitMix64 output
// 2^32 r + j of the stream `seed`, reduced to an index by multiply-high.
void launch_bootstrap(const double *t, const double *x, int64_t n, int64_t n_boot, uint64_t seed, int32_t *cnt,
                      double *bt, double *bx, int sm_count, cudaStream_t st);
// Classic-FFT estimator on a regular lattice t = m dt (k_regular.cu).
size_t regular_stats_bytes();
int regular_lg(int64_t span, double max_tau, double reach, double dt);
size_t regular_workspace_bytes(int lg, bool ccf, int64_t K);
ncf_status regular_stats(const int64_t *mx, const double *x, int64_t nx, const int64_t *my, const double *y,
                         int64_t ny, char *stat_buf, char *pinned, int64_t *m0, int64_t *m1, cudaStream_t st,
                         std::string *msg);
ncf_status regular_launch(const int64_t *mx, const double *x, int64_t nx, const int64_t *my, const double *y,
                          int64_t ny, const char *stat_buf, int64_t m0, int lg, double dt, const double *lags,
                          int64_t K, int kernel, double h, int lag0, char *ws, double *c_out, double *b_out,
                          int64_t *count_out, cudaStream_t st, std::string *msg);
// Outer points per scan tile.
int scan_tile_points();
// Pearson scale per series from lag-0 ACF accumulators of x (and y for a CCF):
// scale = c_xx(0) or sqrt(c_xx(0) * c_yy(0)) (Algorithms 4 and 10).
void launch_lag0_scale_rect(const unsigned long long *cnt_x, const unsigned long long *num_x,
                            const unsigned long long *cnt_y, const unsigned long long *num_y,
                            int64_t B, ValueBits vb, double *scale, cudaStream_t st);
void launch_lag0_scale_gauss(const double *num_x, const double *den_x, const double *num_y,
                             const double *den_y, int64_t B, double *scale, cudaStream_t st);
// Small staging copies between device memory and a context's pinned host
// buffer (allocated device-mapped), done by a kernel instead of a copy engine:
// a kernel's loads and stores do not queue behind bulk copies that other
// streams have put on the copy engines (a concurrent upload of a whole batch
// would otherwise hold up every statistics read-back and table upload).  dst
// and src 8-byte aligned; stream-ordered like cudaMemcpyAsync.
void copy_pinned(void *dst, const void *src, size_t bytes, cudaStream_t st);
// c = N / max(B, 1e-16) from the scan accumulators; optional lag-0 scaling.
// status (nullable): a nonzero status word turns every result into NaN
// (count -1): a device-side check of an executed plan failed.
// N in units of 2^(px + py) of series b (ValueBits).
void launch_finish_rect(const unsigned long long *cnt, const unsigned long long *num128,
                        int64_t B, int64_t K, ValueBits vb, const double *scale, const int *status,
                        double *c, double *b, int64_t *count, cudaStream_t st);
void launch_finish_gauss(const double *num, const double *den, const unsigned long long *cnt,
                         int64_t B, int64_t K, const double *scale, const int *status, double *c,
                         double *b, int64_t *count, cudaStream_t st);


#ifdef __CUDACC__
// v as an unevaluated sum hi + lo of two floats (about 48 significant bits),
// from the bit pattern when the exponent allows, else by conversion.  The
// conversion path is out of line: inlined, the compiler predicates it into the
// common path, and its FP64 conversions then occupy the (slow) FP64 pipe for
// every value.
static __device__ __noinline__ float2 split_df_slow(double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}
__device__ __forceinline__ void split_df(double v, float &hi, float &lo) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((u >> 52) & 0x7FF);
    if (e >= 949 && e <= 1150) {
        const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
        const unsigned long long m = u & 0xFFFFFFFFFFFFFull;
        hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | (unsigned)(m >> 29));
        const float scale = __uint_as_float((unsigned)(e - 948) << 23);  // 2^(e - 1075)
        const float r = (float)(unsigned)(m & 0x1FFFFFFFull) * scale;
        lo = sign ? -r : r;
    } else {
        const float2 f = split_df_slow(v);
        hi = f.x;
        lo = f.y;
    }
}
#endif

}  // namespace ncf

namespace ncf {
// Runs set() once per device for one call site: kernel attributes such as the
// dynamic shared-memory limit belong to a device, and call sites are reached from
// several threads (the server's slots).  Two threads may both run set() the first
// time; it only repeats the same idempotent settings.  set() returns whether every
// setting took; a device is marked done only then, so a failed setting is tried
// again on the next call (and the launch after it reports the error).
template <typename F>
inline void once_per_device(std::atomic<unsigned long long> &done, F &&set) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        set();
        return;
    }
    const unsigned long long bit = 1ull << dev;
    if (done.load(std::memory_order_acquire) & bit) return;
    if (set()) done.fetch_or(bit, std::memory_order_release);
}
// the dynamic shared-memory limit of one kernel; true when it took
template <typename K>
inline bool set_smem_limit(K *kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess;
}
}  // namespace ncf

// Launch bookkeeping: every kernel launch in the library goes through
// NCF_LAUNCH, which counts it, marks it as an NVTX range named for the kernel
// and, when the context's profiler is on, brackets it with CUDA events
// recorded on the launch stream.
namespace ncf {
struct LaunchMark {
    LaunchMark(const char *name, cudaStream_t st);
    ~LaunchMark();
    int slot;
    cudaStream_t st;
};
}  // namespace ncf
#define NCF_LAUNCH(name, st, ...)              \
    do {                                       \
        ::ncf::LaunchMark ncf_mark_(name, st); \
        __VA_ARGS__;                           \
    } while (0)
