// api.cu -- the C ABI of libncf (include/ncf.h): contexts, validation,
// planning and dispatch of the stream-ordered kernels.
//
// Call flow of ncf_corr_batch (see the header for the contract):
//   1. host-side argument checks (pointers, sizes, enums, CSR offsets);
//   2. upload of the small host tables (offsets, chunk and tile lists) through
//      a pinned staging buffer, statistics kernels on every series, one
//      synchronisation to read back per-series statistics and the lags;
//   3. data checks (sorted, finite, positive variance) -> status codes;
//   4. the evaluation path: exact rectangle scan, Gaussian windowed scan, or
//      the spectral (NUFFT) path, then normalisation, all on `stream`.
#include <algorithm>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>

#include <nvtx3/nvToolsExt.h>  // header-only; each launch is a named range for a tracing tool
#include <vector>

#include "common.cuh"
#include "spectral.cuh"

#include <map>
#include <mutex>

// Per-context kernel profiler: CUDA events around every launch while enabled.
struct NcfProfiler {
    bool on = false;
    std::vector<cudaEvent_t> pool;                 // begin/end pairs, reused after a report
    size_t next = 0;
    std::vector<std::pair<const char *, size_t>> recs;  // kernel name, index of its begin event
    std::map<std::string, std::pair<int64_t, double>> totals;  // name -> (launches, ms)
};

struct ncf_ctx {
    int device = 0;
    int sm_count = 0;
    char *ws = nullptr;          // pre-statistics workspace
    size_t ws_cap = 0;
    char *ws2 = nullptr;         // post-statistics workspace (sized from the data)
    size_t ws2_cap = 0;
    char *pinned = nullptr;      // host staging for uploads and read-backs
    size_t pinned_cap = 0;
    // host-buffer calls: the next chunk's statistics stage runs on a stream of its
    // own beside the current chunk's evaluation, with a second pre-statistics
    // workspace (chunks alternate between ws and ws_alt) and its own staging
    char *ws_alt = nullptr;
    size_t ws_alt_cap = 0;
    char *pinned_pre = nullptr;
    size_t pinned_pre_cap = 0;
    cudaStream_t prep_st = nullptr;
    char *hbuf = nullptr;        // device copies of host inputs (ncf_corr_batch_host)
    size_t hbuf_cap = 0;
    char *boot = nullptr;        // bootstrap replicates and their multiplicities
    size_t boot_cap = 0;
    char *paper = nullptr;       // the paper's NUFFT variant (ncf_corr_paper)
    size_t paper_cap = 0;
    uint64_t launches = 0;
    size_t dev_hwm = 0;          // largest device footprint of the workspaces so far
    cudaEvent_t staged = nullptr;  // recorded after staging copies issued past the read-back sync
    cudaStream_t copy_st = nullptr;  // host-buffer calls: uploads beside the compute stream
    cudaStream_t back_st = nullptr;  // and read-backs, on a stream of their own
    std::vector<cudaEvent_t> copy_ev;
    NcfProfiler prof;
    ncf_plan_info plan{0.0, 0, 0, 0, 0, 0, 0};
    ncf_tuning tuning{-1, -1, -1, -1};
    std::string err;
};

static thread_local ncf_ctx *tls_ctx = nullptr;

namespace ncf {
LaunchMark::LaunchMark(const char *name, cudaStream_t s) : slot(-1), st(s) {
    nvtxRangePushA(name);  // no-op unless a tracing tool is attached
    ncf_ctx *c = tls_ctx;
    if (!c) return;
    ++c->launches;
    NcfProfiler &p = c->prof;
    if (!p.on) return;
    if (p.next + 2 > p.pool.size()) {
        for (int q = 0; q < 64; ++q) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return;
            p.pool.push_back(e);
        }
    }
    slot = (int)p.next;
    p.next += 2;
    cudaEventRecord(p.pool[slot], st);
    p.recs.emplace_back(name, (size_t)slot);
}
LaunchMark::~LaunchMark() {
    if (slot >= 0 && tls_ctx) cudaEventRecord(tls_ctx->prof.pool[slot + 1], st);
    nvtxRangePop();
}
}  // namespace ncf

namespace ncf {
namespace {

struct LaunchScope {
    ncf_ctx *prev;
    explicit LaunchScope(ncf_ctx *c) : prev(tls_ctx) { tls_ctx = c; }
    ~LaunchScope() { tls_ctx = prev; }
};

ncf_status fail(ncf_ctx *ctx, ncf_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    return s;
}

#define NCF_CUDA(call)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(ctx, NCF_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// device bytes the context holds now (its workspaces only grow)
size_t ctx_device_bytes(const ncf_ctx *ctx) {
    return ctx->ws_cap + ctx->ws_alt_cap + ctx->ws2_cap + ctx->hbuf_cap + ctx->boot_cap + ctx->paper_cap;
}

ncf_status grow(ncf_ctx *ctx, char **buf, size_t *cap, size_t need, cudaStream_t st) {
    if (need <= *cap) return NCF_OK;
    size_t ncap = std::max(need, *cap + *cap / 2);
    if (*buf) {
        NCF_CUDA(cudaStreamSynchronize(st));
        NCF_CUDA(cudaFree(*buf));
        *buf = nullptr;
        *cap = 0;
    }
    if (cudaMalloc(buf, ncap) != cudaSuccess) {
        cudaGetLastError();
        *buf = nullptr;
        return fail(ctx, NCF_ENOMEM, "cudaMalloc of %zu bytes failed", ncap);
    }
    *cap = ncap;
    ctx->dev_hwm = std::max(ctx->dev_hwm, ctx_device_bytes(ctx));
    return NCF_OK;
}

ncf_status grow_pinned_buf(ncf_ctx *ctx, char **buf, size_t *cap, size_t need, cudaStream_t st) {
    if (need <= *cap) return NCF_OK;
    size_t ncap = std::max(need, *cap * 2);
    if (*buf) {
        NCF_CUDA(cudaStreamSynchronize(st));
        NCF_CUDA(cudaFreeHost(*buf));
        *buf = nullptr;
        *cap = 0;
    }
    // device-mapped: small staging copies are done by a kernel (copy_pinned)
    if (cudaHostAlloc(buf, ncap, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
        cudaGetLastError();
        *buf = nullptr;
        return fail(ctx, NCF_ENOMEM, "cudaHostAlloc of %zu bytes failed", ncap);
    }
    *cap = ncap;
    return NCF_OK;
}
ncf_status grow_pinned(ncf_ctx *ctx, size_t need, cudaStream_t st) {
    return grow_pinned_buf(ctx, &ctx->pinned, &ctx->pinned_cap, need, st);
}

size_t al(size_t b) { return (b + 255) & ~size_t(255); }

// One side (x or y) of a batch: device arrays plus host-side chunking.
struct Side {
    const double *t = nullptr, *v = nullptr;
    std::vector<int64_t> offs, chunk_base;
    int64_t n_total = 0, n_chunks = 0, n_max = 0;
    int64_t rect_tiles = 0, scan_tiles = 0;  // outer tiles of the rectangle and windowed scans
    // device
    int64_t *d_offs = nullptr, *d_chunk_base = nullptr;
    int32_t *d_cs = nullptr;  // series of each chunk
    ChunkPartial *d_part = nullptr;
    SeriesStats *d_stats = nullptr;
    std::vector<SeriesStats> stats;
};

void plan_side(Side &sd, const int64_t *offs, int64_t B) {
    sd.offs.assign(offs, offs + B + 1);
    sd.chunk_base.resize(B + 1);
    int64_t c = 0;
    sd.n_max = 0;
    for (int64_t b = 0; b < B; ++b) {
        sd.chunk_base[b] = c;
        const int64_t n = offs[b + 1] - offs[b];
        sd.n_max = std::max(sd.n_max, n);
        c += (n + kPrepChunk - 1) / kPrepChunk;
    }
    sd.chunk_base[B] = c;
    sd.n_chunks = c;
    sd.n_total = offs[B];
    sd.rect_tiles = rect_tiles_of(sd.offs, B);
    const int64_t tj = scan_tile_points();
    sd.scan_tiles = 0;
    for (int64_t b = 0; b < B; ++b) sd.scan_tiles += (offs[b + 1] - offs[b] + tj - 1) / tj;
}

// The largest sum over series of ceil(n_b / chunk) for any split of n points
// into B series: n / chunk + B (chunk - 1) / chunk, rounded down.
int64_t chunks_bound(int64_t n, int64_t B, int64_t chunk) { return (n + B * (chunk - 1)) / chunk; }

// Host-side counts of a side described only by its size: every count that the
// workspace depends on takes its largest value over the splits of n points into
// B series (each of at least 2 points).
void bound_side(Side &sd, int64_t n, int64_t B) {
    sd.n_total = n;
    sd.n_max = n - 2 * (B - 1);
    sd.n_chunks = chunks_bound(n, B, kPrepChunk);
    sd.rect_tiles = chunks_bound(n, B, rect_tile_points());
    sd.scan_tiles = chunks_bound(n, B, scan_tile_points());
}

std::vector<ScanTile> make_tiles(const std::vector<int64_t> &offs, int64_t B, int tileJ) {
    std::vector<ScanTile> tiles;
    for (int64_t b = 0; b < B; ++b)
        for (int64_t j = offs[b]; j < offs[b + 1]; j += tileJ)
            tiles.push_back(ScanTile{(int32_t)b, 0, j, std::min(j + tileJ, offs[b + 1])});
    return tiles;
}

ncf_status check_offsets(ncf_ctx *ctx, const int64_t *offs, int64_t B, const char *name) {
    if (!offs) return fail(ctx, NCF_EINVAL, "%s is NULL", name);
    if (offs[0] != 0) return fail(ctx, NCF_EINVAL, "%s[0] must be 0", name);
    for (int64_t b = 0; b < B; ++b)
        if (offs[b + 1] - offs[b] < 2)
            return fail(ctx, NCF_EINVAL, "series %lld of %s has %lld points (need >= 2)", (long long)b,
                        name, (long long)(offs[b + 1] - offs[b]));
    return NCF_OK;
}

ncf_status check_stats(ncf_ctx *ctx, const Side &sd, int64_t B, const char *name) {
    for (int64_t b = 0; b < B; ++b) {
        const int f = sd.stats[b].flags;
        if (f & STAT_NONFINITE)
            return fail(ctx, NCF_ENONFINITE, "series %lld of %s holds a NaN or infinite time or value",
                        (long long)b, name);
        if (f & STAT_UNSORTED)
            return fail(ctx, NCF_ENOTSORTED, "times of series %lld of %s decrease", (long long)b, name);
        if (f & STAT_DEGENERATE)
            return fail(ctx, NCF_EDEGENERATE, "series %lld of %s has zero variance", (long long)b, name);
    }
    return NCF_OK;
}

// Time-key scale of a rectangle scan from the largest |time| it compares (the
// value bits are per series side: value_bits in common.cuh).
FixedScales choose_scales(double m_abs) {
    FixedScales fs{};
    int e = 0;
    std::frexp(std::max(m_abs, 1e-300), &e);  // m_abs < 2^e
    fs.q = std::max(-1000, std::min(1000, 60 - e));
    fs.tscale = std::ldexp(1.0, fs.q);
    // two FP64 roundings of magnitude <= m_abs, plus three floor() truncations
    fs.eta = 4 + (int64_t)std::ldexp(1.0, e - 52 + fs.q);
    return fs;
}

// ----------------------------------------------------------------------------
// One evaluation (a batch, a lag set, options): host analysis, device tables
// and work buffers.  One-shot calls build it in the context's workspace and
// launch it once; an ncf_plan owns its memory and launches it many times.
// ----------------------------------------------------------------------------
struct Eval {
    bool acf = true, lag0 = false;
    int64_t B = 0, K = 0;
    ncf_options opt{};
    int path = NCF_PATH_AUTO;
    bool den_only = false;  // windowed path: the pair sums alone (PairCount), no numerator
    const ncf_pooled_stats *pooled = nullptr;  // statistics pooled over a series' shards (ncf_corr_pooled)
    Side X, Y;
    std::vector<double> lagv;
    double max_tau = 0.0, t_abs = 0.0;
    const double *d_lags = nullptr;  // device lags used by the windowed path
    int *status = nullptr;           // device status word (plans: guard / bounded waits)
    // rectangle
    FixedScales fs{};
    RectPrepared r_main, r_x, r_y;
    int64_t *kxT = nullptr, *kxX = nullptr, *kxP = nullptr, *kxC = nullptr;
    int64_t *kyT = nullptr, *kyX = nullptr, *kyP = nullptr, *kyC = nullptr;
    unsigned long long *cnt = nullptr, *num = nullptr, *cnt0 = nullptr, *num0 = nullptr;
    double *scale = nullptr, *zero_lag = nullptr;
    // Gaussian windowed
    ScanTile *g_tiles = nullptr, *g_xtiles = nullptr;
    int64_t g_ntiles = 0, g_nxtiles = 0;
    double *gnum = nullptr, *gden = nullptr, *gn0 = nullptr, *gd0 = nullptr;
    unsigned long long *gcnt = nullptr, *gc0 = nullptr;
    // spectral
    SpectralPrepared sp;
    char *spec_ws = nullptr;
    Side &outer() { return acf ? X : Y; }
};

// Options, sizes and the path they select (AUTO resolved where the options alone
// decide it; the FP64 Gaussian stays AUTO until the statistics are known).
ncf_status check_options(ncf_ctx *ctx, const ncf_options *opt, int64_t B, int64_t K, int *path_out) {
    if (!opt) return fail(ctx, NCF_EINVAL, "options are NULL");
    if (B < 1) return fail(ctx, NCF_EINVAL, "B = %lld (need >= 1)", (long long)B);
    if (K < 1) return fail(ctx, NCF_EINVAL, "K = %lld (need >= 1)", (long long)K);
    if (!(opt->h > 0.0) || !std::isfinite(opt->h))
        return fail(ctx, NCF_EINVAL, "h = %g (need finite h > 0)", opt->h);
    if (opt->kernel != NCF_GAUSSIAN && opt->kernel != NCF_RECTANGLE && opt->kernel != NCF_HANNING)
        return fail(ctx, NCF_EINVAL, "unknown kernel %d", opt->kernel);
    if (opt->path < NCF_PATH_AUTO || opt->path > NCF_PATH_WINDOWED)
        return fail(ctx, NCF_EINVAL, "unknown path %d", opt->path);
    if (opt->precision != NCF_FP64 && opt->precision != NCF_FP32)
        return fail(ctx, NCF_EINVAL, "unknown precision %d", opt->precision);
    if (opt->norm != NCF_NORM_NONE && opt->norm != NCF_NORM_LAG0)
        return fail(ctx, NCF_EINVAL, "unknown normalisation %d", opt->norm);
    if (!(opt->trunc_R >= 0.0) || !(opt->tol >= 0.0) || opt->tol >= 1.0)
        return fail(ctx, NCF_EINVAL, "trunc_R must be >= 0 and tol in [0, 1)");
    int path = opt->path;
    if (opt->kernel == NCF_GAUSSIAN && path == NCF_PATH_WINDOWED && opt->precision == NCF_FP32)
        return fail(ctx, NCF_EUNSUPPORTED, "the windowed Gaussian path is FP64 only");
    if (opt->kernel == NCF_HANNING && (path == NCF_PATH_SPECTRAL || opt->precision == NCF_FP32))
        return fail(ctx, NCF_EUNSUPPORTED,
                    "Hanning kernel: FP64 windowed path only (its transform decays as 1/f^3)");
    if (path == NCF_PATH_AUTO) {
        if (opt->kernel == NCF_RECTANGLE || opt->kernel == NCF_HANNING) path = NCF_PATH_WINDOWED;
        else if (opt->precision == NCF_FP32) path = NCF_PATH_SPECTRAL;
        // FP64 Gaussian: decided after the statistics pass (choose_path)
    }
    *path_out = path;
    return NCF_OK;
}

ncf_status check_args(ncf_ctx *ctx, const int64_t *offs_x, const double *t, const double *x,
                      const int64_t *offs_y, const double *s, const double *y, int64_t B,
                      const double *lags, int64_t K, const ncf_options *opt, Eval &ev) {
    int path = 0;
    ncf_status rc = check_options(ctx, opt, B, K, &path);
    if (rc) return rc;
    if (!t || !x || !lags) return fail(ctx, NCF_EINVAL, "NULL t, x or lags");
    const bool acf = (s == nullptr && y == nullptr);
    if (!acf && (!s || !y || !offs_y)) return fail(ctx, NCF_EINVAL, "CCF needs s, y and offs_y");
    if ((rc = check_offsets(ctx, offs_x, B, "offs_x"))) return rc;
    if (!acf && (rc = check_offsets(ctx, offs_y, B, "offs_y"))) return rc;
    ev.acf = acf;
    ev.B = B;
    ev.K = K;
    ev.opt = *opt;
    ev.path = path;
    ev.lag0 = opt->norm == NCF_NORM_LAG0;
    plan_side(ev.X, offs_x, B);
    if (!acf) plan_side(ev.Y, offs_y, B);
    return NCF_OK;
}

// The rectangle runs on the exact scan unless the spectral-sinc variant was asked for.
bool rect_scan(const Eval &ev) { return ev.opt.kernel == NCF_RECTANGLE && ev.path != NCF_PATH_SPECTRAL; }

size_t pre_bytes(const Eval &ev) {
    auto side = [&](const Side &sd) {
        return al((ev.B + 1) * 8) * 2 + al(sd.n_chunks * sizeof(ChunkPartial)) +
               al(ev.B * sizeof(SeriesStats)) + al(sd.n_chunks * 4);
    };
    return side(ev.X) + (ev.acf ? 0 : side(ev.Y)) + al(4) + al(8) + 1024;
}

void carve_pre(Eval &ev, char *mem) {
    Arena ar{mem, SIZE_MAX, 0};
    auto carve = [&](Side &sd) {
        sd.d_offs = ar.take<int64_t>(ev.B + 1);
        sd.d_chunk_base = ar.take<int64_t>(ev.B + 1);
        sd.d_part = ar.take<ChunkPartial>(sd.n_chunks);
        sd.d_stats = ar.take<SeriesStats>(ev.B);
        sd.d_cs = ar.take<int32_t>(sd.n_chunks);
    };
    carve(ev.X);
    if (!ev.acf) carve(ev.Y);
    ev.status = ar.take<int>(1);
    ev.zero_lag = ar.take<double>(1);
}

void run_stats(Eval &ev, cudaStream_t st) {
    auto one = [&](Side &sd) {
        launch_stats_chunks(sd.t, sd.v, sd.d_offs, sd.d_chunk_base, sd.d_cs, sd.n_chunks, kPrepChunk,
                            sd.d_part, st);
        launch_stats_finish(sd.t, sd.v, sd.d_offs, sd.d_chunk_base, ev.B, sd.d_part, sd.d_stats, st);
    };
    one(ev.X);
    if (!ev.acf) one(ev.Y);
}

// Uploads the CSR tables, runs the statistics pass and reads back the
// per-series statistics and the lags (the one host synchronisation).
// `pre_staging`: stage through the context's second pinned buffer, not the one the
// evaluations' preparation uses (a statistics stage that runs beside another
// chunk's evaluation).
ncf_status analyze(ncf_ctx *ctx, Eval &ev, const double *lags, cudaStream_t st, bool pre_staging = false) {
    const int64_t B = ev.B, K = ev.K;
    ncf_status rc;
    const size_t up_bytes = al((B + 1) * 8) * 4;
    const size_t down_bytes = al(B * sizeof(SeriesStats)) * 2 + al(K * 8);
    char **pin = pre_staging ? &ctx->pinned_pre : &ctx->pinned;
    size_t *pin_cap = pre_staging ? &ctx->pinned_pre_cap : &ctx->pinned_cap;
    if ((rc = grow_pinned_buf(ctx, pin, pin_cap, up_bytes + down_bytes, st))) return rc;
    char *hp = *pin;
    auto upload = [&](void *dst, const void *src, size_t bytes) -> ncf_status {
        std::memcpy(hp, src, bytes);
        copy_pinned(dst, hp, bytes, st);
        hp += al(bytes);
        return NCF_OK;
    };
    if ((rc = upload(ev.X.d_offs, ev.X.offs.data(), (B + 1) * 8))) return rc;
    if ((rc = upload(ev.X.d_chunk_base, ev.X.chunk_base.data(), (B + 1) * 8))) return rc;
    if (!ev.acf) {
        if ((rc = upload(ev.Y.d_offs, ev.Y.offs.data(), (B + 1) * 8))) return rc;
        if ((rc = upload(ev.Y.d_chunk_base, ev.Y.chunk_base.data(), (B + 1) * 8))) return rc;
    }
    launch_chunk_series(ev.X.d_chunk_base, B, ev.X.d_cs, st);
    if (!ev.acf) launch_chunk_series(ev.Y.d_chunk_base, B, ev.Y.d_cs, st);
    run_stats(ev, st);
    char *down = *pin + up_bytes;
    copy_pinned(down, ev.X.d_stats, B * sizeof(SeriesStats), st);
    if (!ev.acf) copy_pinned(down + al(B * sizeof(SeriesStats)), ev.Y.d_stats, B * sizeof(SeriesStats), st);
    double *h_lags = reinterpret_cast<double *>(down + 2 * al(B * sizeof(SeriesStats)));
    copy_pinned(h_lags, lags, K * 8, st);
    NCF_CUDA(cudaStreamSynchronize(st));
    NCF_CUDA(cudaGetLastError());
    auto *hs = reinterpret_cast<SeriesStats *>(down);
    ev.X.stats.assign(hs, hs + B);
    if (!ev.acf) {
        auto *hy = reinterpret_cast<SeriesStats *>(down + al(B * sizeof(SeriesStats)));
        ev.Y.stats.assign(hy, hy + B);
    }
    if (ev.pooled) {
        // standardise with the statistics pooled over the shards; this shard's own
        // pass still validates order and finiteness (a shard may be constant)
        auto patch = [&](Side &sd, double mean, double sdv) -> ncf_status {
            sd.stats[0].mean = mean;
            sd.stats[0].inv_std = 1.0 / sdv;
            sd.stats[0].flags &= ~STAT_DEGENERATE;
            NCF_CUDA(cudaMemcpyAsync(sd.d_stats, sd.stats.data(), sizeof(SeriesStats), cudaMemcpyHostToDevice, st));
            return NCF_OK;
        };
        if ((rc = patch(ev.X, ev.pooled->mean_x, ev.pooled->std_x))) return rc;
        if (!ev.acf && (rc = patch(ev.Y, ev.pooled->mean_y, ev.pooled->std_y))) return rc;
        NCF_CUDA(cudaStreamSynchronize(st));
    }
    if ((rc = check_stats(ctx, ev.X, B, "x"))) return rc;
    if (!ev.acf && (rc = check_stats(ctx, ev.Y, B, "y"))) return rc;
    ev.lagv.assign(h_lags, h_lags + K);
    ev.max_tau = 0.0;
    for (int64_t k = 0; k < K; ++k) {
        if (!std::isfinite(ev.lagv[k])) return fail(ctx, NCF_ENONFINITE, "lag %lld is not finite", (long long)k);
        ev.max_tau = std::max(ev.max_tau, std::fabs(ev.lagv[k]));
    }
    ev.t_abs = 0.0;
    for (int64_t b = 0; b < B; ++b) {
        ev.t_abs = std::max({ev.t_abs, std::fabs(ev.X.stats[b].t_first), std::fabs(ev.X.stats[b].t_last)});
        if (!ev.acf)
            ev.t_abs = std::max({ev.t_abs, std::fabs(ev.Y.stats[b].t_first), std::fabs(ev.Y.stats[b].t_last)});
    }
    return NCF_OK;
}

// Value bits of a rectangle evaluation's sides: each series side by its own
// size; a shard standardised with pooled statistics by the whole series' size,
// so that shards of one series quantise alike.
ValueBits value_bits_of(const Eval &ev) {
    ValueBits vb;
    vb.offs_x = ev.X.d_offs;
    vb.offs_y = ev.acf ? nullptr : ev.Y.d_offs;
    if (ev.pooled) {
        vb.nfx = ev.pooled->n_x;
        vb.nfy = ev.acf ? 0 : ev.pooled->n_y;
    }
    return vb;
}

SpectralArgs spectral_args(const Eval &ev, double *c_out, double *b_out, int64_t *count_out) {
    SpectralArgs sa;
    sa.acf = ev.acf;
    sa.B = ev.B;
    sa.K = ev.K;
    sa.h = ev.opt.h;
    sa.fp32 = ev.opt.precision == NCF_FP32;
    sa.kernel = ev.opt.kernel == NCF_RECTANGLE ? 1 : 0;
    if (sa.kernel == 1)
        sa.tol = ev.opt.tol > 0.0 ? ev.opt.tol : 1e-3;  // the spectral-sinc truncation
    else
        sa.tol = ev.opt.tol > 0.0 ? ev.opt.tol : (sa.fp32 ? 1e-7 : 1e-14);
    sa.max_tau = ev.max_tau;
    sa.lag0 = ev.lag0;
    sa.h_lags = ev.lagv.data();
    const Side &X = ev.X, &Y = ev.Y;
    sa.x = {X.t, X.v, X.d_offs, X.d_stats, X.offs.data(), X.stats.data(), X.n_total, X.n_max,
            X.d_chunk_base, X.n_chunks, X.d_cs};
    if (!ev.acf)
        sa.y = {Y.t, Y.v, Y.d_offs, Y.d_stats, Y.offs.data(), Y.stats.data(), Y.n_total, Y.n_max,
                Y.d_chunk_base, Y.n_chunks, Y.d_cs};
    sa.c_out = c_out;
    sa.b_out = b_out;
    sa.count_out = count_out;
    return sa;
}

size_t key_bytes(const Side &sd) {
    return al(sd.n_total * 8) * 2 + al((sd.n_total + 1) * 8) + al((sd.n_chunks + 1) * 8);
}

// Sizes of the path-specific device memory and of its host staging.
ncf_status main_bytes(ncf_ctx *ctx, Eval &ev, size_t *dev, size_t *pin) {
    const int64_t B = ev.B, K = ev.K;
    if (rect_scan(ev)) {
        const Side &O = ev.outer();
        const size_t rw = rect_workspace_bytes(O.rect_tiles, K);
        const size_t rwx = ev.lag0 ? rect_workspace_bytes(ev.X.rect_tiles, 1) : 0;
        const size_t rwy = (ev.lag0 && !ev.acf) ? rect_workspace_bytes(ev.Y.rect_tiles, 1) : 0;
        *dev = al(K * 8) + key_bytes(ev.X) + (ev.acf ? 0 : key_bytes(ev.Y)) + al(B * K * 8) * 3 +
               al(B * 8) * 8 + 1024 + rw + rwx + rwy;
        *pin = rect_staging_bytes(O.rect_tiles, K) + (ev.lag0 ? rect_staging_bytes(ev.X.rect_tiles, 1) : 0) +
               ((ev.lag0 && !ev.acf) ? rect_staging_bytes(ev.Y.rect_tiles, 1) : 0);
        return NCF_OK;
    }
    if (ev.path == NCF_PATH_WINDOWED) {
        const int64_t nt = ev.outer().scan_tiles;
        const int64_t nxt = (ev.lag0 && !ev.acf) ? ev.X.scan_tiles : 0;
        *dev = al(B * K * 8) * 3 + al(B * 8) * 8 + al(nt * sizeof(ScanTile)) + al(nxt * sizeof(ScanTile)) +
               al(K * 8) + 1024;
        *pin = al(nt * sizeof(ScanTile)) + al(nxt * sizeof(ScanTile)) + 256;
        return NCF_OK;
    }
    std::string msg;
    size_t ws = 0, pb = 0;
    ncf_status rc = spectral_plan(spectral_args(ev, nullptr, nullptr, nullptr), &ev.sp, &ws, &pb, &msg);
    if (rc) return fail(ctx, rc, "%s", msg.c_str());
    *dev = ws + al(K * 8) + 1024;
    *pin = pb;
    return NCF_OK;
}

// Carves the path-specific memory and uploads / builds its tables.
ncf_status prepare(ncf_ctx *ctx, Eval &ev, char *mem, size_t cap, char *pinned, size_t pin_cap,
                   const double *lags, cudaStream_t st) {
    const int64_t B = ev.B, K = ev.K;
    Arena a2{mem, cap, 0};
    std::string msg;
    ncf_status rc;
    // a private copy of the lags for the windowed path (plans outlive the caller's array)
    double *d_lags = a2.take<double>(K);
    if (!d_lags) return fail(ctx, NCF_ENOMEM, "internal: workspace estimate too small");
    NCF_CUDA(cudaMemcpyAsync(d_lags, lags, K * 8, cudaMemcpyDeviceToDevice, st));
    ev.d_lags = d_lags;
    if (rect_scan(ev)) {
        Side &X = ev.X, &O = ev.outer();
        ev.fs = choose_scales(ev.t_abs + ev.max_tau + ev.opt.h + 1.0);
        auto keys = [&](const Side &sd, int64_t *&T, int64_t *&Xq, int64_t *&P, int64_t *&C) {
            T = a2.take<int64_t>(sd.n_total);
            Xq = a2.take<int64_t>(sd.n_total);
            P = a2.take<int64_t>(sd.n_total + 1);
            C = a2.take<int64_t>(sd.n_chunks + 1);
        };
        keys(X, ev.kxT, ev.kxX, ev.kxP, ev.kxC);
        if (ev.acf) {
            ev.kyT = ev.kxT; ev.kyX = ev.kxX; ev.kyP = ev.kxP; ev.kyC = ev.kxC;
        } else {
            keys(ev.Y, ev.kyT, ev.kyX, ev.kyP, ev.kyC);
        }
        ev.cnt = a2.take<unsigned long long>(B * K);
        ev.num = a2.take<unsigned long long>(2 * B * K);
        ev.cnt0 = a2.take<unsigned long long>(2 * B);
        ev.num0 = a2.take<unsigned long long>(4 * B);
        ev.scale = a2.take<double>(B);
        const size_t rw = rect_workspace_bytes(rect_tiles_of(O.offs, B), K);
        char *rws = a2.take<char>(rw);
        if (!rws || !ev.scale) return fail(ctx, NCF_ENOMEM, "internal: workspace estimate too small");
        const int eps = ev.acf ? +1 : -1;
        RectArgs ra{ev.kxT, ev.kxP, X.t, X.d_offs, ev.kyT, ev.kyX, O.t, &O.offs, B, K, ev.lagv.data(), eps,
                    ev.opt.h, ev.fs, ev.cnt, ev.num};
        size_t poff = 0;
        const size_t rs = rect_staging_bytes(rect_tiles_of(O.offs, B), K);
        if ((rc = rect_prepare(ra, rws, rw, pinned, rs, st, &ev.r_main, &msg))) return fail(ctx, rc, "%s", msg.c_str());
        poff += rs;
        if (ev.lag0) {
            static const double zero = 0.0;
            const size_t rwx = rect_workspace_bytes(rect_tiles_of(X.offs, B), 1);
            const size_t rsx = rect_staging_bytes(rect_tiles_of(X.offs, B), 1);
            char *rx = a2.take<char>(rwx);
            if (!rx) return fail(ctx, NCF_ENOMEM, "internal: workspace estimate too small");
            RectArgs ax{ev.kxT, ev.kxP, X.t, X.d_offs, ev.kxT, ev.kxX, X.t, &X.offs, B, 1, &zero, +1, ev.opt.h,
                        ev.fs, ev.cnt0, ev.num0};
            if ((rc = rect_prepare(ax, rx, rwx, pinned + poff, rsx, st, &ev.r_x, &msg)))
                return fail(ctx, rc, "%s", msg.c_str());
            poff += rsx;
            if (!ev.acf) {
                Side &Y = ev.Y;
                const size_t rwy = rect_workspace_bytes(rect_tiles_of(Y.offs, B), 1);
                const size_t rsy = rect_staging_bytes(rect_tiles_of(Y.offs, B), 1);
                char *ry = a2.take<char>(rwy);
                if (!ry) return fail(ctx, NCF_ENOMEM, "internal: workspace estimate too small");
                RectArgs ay{ev.kyT, ev.kyP, Y.t, Y.d_offs, ev.kyT, ev.kyX, Y.t, &Y.offs, B, 1, &zero, +1,
                            ev.opt.h, ev.fs, ev.cnt0 + B, ev.num0 + 2 * B};
                if ((rc = rect_prepare(ay, ry, rwy, pinned + poff, rsy, st, &ev.r_y, &msg)))
                    return fail(ctx, rc, "%s", msg.c_str());
            }
        }
        (void)pin_cap;
        return NCF_OK;
    }
    if (ev.path == NCF_PATH_WINDOWED) {
        const int tj = scan_tile_points();
        std::vector<ScanTile> t1 = make_tiles(ev.outer().offs, B, tj);
        ev.g_ntiles = (int64_t)t1.size();
        ev.g_tiles = a2.take<ScanTile>(ev.g_ntiles);
        ev.gnum = a2.take<double>(B * K);
        ev.gden = a2.take<double>(B * K);
        ev.gcnt = a2.take<unsigned long long>(B * K);
        ev.gn0 = a2.take<double>(2 * B);
        ev.gd0 = a2.take<double>(2 * B);
        ev.gc0 = a2.take<unsigned long long>(2 * B);
        ev.scale = a2.take<double>(B);
        size_t off = 0;
        std::memcpy(pinned + off, t1.data(), t1.size() * sizeof(ScanTile));
        copy_pinned(ev.g_tiles, pinned + off, t1.size() * sizeof(ScanTile), st);
        off += al(t1.size() * sizeof(ScanTile));
        if (ev.lag0 && !ev.acf) {
            std::vector<ScanTile> t2 = make_tiles(ev.X.offs, B, tj);
            ev.g_nxtiles = (int64_t)t2.size();
            ev.g_xtiles = a2.take<ScanTile>(ev.g_nxtiles);
            if (!ev.g_xtiles) return fail(ctx, NCF_ENOMEM, "internal: workspace estimate too small");
            std::memcpy(pinned + off, t2.data(), t2.size() * sizeof(ScanTile));
            copy_pinned(ev.g_xtiles, pinned + off, t2.size() * sizeof(ScanTile), st);
        } else {
            ev.g_xtiles = ev.g_tiles;
            ev.g_nxtiles = ev.g_ntiles;
        }
        if (!ev.scale) return fail(ctx, NCF_ENOMEM, "internal: workspace estimate too small");
        return NCF_OK;
    }
    ev.spec_ws = mem + a2.used;  // the spectral workspace starts here (256-aligned)
    spectral_prepare(ev.sp, ev.spec_ws, pinned, st);
    ctx->plan = ncf_plan_info{ev.sp.L, ev.sp.M, ev.sp.nf, ev.sp.W, B, K,
                              std::max<int64_t>(1, (int64_t)ev.sp.buckets.size())};
    return NCF_OK;
}

// The per-data kernels of an evaluation; `stats_fresh` skips the statistics
// pass when `analyze` has just run it on the same data.
ncf_status launch(ncf_ctx *ctx, Eval &ev, bool stats_fresh, bool guard, double *c_out, double *b_out,
                  int64_t *count_out, cudaStream_t st, bool first = true) {
    const int64_t B = ev.B, K = ev.K;
    std::string msg;
    ncf_status rc;
    // the status word and the statistics belong to the first option set of an evaluation
    if (first) NCF_CUDA(cudaMemsetAsync(ev.status, 0, sizeof(int), st));
    if (!stats_fresh) run_stats(ev, st);
    if (guard && first) launch_stats_guard(ev.X.d_stats, ev.acf ? nullptr : ev.Y.d_stats, B, ev.status, st);
    Side &X = ev.X, &O = ev.outer();
    if (rect_scan(ev)) {
        const ValueBits vb = value_bits_of(ev);
        launch_keys_prefix(X.t, X.v, X.d_offs, X.d_chunk_base, X.d_cs, X.n_chunks, kPrepChunk, X.d_stats, ev.fs,
                           vb.nfx, ev.kxT, ev.kxX, ev.kxP, ev.kxC, X.n_total, st);
        if (!ev.acf)
            launch_keys_prefix(ev.Y.t, ev.Y.v, ev.Y.d_offs, ev.Y.d_chunk_base, ev.Y.d_cs, ev.Y.n_chunks, kPrepChunk,
                               ev.Y.d_stats, ev.fs, vb.nfy, ev.kyT, ev.kyX, ev.kyP, ev.kyC, ev.Y.n_total, st);
        if (guard) launch_keys_guard(ev.X.d_stats, ev.acf ? nullptr : ev.Y.d_stats, B, ev.t_abs, ev.status, st);
        NCF_CUDA(cudaMemsetAsync(ev.cnt, 0, B * K * 8, st));
        NCF_CUDA(cudaMemsetAsync(ev.num, 0, 2 * B * K * 8, st));
        const int eps = ev.acf ? +1 : -1;
        RectArgs ra{ev.kxT, ev.kxP, X.t, X.d_offs, ev.kyT, ev.kyX, O.t, &O.offs, B, K, ev.lagv.data(), eps,
                    ev.opt.h, ev.fs, ev.cnt, ev.num};
        if ((rc = rect_launch(ra, ev.r_main, st, &msg))) return fail(ctx, rc, "%s", msg.c_str());
        if (ev.lag0) {
            NCF_CUDA(cudaMemsetAsync(ev.cnt0, 0, 2 * B * 8, st));
            NCF_CUDA(cudaMemsetAsync(ev.num0, 0, 4 * B * 8, st));
            static const double zero = 0.0;
            RectArgs ax{ev.kxT, ev.kxP, X.t, X.d_offs, ev.kxT, ev.kxX, X.t, &X.offs, B, 1, &zero, +1, ev.opt.h,
                        ev.fs, ev.cnt0, ev.num0};
            if ((rc = rect_launch(ax, ev.r_x, st, &msg))) return fail(ctx, rc, "%s", msg.c_str());
            if (!ev.acf) {
                Side &Y = ev.Y;
                RectArgs ay{ev.kyT, ev.kyP, Y.t, Y.d_offs, ev.kyT, ev.kyX, Y.t, &Y.offs, B, 1, &zero, +1,
                            ev.opt.h, ev.fs, ev.cnt0 + B, ev.num0 + 2 * B};
                if ((rc = rect_launch(ay, ev.r_y, st, &msg))) return fail(ctx, rc, "%s", msg.c_str());
            }
            launch_lag0_scale_rect(ev.cnt0, ev.num0, ev.acf ? nullptr : ev.cnt0 + B,
                                   ev.acf ? nullptr : ev.num0 + 2 * B, B, vb, ev.scale, st);
        }
        launch_finish_rect(ev.cnt, ev.num, B, K, vb, ev.lag0 ? ev.scale : nullptr, ev.status, c_out, b_out,
                           count_out, st);
    } else if (ev.path == NCF_PATH_WINDOWED) {
        const int hann = ev.opt.kernel == NCF_HANNING;
        const double R = hann ? 1.0 : (ev.opt.trunc_R > 0.0 ? ev.opt.trunc_R : 8.0);
        const double Rh = R * ev.opt.h;
        NCF_CUDA(cudaMemsetAsync(ev.gnum, 0, B * K * 8, st));
        NCF_CUDA(cudaMemsetAsync(ev.gden, 0, B * K * 8, st));
        NCF_CUDA(cudaMemsetAsync(ev.gcnt, 0, B * K * 8, st));
        const int eps = ev.acf ? +1 : -1;
        launch_gauss_window(X.t, ev.den_only ? nullptr : X.v, X.d_offs, X.d_stats, O.t, O.v, O.d_stats, ev.g_tiles,
                            ev.g_ntiles, ev.d_lags, K, eps, ev.opt.h, Rh, hann, ev.gnum, ev.gden, ev.gcnt, st);
        if (ev.lag0) {
            NCF_CUDA(cudaMemsetAsync(ev.zero_lag, 0, 8, st));
            NCF_CUDA(cudaMemsetAsync(ev.gn0, 0, 2 * B * 8, st));
            NCF_CUDA(cudaMemsetAsync(ev.gd0, 0, 2 * B * 8, st));
            NCF_CUDA(cudaMemsetAsync(ev.gc0, 0, 2 * B * 8, st));
            launch_gauss_window(X.t, X.v, X.d_offs, X.d_stats, X.t, X.v, X.d_stats, ev.g_xtiles, ev.g_nxtiles,
                                ev.zero_lag, 1, +1, ev.opt.h, Rh, hann, ev.gn0, ev.gd0, ev.gc0, st);
            if (!ev.acf)
                launch_gauss_window(ev.Y.t, ev.Y.v, ev.Y.d_offs, ev.Y.d_stats, ev.Y.t, ev.Y.v, ev.Y.d_stats,
                                    ev.g_tiles, ev.g_ntiles, ev.zero_lag, 1, +1, ev.opt.h, Rh, hann, ev.gn0 + B,
                                    ev.gd0 + B, ev.gc0 + B, st);
            launch_lag0_scale_gauss(ev.gn0, ev.gd0, ev.acf ? nullptr : ev.gn0 + B, ev.acf ? nullptr : ev.gd0 + B, B,
                                    ev.scale, st);
        }
        launch_finish_gauss(ev.gnum, ev.gden, ev.gcnt, B, K, ev.lag0 ? ev.scale : nullptr, ev.status, c_out, b_out,
                            count_out, st);
    } else {
        SpectralArgs sa = spectral_args(ev, c_out, b_out, count_out);
        if (guard) spectral_guard(sa, ev.sp, ev.spec_ws, ev.status, st);
        if ((rc = spectral_launch(sa, ev.sp, ev.spec_ws, ev.status, st, &msg))) return fail(ctx, rc, "%s", msg.c_str());
    }
    NCF_CUDA(cudaGetLastError());
    return NCF_OK;
}

// FP64 Gaussian with NCF_PATH_AUTO: the windowed scan costs one FP64 exp per
// pair inside the window, O(n K n_window); the spectral path costs the
// spreading, the FFT and the mode sums, O(n W + n_f log n_f + M K) per series.
// The crossover in K is the paper's K* (Sec. 5.1); here it is a cost model
// with constants measured on B300 (windowed 44 ps per pair; FP64 spreading
// 0.4 ns per point; FP64 FFT 16 B per cell and pass at 5 TB/s; FP64 mode sums
// at 0.57 T FMA/s).
void choose_path(Eval &ev) {
    if (ev.path != NCF_PATH_AUTO) return;
    const double R = ev.opt.trunc_R > 0.0 ? ev.opt.trunc_R : 8.0;
    double win = 0.0, spread = 0.0, max_span = 0.0;
    for (int64_t b = 0; b < ev.B; ++b) {
        const SeriesStats &sx = ev.X.stats[b];
        const SeriesStats &so = ev.acf ? sx : ev.Y.stats[b];
        double lo = sx.t_first, hi = sx.t_last;
        if (!ev.acf) { lo = std::min(lo, so.t_first); hi = std::max(hi, so.t_last); }
        max_span = std::max(max_span, hi - lo);
        const double span = std::max(sx.t_last - sx.t_first, 1e-300);
        const double in_window = std::min((double)sx.n, (double)sx.n / span * 2.0 * R * ev.opt.h + 1.0);
        win += (double)so.n * (double)ev.K * in_window;
        spread += (double)(sx.n + (ev.acf ? 0 : so.n));
    }
    const double L = max_span + ev.max_tau + 8.6 * ev.opt.h;
    const double M = L * 1.408 / ev.opt.h + 1.0;
    double nf = 1.0;
    while (nf < 4.0 * M + 16.0) nf *= 2.0;
    const double passes = std::ceil(std::log2(nf) / 3.0) * (ev.acf ? 1.0 : 2.0);
    const double t_win = win * 44e-12;
    const double t_spec = spread * 0.4e-9 + (double)ev.B * nf * 16.0 * 2.0 * passes / 5e12 +
                          (double)ev.B * M * (ev.K + 1.0) * 2.0 * (ev.acf ? 1.0 : 2.0) / 0.57e12;
    ev.path = t_win < t_spec ? NCF_PATH_WINDOWED : NCF_PATH_SPECTRAL;
}

uint64_t rect_tune_key(const Eval &ev) {
    auto lg = [](double v) { return (uint64_t)std::max(0.0, std::floor(std::log2(std::max(v, 1.0)))); };
    const Side &O = ev.acf ? ev.X : ev.Y;
    return lg((double)O.n_total) | (lg((double)O.n_total / (double)ev.B) << 8) | (lg((double)ev.K) << 16) |
           ((uint64_t)ev.acf << 24);
}

// Autotuned rectangle-scan variant per (device, problem bucket), shared by
// every context of the process (server slots, plans, one-shot calls).
std::mutex g_tune_mu;
std::map<std::pair<int, uint64_t>, int> g_tune_rect;

// Times the rectangle-scan variants once per problem bucket (they give
// identical, exact results) and keeps the fastest for the process.
ncf_status tune_rect(ncf_ctx *ctx, Eval &ev, cudaStream_t st) {
    // NCF_RECT_VARIANT=0|1|2|3 pins a variant (tests, measurements) and skips the timing
    if (const char *pin = std::getenv("NCF_RECT_VARIANT")) {
        const int v = std::atoi(pin);
        if (v >= 0 && v < kRectVariants) {
            ev.r_main.variant = ev.r_x.variant = ev.r_y.variant = v;
            ctx->tuning.rect_variant = v;
            return NCF_OK;
        }
    }
    const std::pair<int, uint64_t> key{ctx->device, rect_tune_key(ev)};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_rect.find(key);
        if (it != g_tune_rect.end()) {
            ev.r_main.variant = ev.r_x.variant = ev.r_y.variant = it->second;
            ctx->tuning.rect_variant = it->second;
            return NCF_OK;
        }
    }
    const int64_t B = ev.B, K = ev.K;
    Side &X = ev.X, &O = ev.outer();
    const ValueBits vb = value_bits_of(ev);
    launch_keys_prefix(X.t, X.v, X.d_offs, X.d_chunk_base, X.d_cs, X.n_chunks, kPrepChunk, X.d_stats, ev.fs,
                       vb.nfx, ev.kxT, ev.kxX, ev.kxP, ev.kxC, X.n_total, st);
    if (!ev.acf)
        launch_keys_prefix(ev.Y.t, ev.Y.v, ev.Y.d_offs, ev.Y.d_chunk_base, ev.Y.d_cs, ev.Y.n_chunks, kPrepChunk,
                           ev.Y.d_stats, ev.fs, vb.nfy, ev.kyT, ev.kyX, ev.kyP, ev.kyC, ev.Y.n_total, st);
    cudaEvent_t e[kRectVariants + 1];
    for (auto &x : e) NCF_CUDA(cudaEventCreate(&x));
    std::string msg;
    const int eps = ev.acf ? +1 : -1;
    RectArgs ra{ev.kxT, ev.kxP, X.t, X.d_offs, ev.kyT, ev.kyX, O.t, &O.offs, B, K, ev.lagv.data(), eps,
                ev.opt.h, ev.fs, ev.cnt, ev.num};
    NCF_CUDA(cudaEventRecord(e[0], st));
    for (int v = 0; v < kRectVariants; ++v) {
        ev.r_main.variant = v;
        ncf_status rc = rect_launch(ra, ev.r_main, st, &msg);
        if (rc) return fail(ctx, rc, "%s", msg.c_str());
        NCF_CUDA(cudaEventRecord(e[v + 1], st));
    }
    NCF_CUDA(cudaEventSynchronize(e[kRectVariants]));
    int best = 1;
    float best_ms = 1e30f;
    for (int v = 0; v < kRectVariants; ++v) {
        float ms = 0.0f;
        NCF_CUDA(cudaEventElapsedTime(&ms, e[v], e[v + 1]));
        if (ms < best_ms) { best_ms = ms; best = v; }
    }
    for (auto &x : e) cudaEventDestroy(x);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_rect[key] = best;
    }
    ev.r_main.variant = ev.r_x.variant = ev.r_y.variant = best;
    ctx->tuning.rect_variant = best;
    return NCF_OK;
}


// Autotuned FP32 spectral shapes per (device, problem bucket): the spreading
// (CTAs of a statistics chunk of points or of half of one; tile sums in FP32 by
// compare-and-swap or in fixed point by integer atomics), the FFT of an ACF
// grid that fits shared memory (there, fused with its spectrum, or as global
// passes) and the mode-to-lag contraction (tensor cores or the FP32 pipe).  The
// candidates agree within the FP32 form's error, not bit for bit; the one kept
// is the fastest on the first batch of its bucket, and the caller's evaluation
// then runs with it.
std::map<std::pair<int, uint64_t>, int> g_tune_spec;
// v = fft + 2 contraction + 4 spreading: fft 1 = global passes, contraction 1 = the
// FP32 pipe, spreading bit 0 = CTAs of half a statistics chunk, bit 1 = fixed-point
// tile sums
constexpr int kSpecVariants = 16;

uint64_t spec_tune_key(const Eval &ev) {
    auto lg = [](double v) { return (uint64_t)std::max(0.0, std::floor(std::log2(std::max(v, 1.0)))); };
    return lg((double)ev.B) | ((uint64_t)ev.sp.lg << 8) | (lg((double)ev.K) << 16) | ((uint64_t)ev.acf << 24) |
           ((uint64_t)ev.sp.kernel << 25);
}

void set_spec_variant(ncf_ctx *ctx, Eval &ev, int v) {
    ev.sp.fft_variant = v & 1;
    ev.sp.contract_variant = (v >> 1) & 1;
    ev.sp.spread_variant = v >> 2;
    // the shared-memory FFT applies to ACF grids of 2^7..2^14 cells only
    const bool fft_choice = ev.acf && ev.sp.lg >= 7 && ev.sp.lg <= 14;
    ctx->tuning.fft_variant = fft_choice ? ev.sp.fft_variant : 1;
    ctx->tuning.contract_variant = ev.sp.contract_variant;
    ctx->tuning.spread_variant = ev.sp.spread_variant;
}

ncf_status tune_spectral(ncf_ctx *ctx, Eval &ev, cudaStream_t st) {
    if (rect_scan(ev) || ev.path == NCF_PATH_WINDOWED || !ev.sp.fp32 || ev.sp.direct) return NCF_OK;
    // NCF_SPEC_VARIANT=0..15 pins the shapes (tests, measurements) and skips the timing
    if (const char *pin = std::getenv("NCF_SPEC_VARIANT")) {
        const int v = std::atoi(pin);
        if (v >= 0 && v < kSpecVariants) {
            set_spec_variant(ctx, ev, v);
            return NCF_OK;
        }
    }
    const std::pair<int, uint64_t> key{ctx->device, spec_tune_key(ev)};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_spec.find(key);
        if (it != g_tune_spec.end()) {
            set_spec_variant(ctx, ev, it->second);
            return NCF_OK;
        }
    }
    // the FFT choice exists only where the shared-memory FFT applies
    const bool fft_choice = ev.acf && ev.sp.lg >= 7 && ev.sp.lg <= 14;
    std::vector<int> cands;
    for (int v = 0; v < kSpecVariants; ++v)
        if (fft_choice || !(v & 1)) cands.push_back(v);
    // scratch outputs: the timing runs write results that the evaluation proper overwrites
    const int64_t BK = ev.B * ev.K;
    double *scratch = nullptr;
    NCF_CUDA(cudaMallocAsync(reinterpret_cast<void **>(&scratch), (size_t)BK * 24, st));
    SpectralArgs sa = spectral_args(ev, scratch, scratch + BK, reinterpret_cast<int64_t *>(scratch + 2 * BK));
    std::vector<cudaEvent_t> e(cands.size() + 1);
    for (auto &x : e) NCF_CUDA(cudaEventCreate(&x));
    std::string msg;
    ncf_status rc = NCF_OK;
    NCF_CUDA(cudaEventRecord(e[0], st));
    for (size_t i = 0; i < cands.size() && !rc; ++i) {
        set_spec_variant(ctx, ev, cands[i]);
        rc = spectral_launch(sa, ev.sp, ev.spec_ws, ev.status, st, &msg);
        cudaEventRecord(e[i + 1], st);
    }
    int best = 0;
    if (!rc) {
        NCF_CUDA(cudaEventSynchronize(e.back()));
        float best_ms = 1e30f;
        for (size_t i = 0; i < cands.size(); ++i) {
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e[i], e[i + 1]);
            if (ms < best_ms) {
                best_ms = ms;
                best = cands[i];
            }
        }
    }
    for (auto &x : e) cudaEventDestroy(x);
    cudaFreeAsync(scratch, st);
    if (rc) return fail(ctx, rc, "%s", msg.c_str());
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_spec[key] = best;
    }
    set_spec_variant(ctx, ev, best);
    return NCF_OK;
}

}  // namespace

// ----------------------------------------------------------------------------
// The batch driver.  All device pointers come from the caller; offsets are host.
// ----------------------------------------------------------------------------
static ncf_status corr_batch_impl(ncf_ctx *ctx, const int64_t *offs_x, const double *t,
                                  const double *x, const int64_t *offs_y, const double *s,
                                  const double *y, int64_t B, const double *lags, int64_t K,
                                  const ncf_options *opt, double *c_out, double *b_out,
                                  int64_t *count_out, cudaStream_t st, bool den_only = false,
                                  const ncf_pooled_stats *pooled = nullptr) {
    LaunchScope scope(ctx);
    ctx->err.clear();
    // the pinned staging buffer may still feed a copy queued by the previous call
    if (ctx->staged) NCF_CUDA(cudaEventSynchronize(ctx->staged));
    Eval ev;
    ncf_status rc = check_args(ctx, offs_x, t, x, offs_y, s, y, B, lags, K, opt, ev);
    if (rc) return rc;
    ev.den_only = den_only;
    ev.pooled = pooled;
    if (!c_out) return fail(ctx, NCF_EINVAL, "c_out is NULL");
    ev.X.t = t; ev.X.v = x;
    if (!ev.acf) { ev.Y.t = s; ev.Y.v = y; }
    if ((rc = grow(ctx, &ctx->ws, &ctx->ws_cap, pre_bytes(ev), st))) return rc;
    carve_pre(ev, ctx->ws);
    if ((rc = analyze(ctx, ev, lags, st))) return rc;
    choose_path(ev);
    size_t dev = 0, pin = 0;
    if ((rc = main_bytes(ctx, ev, &dev, &pin))) return rc;
    if ((rc = grow(ctx, &ctx->ws2, &ctx->ws2_cap, dev, st))) return rc;
    if ((rc = grow_pinned(ctx, pin, st))) return rc;
    if ((rc = prepare(ctx, ev, ctx->ws2, ctx->ws2_cap, ctx->pinned, ctx->pinned_cap, lags, st))) return rc;
    NCF_CUDA(cudaEventRecord(ctx->staged, st));
    if (rect_scan(ev) && (rc = tune_rect(ctx, ev, st))) return rc;
    if ((rc = tune_spectral(ctx, ev, st))) return rc;
    return launch(ctx, ev, /*stats_fresh=*/true, /*guard=*/false, c_out, b_out, count_out, st);
}

// Several option sets (estimators) on one batch: the statistics pass and its
// read-back run once, then each option set prepares and launches its own path
// on the same statistics.
// The statistics stage of a batched call with several option sets: arguments
// checked, the pre-statistics workspace carved from *ws, the statistics pass run
// on `st` and read back (the host waits for `st` here).  `pre_staging`: the
// stage runs beside another chunk's evaluation and stages through the second
// pinned buffer.
static ncf_status batch_pre(ncf_ctx *ctx, const int64_t *offs_x, const double *t, const double *x,
                            const int64_t *offs_y, const double *s, const double *y, int64_t B, const double *lags,
                            int64_t K, const ncf_options *opts, int n_opts, double *const *c_out, Eval &ev,
                            std::vector<int> &paths, char **ws, size_t *ws_cap, bool pre_staging, cudaStream_t st) {
    if (!opts || n_opts < 1 || !c_out) return fail(ctx, NCF_EINVAL, "no option set or c_out is NULL");
    if (!pre_staging && ctx->staged) NCF_CUDA(cudaEventSynchronize(ctx->staged));
    ncf_status rc = check_args(ctx, offs_x, t, x, offs_y, s, y, B, lags, K, &opts[0], ev);
    if (rc) return rc;
    paths.assign(n_opts, 0);
    for (int o = 0; o < n_opts; ++o) {
        if (!c_out[o]) return fail(ctx, NCF_EINVAL, "c_out of option set %d is NULL", o);
        if ((rc = check_options(ctx, &opts[o], B, K, &paths[o]))) return rc;
    }
    ev.X.t = t; ev.X.v = x;
    if (!ev.acf) { ev.Y.t = s; ev.Y.v = y; }
    if ((rc = grow(ctx, ws, ws_cap, pre_bytes(ev), st))) return rc;
    carve_pre(ev, *ws);
    return analyze(ctx, ev, lags, st, pre_staging);
}

// The rest of a batched call, on `st` after its statistics stage: each option
// set prepared and launched.
static ncf_status batch_main(ncf_ctx *ctx, const Eval &ev, const std::vector<int> &paths, const double *lags,
                             const ncf_options *opts, int n_opts, double *const *c_out, double *const *b_out,
                             int64_t *const *count_out, cudaStream_t st) {
    ncf_status rc;
    // the pinned staging may still feed the previous evaluation's uploads
    if (ctx->staged) NCF_CUDA(cudaEventSynchronize(ctx->staged));
    // The host prepares each option set after the statistics read-back while the
    // GPU runs what is already queued: the long real-space scans go first, so the
    // spectral sets' host preparation hides behind them.
    std::vector<Eval> evs(n_opts, ev);  // the sides, their statistics and the lags, shared
    std::vector<int> order(n_opts);
    for (int o = 0; o < n_opts; ++o) {
        evs[o].opt = opts[o];
        evs[o].path = paths[o];
        evs[o].lag0 = opts[o].norm == NCF_NORM_LAG0;
        choose_path(evs[o]);
        order[o] = o;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (evs[a].path == NCF_PATH_SPECTRAL) < (evs[b].path == NCF_PATH_SPECTRAL);
    });
    for (int q = 0; q < n_opts; ++q) {
        const int o = order[q];
        Eval &eo = evs[o];
        size_t dev = 0, pin = 0;
        if ((rc = main_bytes(ctx, eo, &dev, &pin))) return rc;
        // the pinned staging may still feed the previous option set's uploads
        if (q > 0 && ctx->staged) NCF_CUDA(cudaEventSynchronize(ctx->staged));
        if ((rc = grow(ctx, &ctx->ws2, &ctx->ws2_cap, dev, st))) return rc;
        if ((rc = grow_pinned(ctx, pin, st))) return rc;
        if ((rc = prepare(ctx, eo, ctx->ws2, ctx->ws2_cap, ctx->pinned, ctx->pinned_cap, lags, st))) return rc;
        NCF_CUDA(cudaEventRecord(ctx->staged, st));
        if (rect_scan(eo) && (rc = tune_rect(ctx, eo, st))) return rc;
        if ((rc = tune_spectral(ctx, eo, st))) return rc;
        if ((rc = launch(ctx, eo, /*stats_fresh=*/true, /*guard=*/false, c_out[o], b_out ? b_out[o] : nullptr,
                         count_out ? count_out[o] : nullptr, st)))
            return rc;
    }
    return NCF_OK;
}

static ncf_status corr_batch_multi_impl(ncf_ctx *ctx, const int64_t *offs_x, const double *t, const double *x,
                                        const int64_t *offs_y, const double *s, const double *y, int64_t B,
                                        const double *lags, int64_t K, const ncf_options *opts, int n_opts,
                                        double *const *c_out, double *const *b_out, int64_t *const *count_out,
                                        cudaStream_t st) {
    LaunchScope scope(ctx);
    ctx->err.clear();
    Eval ev;
    std::vector<int> paths;
    ncf_status rc = batch_pre(ctx, offs_x, t, x, offs_y, s, y, B, lags, K, opts, n_opts, c_out, ev, paths, &ctx->ws,
                              &ctx->ws_cap, false, st);
    if (rc) return rc;
    return batch_main(ctx, ev, paths, lags, opts, n_opts, c_out, b_out, count_out, st);
}

// frac(tau / L) 2^64 to about one unit: q = fl(tau / L), the exact remainder
// e = tau - q L from one FMA, then the fraction of q plus e / L.
static unsigned long long lag_phase(double tau, double L) {
    const double q = tau / L;
    const double e = std::fma(-q, L, tau);
    const double fq = q - std::floor(q);                                  // exact, in [0, 1)
    const unsigned long long hi = (unsigned long long)std::ldexp(fq, 64);  // exact above 2^-11
    const long long lo = std::llround(std::ldexp(e / L, 64));
    return hi + (unsigned long long)lo;
}

constexpr int64_t kPaperType2Lags = 48;

static ncf_status corr_paper_impl(ncf_ctx *ctx, const double *t, const double *x, int64_t nx, const double *s,
                                  const double *y, int64_t ny, const double *lags, int64_t K, ncf_kernel kernel,
                                  double h, int64_t N1, double *c_out, double *b_out, cudaStream_t st) {
    LaunchScope scope(ctx);
    ctx->err.clear();
    if (ctx->staged) NCF_CUDA(cudaEventSynchronize(ctx->staged));
    if (kernel != NCF_GAUSSIAN && kernel != NCF_RECTANGLE)
        return fail(ctx, NCF_EUNSUPPORTED, "the paper's NUFFT estimators smooth with a Gaussian or a box only");
    if (!(h > 0.0) || !std::isfinite(h)) return fail(ctx, NCF_EINVAL, "h = %g (need finite h > 0)", h);
    const int box = kernel == NCF_RECTANGLE ? (int)std::nearbyint(2.0 * h) : 0;
    if (kernel == NCF_RECTANGLE && box < 1)
        return fail(ctx, NCF_EINVAL, "box filter size round(2h) = %d for h = %g (need >= 1)", box, h);
    if (N1 < 0) return fail(ctx, NCF_EINVAL, "N1 = %lld (need >= 0; 0 = the default rule)", (long long)N1);
    if (!c_out) return fail(ctx, NCF_EINVAL, "c_out is NULL");
    ncf_options opt;
    ncf_options_default(&opt);
    opt.kernel = kernel;
    opt.h = h;
    opt.path = NCF_PATH_WINDOWED;
    opt.precision = NCF_FP64;
    opt.norm = NCF_NORM_NONE;
    opt.trunc_R = kernel == NCF_GAUSSIAN ? 6.0 : 0.0;  // PairCount's window [c - 6h, c + 6h)
    const int64_t ox[2] = {0, nx}, oy[2] = {0, ny};
    const bool acf = (s == nullptr && y == nullptr);
    Eval ev;
    ncf_status rc = check_args(ctx, ox, t, x, acf ? nullptr : oy, s, y, 1, lags, K, &opt, ev);
    if (rc) return rc;
    ev.X.t = t; ev.X.v = x;
    if (!acf) { ev.Y.t = s; ev.Y.v = y; }
    if ((rc = grow(ctx, &ctx->ws, &ctx->ws_cap, pre_bytes(ev), st))) return rc;
    carve_pre(ev, ctx->ws);
    if ((rc = analyze(ctx, ev, lags, st))) return rc;

    // Algorithms 2 and 4, first steps: lag 0 prepended, stable sort
    const int64_t K1 = K + 1;
    std::vector<double> tau_eval(K1);
    tau_eval[0] = 0.0;
    for (int64_t k = 0; k < K; ++k) tau_eval[k + 1] = ev.lagv[k];
    std::vector<int64_t> perm(K1);
    std::iota(perm.begin(), perm.end(), 0);
    std::stable_sort(perm.begin(), perm.end(), [&](int64_t a, int64_t b) { return tau_eval[a] < tau_eval[b]; });
    std::vector<double> tau_srt(K1);
    int64_t pos0 = 0;
    for (int64_t i = 0; i < K1; ++i) {
        tau_srt[i] = tau_eval[perm[i]];
        if (perm[i] == 0) pos0 = i;
    }
    // Algorithm 1 on the union of both series' extents
    double t_min = ev.X.stats[0].t_first, t_max = ev.X.stats[0].t_last;
    int64_t n_max = nx;
    if (!acf) {
        t_min = std::min(t_min, ev.Y.stats[0].t_first);
        t_max = std::max(t_max, ev.Y.stats[0].t_last);
        n_max = std::max(nx, ny);
    }
    const double span = t_max - t_min;
    if (!(span > 0.0)) return fail(ctx, NCF_EDEGENERATE, "the times span no interval (span = %g)", span);
    double max_tau = 0.0;
    for (double v : tau_srt) max_tau = std::max(max_tau, std::fabs(v));
    const double L = span + 2.0 * max_tau;
    const double tc = t_min + span / 2.0;
    const double n1f = N1 > 0 ? (double)N1 : std::nearbyint(32.0 * (double)n_max * L / span);
    if (!(n1f >= 1.0) || n1f > 1e12) return fail(ctx, NCF_EUNSUPPORTED, "N1 = %g out of range", n1f);
    PaperModes pm;
    std::string msg;
    if ((rc = paper_modes_plan(L, tc, (int64_t)n1f, &pm, &msg))) return fail(ctx, rc, "%s", msg.c_str());
    // Algorithm 3's symmetric array, the smoothing weights and the lag phases
    const int n_h = std::max((int)std::ceil(4.0 * h) + 2, 5);
    const int64_t nsym = 2 * n_h + 1;
    std::vector<double> w;
    int o0 = 0;
    if (kernel == NCF_GAUSSIAN) {
        const int r = (int)(4.0 * h + 0.5);
        double sum = 0.0;
        for (int j = -r; j <= r; ++j) {
            w.push_back(std::exp(-0.5 / (h * h) * (double)j * (double)j));
            sum += w.back();
        }
        for (double &v : w) v /= sum;
        o0 = -r;
    } else {
        w.assign(box, 1.0 / box);
        o0 = -(box / 2);
    }
    std::vector<unsigned long long> phi(K1 + nsym);
    for (int64_t i = 0; i < K1; ++i) phi[i] = lag_phase(tau_srt[i], L);
    for (int64_t j = 0; j < nsym; ++j) phi[K1 + j] = lag_phase((double)(j - n_h), L);
    const double zero = 0.0;

    // device memory of the variant (ctx->paper; the nested pair-count calls use ws, ws2, pinned)
    const int64_t Mh = pm.Mh;
    const size_t modes_b = paper_modes_bytes(pm, !acf);
    const size_t need = modes_b + al((Mh + 1) * 16) * (acf ? 1 : 3) + al((K1 + nsym) * 8) +
                        al(K1 * 8) * 5 + al(nsym * 8) * 2 + al(8) * 3 + al(K1 * 8) + al(w.size() * 8) + 4096;
    if ((rc = grow(ctx, &ctx->paper, &ctx->paper_cap, need, st))) return rc;
    Arena ar{ctx->paper, ctx->paper_cap, 0};
    char *modes_ws = ar.take<char>(modes_b);
    double2 *A = ar.take<double2>(Mh + 1);
    double2 *Ax = acf ? nullptr : ar.take<double2>(Mh + 1);
    double2 *Ay = acf ? nullptr : ar.take<double2>(Mh + 1);
    auto *d_phi = ar.take<unsigned long long>(K1 + nsym);
    double *craw = ar.take<double>(K1), *bsrt = ar.take<double>(K1), *ctmp = ar.take<double>(K1);
    double *d_tau = ar.take<double>(K1), *tmp = ar.take<double>(K1);
    double *craw_x = ar.take<double>(nsym), *craw_y = ar.take<double>(nsym);
    double *bx0 = ar.take<double>(1), *by0 = ar.take<double>(1), *d_zero = ar.take<double>(1);
    auto *d_perm = ar.take<int64_t>(K1);
    double *d_w = ar.take<double>(w.size());
    if (!modes_ws || !A || (!acf && (!Ax || !Ay)) || !d_phi || !craw || !bsrt || !ctmp || !d_tau || !tmp ||
        !craw_x || !craw_y || !bx0 || !by0 || !d_zero || !d_perm || !d_w)
        return fail(ctx, NCF_ENOMEM, "internal: workspace estimate too small");
    const size_t pin_need = al((K1 + nsym) * 8) + al(K1 * 8) * 2 + al(8) + al(w.size() * 8) +
                            paper_modes_pinned_bytes(pm) + 1024;
    if ((rc = grow_pinned(ctx, pin_need, st))) return rc;
    size_t off = 0;
    auto up = [&](void *dst, const void *src, size_t bytes) -> ncf_status {
        std::memcpy(ctx->pinned + off, src, bytes);
        copy_pinned(dst, ctx->pinned + off, bytes, st);
        off += al(bytes);
        return NCF_OK;
    };
    if ((rc = up(d_phi, phi.data(), (K1 + nsym) * 8))) return rc;
    if ((rc = up(d_tau, tau_srt.data(), K1 * 8))) return rc;
    if ((rc = up(d_perm, perm.data(), K1 * 8))) return rc;
    if ((rc = up(d_zero, &zero, 8))) return rc;
    if ((rc = up(d_w, w.data(), w.size() * 8))) return rc;

    // type-1 coefficients, spectra and the raw correlation (Algorithms 2-4)
    const SpecSide sx{ev.X.t, ev.X.v, ev.X.d_offs, ev.X.d_stats, ev.X.offs.data(), ev.X.stats.data(),
                      ev.X.n_total, ev.X.n_max, ev.X.d_chunk_base, ev.X.n_chunks, ev.X.d_cs};
    SpecSide sy{};
    if (!acf)
        sy = SpecSide{ev.Y.t, ev.Y.v, ev.Y.d_offs, ev.Y.d_stats, ev.Y.offs.data(), ev.Y.stats.data(),
                      ev.Y.n_total, ev.Y.n_max, ev.Y.d_chunk_base, ev.Y.n_chunks, ev.Y.d_cs};
    double2 *Fx = nullptr, *Fy = nullptr;
    paper_modes_run(pm, sx, acf ? nullptr : &sy, modes_ws, ctx->pinned + off, &Fx, &Fy, st);
    NCF_CUDA(cudaEventRecord(ctx->staged, st));
    NCF_CUDA(cudaMemsetAsync(craw, 0, K1 * 8, st));
    if (acf) {
        paper_spectrum(Fx, Fx, Mh, pm.N1, A, st);
    } else {
        paper_spectrum(Fx, Fy, Mh, pm.N1, A, st);
        paper_spectrum(Fx, Fx, Mh, pm.N1, Ax, st);
        paper_spectrum(Fy, Fy, Mh, pm.N1, Ay, st);
        NCF_CUDA(cudaMemsetAsync(craw_x, 0, nsym * 8, st));
        NCF_CUDA(cudaMemsetAsync(craw_y, 0, nsym * 8, st));
        paper_eval(Ax, Mh, d_phi + K1, nsym, craw_x, st, Ay, craw_y);
    }
    // the sorted lags: a direct mode sum for short arrays, a type-2 transform (one FFT
    // and 16 taps per lag) from kPaperType2Lags on
    if (K1 >= kPaperType2Lags)
        paper_type2(pm, !acf, modes_ws, A, d_phi, K1, craw, st);
    else
        paper_eval(A, Mh, d_phi, K1, craw, st);
    // PairCount (Algorithms 5 and 6) through the windowed paths, pair sums alone:
    // the sorted lags and, for the CCF scales, lag 0 of each series' ACF
    if ((rc = corr_batch_impl(ctx, ox, t, x, acf ? nullptr : oy, s, y, 1, d_tau, K1, &opt, ctmp, bsrt, nullptr, st,
                              true)))
        return rc;
    if (!acf) {
        if ((rc = corr_batch_impl(ctx, ox, t, x, nullptr, nullptr, nullptr, 1, d_zero, 1, &opt, ctmp, bx0, nullptr, st,
                                  true)))
            return rc;
        if ((rc = corr_batch_impl(ctx, oy, s, y, nullptr, nullptr, nullptr, 1, d_zero, 1, &opt, ctmp, by0, nullptr, st,
                                  true)))
            return rc;
    }
    paper_finish(craw, bsrt, K1, d_perm, pos0, d_w, (int)w.size(), o0, acf, craw_x, craw_y, nsym, bx0, by0, tmp,
                 c_out, b_out, st);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, NCF_ECUDA, "paper NUFFT launch failed: %s", cudaGetErrorString(e));
    return NCF_OK;
}

}  // namespace ncf

// ----------------------------------------------------------------------------
// Plans: the analysis and tables of one evaluation, kept for repeated launches
// ----------------------------------------------------------------------------
struct ncf_plan {
    ncf_ctx *ctx = nullptr;  // used by execute/status (the context must outlive those calls)
    int device = 0;          // destroy needs no context
    ncf::Eval ev;            // the first option set; it owns the statistics
    char *pre = nullptr, *main = nullptr;
    size_t pre_cap = 0, main_cap = 0;
    // further option sets on the same data and statistics (ncf_plan_create_multi)
    std::vector<ncf::Eval> more;
    std::vector<char *> more_main;
    std::vector<size_t> more_cap;
};

// ----------------------------------------------------------------------------
// extern "C" entry points
// ----------------------------------------------------------------------------
extern "C" {

void ncf_options_default(ncf_options *o) {
    if (!o) return;
    o->kernel = NCF_GAUSSIAN;
    o->path = NCF_PATH_AUTO;
    o->precision = NCF_FP64;
    o->norm = NCF_NORM_NONE;
    o->h = 1.0;
    o->trunc_R = 0.0;
    o->tol = 0.0;
}

const char *ncf_status_string(ncf_status s) {
    switch (s) {
        case NCF_OK: return "NCF_OK";
        case NCF_EINVAL: return "NCF_EINVAL";
        case NCF_ENOTSORTED: return "NCF_ENOTSORTED";
        case NCF_EDEGENERATE: return "NCF_EDEGENERATE";
        case NCF_ENOMEM: return "NCF_ENOMEM";
        case NCF_ECUDA: return "NCF_ECUDA";
        case NCF_ETIMEOUT: return "NCF_ETIMEOUT";
        case NCF_EBUSY: return "NCF_EBUSY";
        case NCF_ENONFINITE: return "NCF_ENONFINITE";
        case NCF_EUNSUPPORTED: return "NCF_EUNSUPPORTED";
    }
    return "NCF_UNKNOWN";
}

ncf_status ncf_create(ncf_ctx **out, int device) {
    if (!out) return NCF_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return NCF_ECUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return NCF_ECUDA;
    ncf_ctx *c = new ncf_ctx();
    c->device = device;
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (cudaEventCreateWithFlags(&c->staged, cudaEventDisableTiming) != cudaSuccess) {
        delete c;
        return NCF_ECUDA;
    }
    *out = c;
    return NCF_OK;
}

void ncf_destroy(ncf_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->ws2) cudaFree(ctx->ws2);
    if (ctx->hbuf) cudaFree(ctx->hbuf);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    if (ctx->ws_alt) cudaFree(ctx->ws_alt);
    if (ctx->pinned_pre) cudaFreeHost(ctx->pinned_pre);
    if (ctx->prep_st) cudaStreamDestroy(ctx->prep_st);
    if (ctx->staged) cudaEventDestroy(ctx->staged);
    for (cudaEvent_t e : ctx->prof.pool) cudaEventDestroy(e);
    if (ctx->copy_st) cudaStreamDestroy(ctx->copy_st);
    if (ctx->back_st) cudaStreamDestroy(ctx->back_st);
    for (cudaEvent_t e : ctx->copy_ev) cudaEventDestroy(e);
    if (ctx->boot) cudaFree(ctx->boot);
    if (ctx->paper) cudaFree(ctx->paper);
    delete ctx;  // last: nothing above may touch ctx after this
}

ncf_status ncf_last_plan(const ncf_ctx *ctx, ncf_plan_info *out) {
    if (!ctx || !out) return NCF_EINVAL;
    *out = ctx->plan;
    return NCF_OK;
}

ncf_status ncf_last_tuning(const ncf_ctx *ctx, ncf_tuning *out) {
    if (!ctx || !out) return NCF_EINVAL;
    *out = ctx->tuning;
    return NCF_OK;
}

ncf_status ncf_profile_enable(ncf_ctx *ctx, int on) {
    if (!ctx) return NCF_EINVAL;
    ctx->prof.on = on != 0;
    return NCF_OK;
}

int64_t ncf_profile_report(ncf_ctx *ctx, char *buf, size_t len) {
    if (!ctx) return -1;
    NcfProfiler &p = ctx->prof;
    for (auto &r : p.recs) {
        float ms = 0.0f;
        if (cudaEventSynchronize(p.pool[r.second + 1]) == cudaSuccess &&
            cudaEventElapsedTime(&ms, p.pool[r.second], p.pool[r.second + 1]) == cudaSuccess) {
            auto &t = p.totals[r.first];
            t.first += 1;
            t.second += ms;
        } else {
            cudaGetLastError();
        }
    }
    p.recs.clear();
    p.next = 0;
    std::string out;
    char line[256];
    for (auto &kv : p.totals) {
        snprintf(line, sizeof line, "%s %lld %.6f\n", kv.first.c_str(), (long long)kv.second.first,
                 kv.second.second);
        out += line;
    }
    if (buf && len) {
        const size_t n = std::min(len - 1, out.size());
        std::memcpy(buf, out.data(), n);
        buf[n] = 0;
    }
    return (int64_t)out.size();
}

void ncf_profile_reset(ncf_ctx *ctx) {
    if (!ctx) return;
    ncf_profile_report(ctx, nullptr, 0);
    ctx->prof.totals.clear();
}

const char *ncf_last_error(const ncf_ctx *ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

uint64_t ncf_launch_count(const ncf_ctx *ctx) { return ctx ? ctx->launches : 0; }

size_t ncf_device_bytes(const ncf_ctx *ctx) { return ctx ? std::max(ctx->dev_hwm, ncf::ctx_device_bytes(ctx)) : 0; }

ncf_status ncf_corr(ncf_ctx *ctx, const double *t, const double *x, int64_t nx, const double *s,
                    const double *y, int64_t ny, const double *lags, int64_t K, const ncf_options *opt,
                    double *c_out, double *b_out, int64_t *count_out, void *stream) {
    if (!ctx) return NCF_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return NCF_ECUDA;
    const int64_t ox[2] = {0, nx};
    const int64_t oy[2] = {0, ny};
    const bool acf = (s == nullptr && y == nullptr);
    return ncf::corr_batch_impl(ctx, ox, t, x, acf ? nullptr : oy, s, y, 1, lags, K, opt, c_out, b_out,
                                count_out, (cudaStream_t)stream);
}

ncf_status ncf_corr_pooled(ncf_ctx *ctx, const double *t, const double *x, int64_t nx, const double *s,
                           const double *y, int64_t ny, const double *lags, int64_t K, const ncf_options *opt,
                           const ncf_pooled_stats *pooled, double *c_out, double *b_out, int64_t *count_out,
                           void *stream) {
    if (!ctx) return NCF_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return NCF_ECUDA;
    if (!pooled) return ncf::fail(ctx, NCF_EINVAL, "pooled statistics are NULL");
    const bool acf = (s == nullptr && y == nullptr);
    auto bad = [](double m, double sd, int64_t n) { return !std::isfinite(m) || !(sd > 0.0) || !std::isfinite(sd) || n < 2; };
    if (bad(pooled->mean_x, pooled->std_x, pooled->n_x) || (!acf && bad(pooled->mean_y, pooled->std_y, pooled->n_y)))
        return ncf::fail(ctx, NCF_EINVAL, "pooled statistics need finite means, std > 0 and n >= 2");
    if (opt && opt->norm != NCF_NORM_NONE)
        return ncf::fail(ctx, NCF_EUNSUPPORTED, "pooled statistics: NORM_NONE only (normalise after the reduction)");
    const int64_t ox[2] = {0, nx};
    const int64_t oy[2] = {0, ny};
    return ncf::corr_batch_impl(ctx, ox, t, x, acf ? nullptr : oy, s, y, 1, lags, K, opt, c_out, b_out,
                                count_out, (cudaStream_t)stream, false, pooled);
}

ncf_status ncf_series_stats(ncf_ctx *ctx, const double *t, const double *x, int64_t n, ncf_series_summary *out,
                            void *stream) {
    using namespace ncf;
    if (!ctx || !t || !x || !out || n < 1) return NCF_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return NCF_ECUDA;
    LaunchScope scope(ctx);
    ctx->err.clear();
    cudaStream_t st = (cudaStream_t)stream;
    if (ctx->staged) NCF_CUDA(cudaEventSynchronize(ctx->staged));
    Eval ev;
    const int64_t offs[2] = {0, n};
    ev.B = 1;
    plan_side(ev.X, offs, 1);
    ev.X.t = t;
    ev.X.v = x;
    ncf_status rc;
    if ((rc = grow(ctx, &ctx->ws, &ctx->ws_cap, pre_bytes(ev), st))) return rc;
    carve_pre(ev, ctx->ws);
    if ((rc = grow_pinned(ctx, 4096, st))) return rc;
    int64_t *hp = reinterpret_cast<int64_t *>(ctx->pinned);
    hp[0] = 0; hp[1] = n;
    hp[2] = 0; hp[3] = ev.X.n_chunks;
    NCF_CUDA(cudaMemcpyAsync(ev.X.d_offs, hp, 16, cudaMemcpyHostToDevice, st));
    NCF_CUDA(cudaMemcpyAsync(ev.X.d_chunk_base, hp + 2, 16, cudaMemcpyHostToDevice, st));
    launch_chunk_series(ev.X.d_chunk_base, 1, ev.X.d_cs, st);
    run_stats(ev, st);
    auto *hs = reinterpret_cast<SeriesStats *>(ctx->pinned + 256);
    NCF_CUDA(cudaMemcpyAsync(hs, ev.X.d_stats, sizeof(SeriesStats), cudaMemcpyDeviceToHost, st));
    NCF_CUDA(cudaStreamSynchronize(st));
    out->n = n;
    out->mean = hs->mean;
    out->m2 = hs->inv_std > 0.0 ? (double)n / (hs->inv_std * hs->inv_std) : 0.0;
    out->t_first = hs->t_first;
    out->t_last = hs->t_last;
    out->flags = hs->flags & ~STAT_DEGENERATE;
    return NCF_OK;
}

ncf_status ncf_corr_paper(ncf_ctx *ctx, const double *t, const double *x, int64_t nx, const double *s,
                          const double *y, int64_t ny, const double *lags, int64_t K, ncf_kernel kernel, double h,
                          int64_t N1, double *c_out, double *b_out, void *stream) {
    if (!ctx) return NCF_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return NCF_ECUDA;
    return ncf::corr_paper_impl(ctx, t, x, nx, s, y, ny, lags, K, kernel, h, N1, c_out, b_out,
                                (cudaStream_t)stream);
}

ncf_status ncf_corr_batch(ncf_ctx *ctx, const int64_t *offs_x, const double *t, const double *x,
                          const int64_t *offs_y, const double *s, const double *y, int64_t B,
                          const double *lags, int64_t K, const ncf_options *opt, double *c_out,
                          double *b_out, int64_t *count_out, void *stream) {
    if (!ctx) return NCF_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return NCF_ECUDA;
    return ncf::corr_batch_impl(ctx, offs_x, t, x, offs_y, s, y, B, lags, K, opt, c_out, b_out, count_out,
                                (cudaStream_t)stream);
}

ncf_status ncf_selftest_bounded_wait(ncf_ctx *ctx, void *stream, int32_t *flags) {
    if (!ctx || !flags) return NCF_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return NCF_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    ncf::LaunchScope scope(ctx);
    ncf_status rc = ncf::grow(ctx, &ctx->ws, &ctx->ws_cap, 256, st);
    if (rc) return rc;
    int *dstat = reinterpret_cast<int *>(ctx->ws);
    if (cudaMemsetAsync(dstat, 0, sizeof(int), st) != cudaSuccess) return NCF_ECUDA;
    ncf::launch_bounded_wait_selftest(dstat, st);
    int h = 0;
    if (cudaMemcpyAsync(&h, dstat, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return ncf::fail(ctx, NCF_ECUDA, "bounded-wait self-test: %s", cudaGetErrorString(cudaGetLastError()));
    *flags = h;
    return (h & ncf::STATUS_TIMEOUT) ? NCF_OK : ncf::fail(ctx, NCF_ECUDA, "bounded wait did not report a timeout");
}

ncf_status ncf_corr_bootstrap(ncf_ctx *ctx, const double *t, const double *x, int64_t nx, const double *s,
                              const double *y, int64_t ny, const double *lags, int64_t K, const ncf_options *opt,
                              int64_t n_boot, uint64_t seed, double *c_out, double *b_out, int64_t *count_out,
                              void *stream) {
    using ncf::al;
    if (!ctx) return NCF_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return NCF_ECUDA;
    const bool acf = (s == nullptr && y == nullptr);
    if (!t || !x || !lags || !c_out || !opt || nx < 2 || K < 1 || n_boot < 1 || (!acf && (!s || !y || ny < 2)) ||
        nx >= ((int64_t)1 << 32) || ny >= ((int64_t)1 << 32) || n_boot >= ((int64_t)1 << 32)) {
        ctx->err = "ncf_corr_bootstrap: NULL pointer, fewer than 2 points, no lags, no replicate, or a size "
                   "of 2^32 or more";
        return NCF_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nyy = acf ? 0 : ny;
    const size_t need = al((size_t)(nx * n_boot) * 8) * 2 + al((size_t)(nyy * n_boot) * 8) * 2 +
                        al((size_t)(std::max(nx, nyy) * n_boot) * 4);
    ncf::LaunchScope scope(ctx);
    ncf_status rc = ncf::grow(ctx, &ctx->boot, &ctx->boot_cap, need, st);
    if (rc) return rc;
    char *p = ctx->boot;
    auto take = [&](size_t bytes) { char *q = p; p += al(bytes); return q; };
    double *bt = reinterpret_cast<double *>(take((size_t)(nx * n_boot) * 8));
    double *bx = reinterpret_cast<double *>(take((size_t)(nx * n_boot) * 8));
    double *bs = acf ? nullptr : reinterpret_cast<double *>(take((size_t)(nyy * n_boot) * 8));
    double *by = acf ? nullptr : reinterpret_cast<double *>(take((size_t)(nyy * n_boot) * 8));
    int32_t *cnt = reinterpret_cast<int32_t *>(take((size_t)(std::max(nx, nyy) * n_boot) * 4));
    // the y side draws from its own stream, seed XOR all-ones
    ncf::launch_bootstrap(t, x, nx, n_boot, seed, cnt, bt, bx, ctx->sm_count, st);
    if (!acf) ncf::launch_bootstrap(s, y, ny, n_boot, ~seed, cnt, bs, by, ctx->sm_count, st);
    if (cudaGetLastError() != cudaSuccess) return ncf::fail(ctx, NCF_ECUDA, "bootstrap kernels failed to launch");
    std::vector<int64_t> ox(n_boot + 1), oy(acf ? 0 : n_boot + 1);
    for (int64_t r = 0; r <= n_boot; ++r) {
        ox[r] = r * nx;
        if (!acf) oy[r] = r * ny;
    }
    return ncf::corr_batch_impl(ctx, ox.data(), bt, bx, acf ? nullptr : oy.data(), bs, by, n_boot, lags, K, opt,
                                c_out, b_out, count_out, st);
}

ncf_status ncf_corr_regular(ncf_ctx *ctx, const int64_t *m_x, const double *x, int64_t nx, const int64_t *m_y,
                            const double *y, int64_t ny, double dt, const double *lags, int64_t K,
                            const ncf_options *opt, double *c_out, double *b_out, int64_t *count_out, void *stream) {
    if (!ctx) return NCF_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return NCF_ECUDA;
    const bool ccf = m_y != nullptr || y != nullptr;
    if (!m_x || !x || !lags || !c_out || !opt || nx < 2 || K < 1 || (ccf && (!m_y || !y || ny < 2)) ||
        !(dt > 0.0) || !std::isfinite(dt) || !(opt->h > 0.0) || !std::isfinite(opt->h) ||
        (opt->kernel != NCF_GAUSSIAN && opt->kernel != NCF_RECTANGLE && opt->kernel != NCF_HANNING) ||
        (opt->norm != NCF_NORM_NONE && opt->norm != NCF_NORM_LAG0)) {
        ctx->err = "ncf_corr_regular: NULL pointer, fewer than 2 points, no lags, dt or h not positive, or an "
                   "unknown kernel or normalisation";
        return NCF_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    ncf::LaunchScope scope(ctx);
    ncf_status rc;
    if ((rc = ncf::grow(ctx, &ctx->ws, &ctx->ws_cap, ncf::regular_stats_bytes(), st))) return rc;
    if ((rc = ncf::grow_pinned(ctx, std::max<size_t>(4096, (size_t)K * 8), st))) return rc;
    // the lags' reach sizes the lattice: read them back with the statistics
    std::vector<double> hl(K);
    if (cudaMemcpyAsync(hl.data(), lags, K * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return ncf::fail(ctx, NCF_ECUDA, "ncf_corr_regular: reading the lags failed");
    std::string msg;
    int64_t m0 = 0, m1 = 0;
    rc = ncf::regular_stats(m_x, x, nx, ccf ? m_y : nullptr, y, ny, ctx->ws, ctx->pinned, &m0, &m1, st, &msg);
    if (rc) return ncf::fail(ctx, rc, "%s", msg.c_str());
    double max_tau = 0.0;
    for (double v : hl) {
        if (!std::isfinite(v)) return ncf::fail(ctx, NCF_EINVAL, "ncf_corr_regular: non-finite lag");
        max_tau = std::max(max_tau, std::fabs(v));
    }
    const double reach = opt->kernel == NCF_GAUSSIAN ? 8.0 * opt->h : opt->h;
    const int lg = ncf::regular_lg(m1 - m0, max_tau, reach, dt);
    if (lg == 0) return ncf::fail(ctx, NCF_EUNSUPPORTED, "ncf_corr_regular: lattice span plus lag reach over 2^29");
    if ((rc = ncf::grow(ctx, &ctx->ws2, &ctx->ws2_cap, ncf::regular_workspace_bytes(lg, ccf, K), st))) return rc;
    rc = ncf::regular_launch(m_x, x, nx, ccf ? m_y : nullptr, y, ny, ctx->ws, m0, lg, dt, lags, K, opt->kernel,
                             opt->h, opt->norm == NCF_NORM_LAG0, ctx->ws2, c_out, b_out, count_out, st, &msg);
    if (rc) return ncf::fail(ctx, rc, "%s", msg.c_str());
    return NCF_OK;
}

}  // extern "C"

namespace ncf {

// The host-buffer calls: one upload of the batch, then n_opts evaluations of it
// (each option set its own result buffers), chunk by chunk.
// growth factor of the host-buffer calls' chunk sizes; the copies (about 55 GB/s)
// stay ahead of the evaluation as long as it is below the ratio of the
// evaluation's time to the upload's (3.2 on the light-curve batch)
constexpr int64_t kChunkGrowth = 3;
static int64_t ipow(int64_t b, int e) {
    int64_t r = 1;
    while (e-- > 0) r *= b;
    return r;
}

static ncf_status host_batch(ncf_ctx *ctx, const int64_t *offs_x, const double *t, const double *x,
                             const int64_t *offs_y, const double *s, const double *y, int64_t B,
                             const double *lags, int64_t K, const ncf_options *opts, int n_opts,
                             double *const *c_out, double *const *b_out, int64_t *const *count_out,
                             cudaStream_t st, const char *who) {
    ctx->err.clear();
    if (!offs_x || B < 1 || K < 1 || !t || !x || !lags || !opts || n_opts < 1 || !c_out) {
        ctx->err = std::string(who) + ": NULL pointer, empty batch or no option set";
        return NCF_EINVAL;
    }
    for (int o = 0; o < n_opts; ++o)
        if (!c_out[o]) {
            ctx->err = std::string(who) + ": c_out of option set " + std::to_string(o) + " is NULL";
            return NCF_EINVAL;
        }
    const bool acf = (s == nullptr && y == nullptr);
    if (!acf && (!s || !y || !offs_y)) {
        ctx->err = std::string(who) + ": CCF needs s, y and offs_y";
        return NCF_EINVAL;
    }
    const int64_t nx = offs_x[B], ny = acf ? 0 : offs_y[B];
    const size_t need = al(nx * 8) * 2 + al(ny * 8) * 2 + al(K * 8) + (size_t)n_opts * al(B * K * 8) * 3;
    ncf_status rc = grow(ctx, &ctx->hbuf, &ctx->hbuf_cap, need, st);
    if (rc) return rc;
    Arena ar{ctx->hbuf, ctx->hbuf_cap, 0};
    double *dt = ar.take<double>(nx), *dx = ar.take<double>(nx);
    double *ds = acf ? nullptr : ar.take<double>(ny), *dy = acf ? nullptr : ar.take<double>(ny);
    double *dl = ar.take<double>(K);
    std::vector<double *> dc(n_opts), db(n_opts);
    std::vector<int64_t *> dn(n_opts);
    for (int o = 0; o < n_opts; ++o) {
        dc[o] = ar.take<double>(B * K);
        db[o] = ar.take<double>(B * K);
        dn[o] = ar.take<int64_t>(B * K);
    }
    auto bo = [&](int o) { return b_out ? b_out[o] : nullptr; };
    auto no = [&](int o) { return count_out ? count_out[o] : nullptr; };
    // Large batches run as up to five chunks of series: every chunk's upload is
    // queued at once on the copy stream, so the link streams the whole batch
    // without a pause, and chunk i's evaluation (the caller's stream) starts when
    // its own upload has landed; each chunk's results come back on a third stream
    // while the next chunk runs.  Chunk sizes triple (1/121, 3/121, ..., 81/121 of
    // the points; kChunkGrowth): only the first, small upload waits with nothing
    // to overlap.  The
    // evaluations' own small transfers (statistics read-back, table uploads) go
    // through copy_pinned, a kernel, so they never wait behind the bulk uploads
    // on the copy engines.  Chunk i + 1's statistics stage (pass, read-back and
    // the host's wait for it) runs on a fourth stream while chunk i's evaluation
    // is on the GPU, so the host prepares chunk i + 1 with no gap on the device;
    // consecutive chunks take turns with two pre-statistics workspaces.  Pinned
    // host buffers are needed for the copies to overlap.
    const int64_t pts = nx + ny;
    const int C = (int)std::min<int64_t>(B, pts * 16 > (int64_t)(256 << 20) ? 5 : 1);
    std::vector<int64_t> cut(C + 1, B);
    cut[0] = 0;
    for (int c = 1; c < C; ++c) {
        const int64_t target = pts * (ipow(kChunkGrowth, c) - 1) / (ipow(kChunkGrowth, C) - 1);
        int64_t b = cut[c - 1];
        while (b < B && offs_x[b] + (acf ? 0 : offs_y[b]) < target) ++b;
        cut[c] = std::max(b, cut[c - 1]);
    }
    if (!ctx->copy_st && cudaStreamCreateWithFlags(&ctx->copy_st, cudaStreamNonBlocking) != cudaSuccess)
        return fail(ctx, NCF_ECUDA, "%s: copy stream creation failed", who);
    if (!ctx->back_st && cudaStreamCreateWithFlags(&ctx->back_st, cudaStreamNonBlocking) != cudaSuccess)
        return fail(ctx, NCF_ECUDA, "%s: copy stream creation failed", who);
    if (!ctx->prep_st && cudaStreamCreateWithFlags(&ctx->prep_st, cudaStreamNonBlocking) != cudaSuccess)
        return fail(ctx, NCF_ECUDA, "%s: stream creation failed", who);
    while ((int)ctx->copy_ev.size() < 2 * C + 2) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return fail(ctx, NCF_ECUDA, "%s: event creation failed", who);
        ctx->copy_ev.push_back(e);
    }
    cudaStream_t cs = ctx->copy_st, rs = ctx->back_st, ps = ctx->prep_st;
    cudaEvent_t *ev_in = ctx->copy_ev.data(), *ev_out = ev_in + C, ev_start = ev_in[2 * C], ev_pre = ev_in[2 * C + 1];
    // the copy and statistics streams start after the work already queued on the caller's stream
    bool ok = cudaEventRecord(ev_start, st) == cudaSuccess && cudaStreamWaitEvent(cs, ev_start, 0) == cudaSuccess &&
              cudaStreamWaitEvent(rs, ev_start, 0) == cudaSuccess &&
              cudaStreamWaitEvent(ps, ev_start, 0) == cudaSuccess;
    auto upload = [&](int c) {
        const int64_t b0 = cut[c], b1 = cut[c + 1];
        const int64_t x0 = offs_x[b0], x1 = offs_x[b1];
        bool k = cudaMemcpyAsync(dt + x0, t + x0, (x1 - x0) * 8, cudaMemcpyHostToDevice, cs) == cudaSuccess &&
                 cudaMemcpyAsync(dx + x0, x + x0, (x1 - x0) * 8, cudaMemcpyHostToDevice, cs) == cudaSuccess;
        if (!acf) {
            const int64_t y0 = offs_y[b0], y1 = offs_y[b1];
            k = k && cudaMemcpyAsync(ds + y0, s + y0, (y1 - y0) * 8, cudaMemcpyHostToDevice, cs) == cudaSuccess &&
                cudaMemcpyAsync(dy + y0, y + y0, (y1 - y0) * 8, cudaMemcpyHostToDevice, cs) == cudaSuccess;
        }
        return k && cudaEventRecord(ev_in[c], cs) == cudaSuccess;
    };
    ok = ok && cudaMemcpyAsync(dl, lags, K * 8, cudaMemcpyHostToDevice, st) == cudaSuccess;
    for (int c = 0; c < C; ++c) ok = ok && upload(c);
    if (!ok) return fail(ctx, NCF_ECUDA, "host-to-device copy failed: %s", cudaGetErrorString(cudaGetLastError()));
    // chunk c's statistics stage, on the statistics stream once its upload has
    // landed and (c >= 2) chunk c - 2's evaluation, the last user of its
    // workspace, has finished
    struct Pre {
        Eval ev;
        std::vector<int> paths;
        std::vector<int64_t> ox, oy;
    };
    Pre pre[2];
    auto run_pre = [&](int c) -> ncf_status {
        const int64_t b0 = cut[c], b1 = cut[c + 1], nb = b1 - b0;
        if (nb <= 0) return NCF_OK;
        Pre &P = pre[c & 1];
        P = Pre{};
        const int64_t x0 = offs_x[b0], y0 = acf ? 0 : offs_y[b0];
        P.ox.assign(offs_x + b0, offs_x + b1 + 1);
        for (auto &v : P.ox) v -= x0;
        if (!acf) {
            P.oy.assign(offs_y + b0, offs_y + b1 + 1);
            for (auto &v : P.oy) v -= y0;
        }
        if (cudaStreamWaitEvent(ps, ev_in[c], 0) != cudaSuccess ||
            (c >= 2 && cudaStreamWaitEvent(ps, ev_out[c - 2], 0) != cudaSuccess))
            return fail(ctx, NCF_ECUDA, "%s: stream wait failed", who);
        std::vector<double *> cc(n_opts);
        for (int o = 0; o < n_opts; ++o) cc[o] = dc[o] + b0 * K;
        return batch_pre(ctx, P.ox.data(), dt + x0, dx + x0, acf ? nullptr : P.oy.data(), acf ? nullptr : ds + y0,
                         acf ? nullptr : dy + y0, nb, dl, K, opts, n_opts, cc.data(), P.ev, P.paths,
                         (c & 1) ? &ctx->ws_alt : &ctx->ws, (c & 1) ? &ctx->ws_alt_cap : &ctx->ws_cap, true, ps);
    };
    auto bail = [&](ncf_status r) {
        cudaStreamSynchronize(cs);
        cudaStreamSynchronize(rs);
        cudaStreamSynchronize(ps);
        return r;
    };
    // the lags go up on the caller's stream; the statistics stages read them too
    if (!ok || cudaEventRecord(ev_pre, st) != cudaSuccess || cudaStreamWaitEvent(ps, ev_pre, 0) != cudaSuccess)
        return bail(fail(ctx, NCF_ECUDA, "%s: stream wait failed", who));
    {
        LaunchScope scope(ctx);
        if ((rc = run_pre(0))) return bail(rc);
    }
    for (int c = 0; c < C; ++c) {
        const int64_t b0 = cut[c], b1 = cut[c + 1], nb = b1 - b0;
        if (nb > 0) {
            LaunchScope scope(ctx);
            // the evaluation waits for its statistics stage
            if (cudaEventRecord(ev_pre, ps) != cudaSuccess || cudaStreamWaitEvent(st, ev_pre, 0) != cudaSuccess)
                return bail(fail(ctx, NCF_ECUDA, "%s: stream wait failed", who));
            std::vector<double *> cc(n_opts), bb(n_opts);
            std::vector<int64_t *> nn(n_opts);
            for (int o = 0; o < n_opts; ++o) {
                cc[o] = dc[o] + b0 * K;
                bb[o] = bo(o) ? db[o] + b0 * K : nullptr;
                nn[o] = no(o) ? dn[o] + b0 * K : nullptr;
            }
            // one statistics pass for every option set of the chunk
            rc = batch_main(ctx, pre[c & 1].ev, pre[c & 1].paths, dl, opts, n_opts, cc.data(), bb.data(), nn.data(),
                            st);
            if (rc) return bail(rc);
        }
        ok = cudaEventRecord(ev_out[c], st) == cudaSuccess;
        ok = ok && cudaStreamWaitEvent(rs, ev_out[c], 0) == cudaSuccess;
        auto d2h = [&](void *h, const void *d) {
            return cudaMemcpyAsync(h, d, nb * K * 8, cudaMemcpyDeviceToHost, rs) == cudaSuccess;
        };
        for (int o = 0; o < n_opts && nb > 0; ++o)
            ok = ok && d2h(c_out[o] + b0 * K, dc[o] + b0 * K) && (!bo(o) || d2h(bo(o) + b0 * K, db[o] + b0 * K)) &&
                 (!no(o) || d2h(no(o) + b0 * K, dn[o] + b0 * K));
        if (!ok) break;
        if (c + 1 < C) {  // the next chunk's statistics, beside this chunk's evaluation
            LaunchScope scope(ctx);
            if ((rc = run_pre(c + 1))) return bail(rc);
        }
    }
    if (!ok || cudaStreamSynchronize(cs) != cudaSuccess || cudaStreamSynchronize(rs) != cudaSuccess ||
        cudaStreamSynchronize(ps) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
        ctx->err = std::string("copy failed: ") + cudaGetErrorString(cudaGetLastError());
        return NCF_ECUDA;
    }
    return NCF_OK;
}

}  // namespace ncf

extern "C" {

ncf_status ncf_corr_batch_host(ncf_ctx *ctx, const int64_t *offs_x, const double *t, const double *x,
                               const int64_t *offs_y, const double *s, const double *y, int64_t B,
                               const double *lags, int64_t K, const ncf_options *opt, double *c_out,
                               double *b_out, int64_t *count_out, void *stream) {
    if (!ctx) return NCF_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return NCF_ECUDA;
    return ncf::host_batch(ctx, offs_x, t, x, offs_y, s, y, B, lags, K, opt, 1, &c_out, &b_out, &count_out,
                           (cudaStream_t)stream, "ncf_corr_batch_host");
}

ncf_status ncf_corr_batch_multi(ncf_ctx *ctx, const int64_t *offs_x, const double *t, const double *x,
                                const int64_t *offs_y, const double *s, const double *y, int64_t B,
                                const double *lags, int64_t K, const ncf_options *opts, int n_opts,
                                double *const *c_out, double *const *b_out, int64_t *const *count_out,
                                void *stream) {
    if (!ctx) return NCF_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return NCF_ECUDA;
    return ncf::corr_batch_multi_impl(ctx, offs_x, t, x, offs_y, s, y, B, lags, K, opts, n_opts, c_out, b_out,
                                      count_out, (cudaStream_t)stream);
}

ncf_status ncf_corr_batch_host_multi(ncf_ctx *ctx, const int64_t *offs_x, const double *t, const double *x,
                                     const int64_t *offs_y, const double *s, const double *y, int64_t B,
                                     const double *lags, int64_t K, const ncf_options *opts, int n_opts,
                                     double *const *c_out, double *const *b_out, int64_t *const *count_out,
                                     void *stream) {
    if (!ctx) return NCF_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return NCF_ECUDA;
    return ncf::host_batch(ctx, offs_x, t, x, offs_y, s, y, B, lags, K, opts, n_opts, c_out, b_out, count_out,
                           (cudaStream_t)stream, "ncf_corr_batch_host_multi");
}

ncf_status ncf_plan_create_multi(ncf_ctx *ctx, const int64_t *offs_x, const double *t, const double *x,
                                 const int64_t *offs_y, const double *s, const double *y, int64_t B,
                                 const double *lags, int64_t K, const ncf_options *opts, int n_opts, void *stream,
                                 ncf_plan **out) {
    using namespace ncf;
    if (!ctx || !out) return NCF_EINVAL;
    *out = nullptr;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return NCF_ECUDA;
    LaunchScope scope(ctx);
    ctx->err.clear();
    if (!opts || n_opts < 1) return fail(ctx, NCF_EINVAL, "no option set");
    cudaStream_t st = (cudaStream_t)stream;
    if (ctx->staged) NCF_CUDA(cudaEventSynchronize(ctx->staged));
    ncf_plan *p = new ncf_plan();
    p->ctx = ctx;
    p->device = ctx->device;
    Eval &ev = p->ev;
    auto bail = [&](ncf_status rc) {
        if (p->pre) cudaFree(p->pre);
        if (p->main) cudaFree(p->main);
        for (char *m : p->more_main) if (m) cudaFree(m);
        delete p;
        return rc;
    };
    ncf_status rc = check_args(ctx, offs_x, t, x, offs_y, s, y, B, lags, K, &opts[0], ev);
    if (rc) return bail(rc);
    std::vector<int> paths(n_opts);
    for (int o = 0; o < n_opts; ++o)
        if ((rc = check_options(ctx, &opts[o], B, K, &paths[o]))) return bail(rc);
    ev.X.t = t; ev.X.v = x;
    if (!ev.acf) { ev.Y.t = s; ev.Y.v = y; }
    p->pre_cap = pre_bytes(ev);
    if (cudaMalloc(&p->pre, p->pre_cap) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(ctx, NCF_ENOMEM, "cudaMalloc of %zu bytes failed", p->pre_cap));
    }
    carve_pre(ev, p->pre);
    if ((rc = analyze(ctx, ev, lags, st))) return bail(rc);
    // option sets 1.. share the sides, their statistics and the lags of set 0
    for (int o = 1; o < n_opts; ++o) {
        Eval eo = ev;
        eo.opt = opts[o];
        eo.path = paths[o];
        eo.lag0 = opts[o].norm == NCF_NORM_LAG0;
        p->more.push_back(eo);
        p->more_main.push_back(nullptr);
        p->more_cap.push_back(0);
    }
    for (int o = 0; o < n_opts; ++o) {
        Eval &eo = o == 0 ? ev : p->more[o - 1];
        char *&mem = o == 0 ? p->main : p->more_main[o - 1];
        size_t &cap = o == 0 ? p->main_cap : p->more_cap[o - 1];
        choose_path(eo);
        size_t dev = 0, pin = 0;
        if ((rc = main_bytes(ctx, eo, &dev, &pin))) return bail(rc);
        cap = dev;
        if (cudaMalloc(&mem, dev) != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(ctx, NCF_ENOMEM, "cudaMalloc of %zu bytes failed", dev));
        }
        if ((rc = grow_pinned(ctx, pin, st))) return bail(rc);
        if ((rc = prepare(ctx, eo, mem, dev, ctx->pinned, ctx->pinned_cap, lags, st))) return bail(rc);
        if (rect_scan(eo) && (rc = tune_rect(ctx, eo, st))) return bail(rc);
        if ((rc = tune_spectral(ctx, eo, st))) return bail(rc);
        // the pinned staging is reused by the next option set's tables
        if (cudaStreamSynchronize(st) != cudaSuccess) return bail(fail(ctx, NCF_ECUDA, "plan set-up failed"));
    }
    *out = p;
    return NCF_OK;
}

ncf_status ncf_plan_create(ncf_ctx *ctx, const int64_t *offs_x, const double *t, const double *x,
                           const int64_t *offs_y, const double *s, const double *y, int64_t B,
                           const double *lags, int64_t K, const ncf_options *opt, void *stream,
                           ncf_plan **out) {
    if (!opt) {
        if (ctx) ctx->err = "options are NULL";
        return NCF_EINVAL;
    }
    return ncf_plan_create_multi(ctx, offs_x, t, x, offs_y, s, y, B, lags, K, opt, 1, stream, out);
}

ncf_status ncf_plan_execute(ncf_plan *plan, const double *t, const double *x, const double *s,
                            const double *y, double *c_out, double *b_out, int64_t *count_out,
                            void *stream) {
    using namespace ncf;
    if (!plan || !t || !x || !c_out) return NCF_EINVAL;
    ncf_ctx *ctx = plan->ctx;
    Eval &ev = plan->ev;
    if (!ev.acf && (!s || !y)) return fail(ctx, NCF_EINVAL, "this plan is a CCF: s and y are needed");
    LaunchScope scope(ctx);
    ev.X.t = t; ev.X.v = x;
    if (!ev.acf) { ev.Y.t = s; ev.Y.v = y; }
    return launch(ctx, ev, /*stats_fresh=*/false, /*guard=*/true, c_out, b_out, count_out, (cudaStream_t)stream);
}

ncf_status ncf_plan_execute_multi(ncf_plan *plan, const double *t, const double *x, const double *s,
                                  const double *y, double *const *c_out, double *const *b_out,
                                  int64_t *const *count_out, void *stream) {
    using namespace ncf;
    if (!plan || !t || !x || !c_out) return NCF_EINVAL;
    ncf_ctx *ctx = plan->ctx;
    const int n = 1 + (int)plan->more.size();
    for (int o = 0; o < n; ++o)
        if (!c_out[o]) return fail(ctx, NCF_EINVAL, "c_out of option set %d is NULL", o);
    if (!plan->ev.acf && (!s || !y)) return fail(ctx, NCF_EINVAL, "this plan is a CCF: s and y are needed");
    LaunchScope scope(ctx);
    cudaStream_t st = (cudaStream_t)stream;
    for (int o = 0; o < n; ++o) {
        Eval &ev = o == 0 ? plan->ev : plan->more[o - 1];
        ev.X.t = t; ev.X.v = x;
        if (!ev.acf) { ev.Y.t = s; ev.Y.v = y; }
        // one statistics pass (set 0) for every option set
        ncf_status rc = launch(ctx, ev, /*stats_fresh=*/o > 0, /*guard=*/true, c_out[o], b_out ? b_out[o] : nullptr,
                               count_out ? count_out[o] : nullptr, st, /*first=*/o == 0);
        if (rc) return rc;
    }
    return NCF_OK;
}

int ncf_plan_option_sets(const ncf_plan *plan) { return plan ? 1 + (int)plan->more.size() : 0; }

ncf_status ncf_plan_status(ncf_plan *plan, void *stream, int32_t *flags) {
    if (!plan || !flags) return NCF_EINVAL;
    int v = 0;
    if (cudaMemcpyAsync(&v, plan->ev.status, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream) !=
            cudaSuccess ||
        cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return NCF_ECUDA;
    }
    *flags = v;
    if (v & ncf::STATUS_TIMEOUT) return NCF_ETIMEOUT;
    if (v & ncf::STATUS_INPUT) return NCF_EINVAL;
    if (v != 0) return NCF_EUNSUPPORTED;
    return NCF_OK;
}

size_t ncf_plan_device_bytes(const ncf_plan *plan) {
    if (!plan) return 0;
    size_t b = plan->pre_cap + plan->main_cap;
    for (size_t c : plan->more_cap) b += c;
    return b;
}

ncf_status ncf_workspace_bytes(ncf_ctx *ctx, int64_t n_x, int64_t n_y, int64_t B, int64_t K, double span,
                               double max_abs_lag, const ncf_options *opt, size_t *device_bytes,
                               size_t *pinned_bytes) {
    using namespace ncf;
    if (ctx) ctx->err.clear();
    if (!device_bytes) return fail(ctx, NCF_EINVAL, "device_bytes is NULL");
    *device_bytes = 0;
    if (pinned_bytes) *pinned_bytes = 0;
    int path = 0;
    ncf_status rc = check_options(ctx, opt, B, K, &path);
    if (rc) return rc;
    const bool acf = n_y == 0;
    if (n_x < 2 * B || (!acf && n_y < 2 * B))
        return fail(ctx, NCF_EINVAL, "n_x = %lld, n_y = %lld: every series needs >= 2 points", (long long)n_x,
                    (long long)n_y);
    if (!(span >= 0.0) || !std::isfinite(span) || !(max_abs_lag >= 0.0) || !std::isfinite(max_abs_lag))
        return fail(ctx, NCF_EINVAL, "span and max_abs_lag must be finite and >= 0");
    Eval ev;
    ev.acf = acf;
    ev.B = B;
    ev.K = K;
    ev.opt = *opt;
    ev.lag0 = opt->norm == NCF_NORM_LAG0;
    bound_side(ev.X, n_x, B);
    if (!acf) bound_side(ev.Y, n_y, B);
    // every series spans `span` (the spectral grid grows with the largest span)
    SeriesStats st{};
    st.t_first = 0.0;
    st.t_last = span;
    st.n = 2;
    ev.X.stats.assign(B, st);
    if (!acf) ev.Y.stats.assign(B, st);
    ev.lagv.assign(K, max_abs_lag);
    ev.max_tau = max_abs_lag;
    ev.t_abs = span;
    const size_t pre = pre_bytes(ev);
    const size_t analyze_pin = al((B + 1) * 8) * 4 + al(B * sizeof(SeriesStats)) * 2 + al(K * 8);
    // the FP64 Gaussian's path is chosen from the data: the larger of both paths
    std::vector<int> paths;
    if (path == NCF_PATH_AUTO) paths = {NCF_PATH_WINDOWED, NCF_PATH_SPECTRAL};
    else paths = {path};
    size_t dev = 0, pin = analyze_pin;
    for (int pth : paths) {
        ev.path = pth;
        size_t d = 0, p = 0;
        if ((rc = main_bytes(ctx, ev, &d, &p))) return rc;
        // a spectral batch of mixed spans may be split into grid-size buckets:
        // no more device memory than one grid, a little more host staging
        if (pth == NCF_PATH_SPECTRAL) p += spectral_bucket_pinned_allowance(B, K, n_x, acf ? 0 : n_y, !acf);
        dev = std::max(dev, d);
        pin = std::max(pin, p);
    }
    *device_bytes = pre + dev;
    if (pinned_bytes) *pinned_bytes = pin;
    return NCF_OK;
}

void ncf_plan_destroy(ncf_plan *plan) {
    if (!plan) return;
    cudaSetDevice(plan->device);
    cudaDeviceSynchronize();
    if (plan->pre) cudaFree(plan->pre);
    if (plan->main) cudaFree(plan->main);
    for (char *m : plan->more_main) if (m) cudaFree(m);
    delete plan;
}

}  // extern "C"
