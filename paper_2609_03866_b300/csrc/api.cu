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
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "spectral.cuh"

#include <map>

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
    char *hbuf = nullptr;        // device copies of host inputs (ncf_corr_batch_host)
    size_t hbuf_cap = 0;
    uint64_t launches = 0;
    cudaEvent_t staged = nullptr;  // recorded after staging copies issued past the read-back sync
    NcfProfiler prof;
    ncf_plan_info plan{0.0, 0, 0, 0, 0, 0};
    std::string err;
};

static thread_local ncf_ctx *tls_ctx = nullptr;

namespace ncf {
LaunchMark::LaunchMark(const char *name, cudaStream_t s) : slot(-1), st(s) {
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
}
}  // namespace ncf

namespace ncf {
namespace {

struct LaunchScope {
    explicit LaunchScope(ncf_ctx *c) { tls_ctx = c; }
    ~LaunchScope() { tls_ctx = nullptr; }
};

ncf_status fail(ncf_ctx *ctx, ncf_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ctx->err = buf;
    return s;
}

#define NCF_CUDA(call)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(ctx, NCF_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

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
    return NCF_OK;
}

ncf_status grow_pinned(ncf_ctx *ctx, size_t need, cudaStream_t st) {
    if (need <= ctx->pinned_cap) return NCF_OK;
    size_t ncap = std::max(need, ctx->pinned_cap * 2);
    if (ctx->pinned) {
        NCF_CUDA(cudaStreamSynchronize(st));
        NCF_CUDA(cudaFreeHost(ctx->pinned));
        ctx->pinned = nullptr;
        ctx->pinned_cap = 0;
    }
    if (cudaHostAlloc(&ctx->pinned, ncap, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        ctx->pinned = nullptr;
        return fail(ctx, NCF_ENOMEM, "cudaHostAlloc of %zu bytes failed", ncap);
    }
    ctx->pinned_cap = ncap;
    return NCF_OK;
}

size_t al(size_t b) { return (b + 255) & ~size_t(255); }

// One side (x or y) of a batch: device arrays plus host-side chunking.
struct Side {
    const double *t = nullptr, *v = nullptr;
    std::vector<int64_t> offs, chunk_base;
    int64_t n_total = 0, n_chunks = 0, n_max = 0;
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

FixedScales choose_scales(double m_abs, int64_t n_max) {
    FixedScales fs;
    int e = 0;
    std::frexp(std::max(m_abs, 1e-300), &e);  // m_abs < 2^e
    fs.q = std::max(-1000, std::min(1000, 60 - e));
    fs.tscale = std::ldexp(1.0, fs.q);
    // two FP64 roundings of magnitude <= m_abs, plus three floor() truncations
    fs.eta = 4 + (int64_t)std::ldexp(1.0, e - 52 + fs.q);
    const double lg = 1.5 * std::log2((double)std::max<int64_t>(n_max, 2));
    fs.p = std::max(8, std::min(40, (int)std::floor(61.0 - lg)));
    fs.vscale = std::ldexp(1.0, fs.p);
    return fs;
}

}  // namespace

// ----------------------------------------------------------------------------
// The batch driver.  All device pointers come from the caller; offsets are host.
// ----------------------------------------------------------------------------
static ncf_status corr_batch_impl(ncf_ctx *ctx, const int64_t *offs_x, const double *t,
                                  const double *x, const int64_t *offs_y, const double *s,
                                  const double *y, int64_t B, const double *lags, int64_t K,
                                  const ncf_options *opt, double *c_out, double *b_out,
                                  int64_t *count_out, cudaStream_t st) {
    LaunchScope scope(ctx);
    ctx->err.clear();
    // the pinned staging buffer may still feed a copy queued by the previous call
    if (ctx->staged) NCF_CUDA(cudaEventSynchronize(ctx->staged));
    if (!opt) return fail(ctx, NCF_EINVAL, "options are NULL");
    if (B < 1) return fail(ctx, NCF_EINVAL, "B = %lld (need >= 1)", (long long)B);
    if (K < 1) return fail(ctx, NCF_EINVAL, "K = %lld (need >= 1)", (long long)K);
    if (!t || !x || !lags || !c_out) return fail(ctx, NCF_EINVAL, "NULL t, x, lags or c_out");
    if (!(opt->h > 0.0) || !std::isfinite(opt->h))
        return fail(ctx, NCF_EINVAL, "h = %g (need finite h > 0)", opt->h);
    if (opt->kernel != NCF_GAUSSIAN && opt->kernel != NCF_RECTANGLE)
        return fail(ctx, NCF_EINVAL, "unknown kernel %d", opt->kernel);
    if (opt->path < NCF_PATH_AUTO || opt->path > NCF_PATH_WINDOWED)
        return fail(ctx, NCF_EINVAL, "unknown path %d", opt->path);
    if (opt->precision != NCF_FP64 && opt->precision != NCF_FP32)
        return fail(ctx, NCF_EINVAL, "unknown precision %d", opt->precision);
    if (opt->norm != NCF_NORM_NONE && opt->norm != NCF_NORM_LAG0)
        return fail(ctx, NCF_EINVAL, "unknown normalisation %d", opt->norm);
    if (!(opt->trunc_R >= 0.0) || !(opt->tol >= 0.0) || opt->tol >= 1.0)
        return fail(ctx, NCF_EINVAL, "trunc_R must be >= 0 and tol in [0, 1)");
    const bool acf = (s == nullptr && y == nullptr);
    if (!acf && (!s || !y || !offs_y)) return fail(ctx, NCF_EINVAL, "CCF needs s, y and offs_y");
    ncf_status rc = check_offsets(ctx, offs_x, B, "offs_x");
    if (rc) return rc;
    if (!acf && (rc = check_offsets(ctx, offs_y, B, "offs_y"))) return rc;
    int path = opt->path;
    if (path == NCF_PATH_AUTO) path = (opt->kernel == NCF_RECTANGLE) ? NCF_PATH_WINDOWED : NCF_PATH_SPECTRAL;
    if (opt->kernel == NCF_RECTANGLE && path == NCF_PATH_SPECTRAL)
        return fail(ctx, NCF_EUNSUPPORTED,
                    "rectangle kernel: only the exact windowed scan is provided (its transform "
                    "decays as 1/f, so a truncated spectrum cannot meet the tolerance)");

    Side X, Y;
    X.t = t; X.v = x;
    plan_side(X, offs_x, B);
    if (!acf) { Y.t = s; Y.v = y; plan_side(Y, offs_y, B); }
    Side &O = acf ? X : Y;  // outer side (j): y for a CCF, x itself for an ACF
    const int tileJ = scan_tile_points();
    std::vector<ScanTile> tiles = make_tiles(O.offs, B, tileJ);
    const int64_t n_tiles = (int64_t)tiles.size();

    // ---- pre-statistics workspace ----
    auto side_bytes = [&](const Side &sd) {
        return al((B + 1) * 8) * 2 + al(sd.n_chunks * sizeof(ChunkPartial)) + al(B * sizeof(SeriesStats)) +
               al(sd.n_chunks * 4);
    };
    size_t need = side_bytes(X) + (acf ? 0 : side_bytes(Y)) + al(n_tiles * sizeof(ScanTile));
    if ((rc = grow(ctx, &ctx->ws, &ctx->ws_cap, need, st))) return rc;
    Arena ar{ctx->ws, ctx->ws_cap, 0};
    auto carve = [&](Side &sd) {
        sd.d_offs = ar.take<int64_t>(B + 1);
        sd.d_chunk_base = ar.take<int64_t>(B + 1);
        sd.d_part = ar.take<ChunkPartial>(sd.n_chunks);
        sd.d_stats = ar.take<SeriesStats>(B);
        sd.d_cs = ar.take<int32_t>(sd.n_chunks);
    };
    carve(X);
    if (!acf) carve(Y);
    ScanTile *d_tiles = ar.take<ScanTile>(n_tiles);
    if (!d_tiles) return fail(ctx, NCF_ENOMEM, "internal: workspace estimate too small");

    // ---- pinned staging: uploads then read-backs ----
    const size_t up_bytes = al((B + 1) * 8) * 4 + al(n_tiles * sizeof(ScanTile));
    const size_t down_bytes = al(B * sizeof(SeriesStats)) * 2 + al(K * 8);
    if ((rc = grow_pinned(ctx, up_bytes + down_bytes, st))) return rc;
    char *hp = ctx->pinned;
    auto upload = [&](void *dst, const void *src, size_t bytes) -> ncf_status {
        std::memcpy(hp, src, bytes);
        NCF_CUDA(cudaMemcpyAsync(dst, hp, bytes, cudaMemcpyHostToDevice, st));
        hp += al(bytes);
        return NCF_OK;
    };
    if ((rc = upload(X.d_offs, X.offs.data(), (B + 1) * 8))) return rc;
    if ((rc = upload(X.d_chunk_base, X.chunk_base.data(), (B + 1) * 8))) return rc;
    if (!acf) {
        if ((rc = upload(Y.d_offs, Y.offs.data(), (B + 1) * 8))) return rc;
        if ((rc = upload(Y.d_chunk_base, Y.chunk_base.data(), (B + 1) * 8))) return rc;
    }
    if ((rc = upload(d_tiles, tiles.data(), n_tiles * sizeof(ScanTile)))) return rc;

    auto run_stats = [&](Side &sd) {
        launch_chunk_series(sd.d_chunk_base, B, sd.d_cs, st);
        launch_stats_chunks(sd.t, sd.v, sd.d_offs, sd.d_chunk_base, sd.d_cs, sd.n_chunks, kPrepChunk,
                            sd.d_part, st);
        launch_stats_finish(sd.t, sd.v, sd.d_offs, sd.d_chunk_base, B, sd.d_part, sd.d_stats, st);
    };
    run_stats(X);
    if (!acf) run_stats(Y);
    char *down = ctx->pinned + up_bytes;
    NCF_CUDA(cudaMemcpyAsync(down, X.d_stats, B * sizeof(SeriesStats), cudaMemcpyDeviceToHost, st));
    if (!acf)
        NCF_CUDA(cudaMemcpyAsync(down + al(B * sizeof(SeriesStats)), Y.d_stats, B * sizeof(SeriesStats),
                                 cudaMemcpyDeviceToHost, st));
    double *h_lags = reinterpret_cast<double *>(down + 2 * al(B * sizeof(SeriesStats)));
    NCF_CUDA(cudaMemcpyAsync(h_lags, lags, K * 8, cudaMemcpyDeviceToHost, st));
    NCF_CUDA(cudaStreamSynchronize(st));
    NCF_CUDA(cudaGetLastError());
    X.stats.assign(reinterpret_cast<SeriesStats *>(down), reinterpret_cast<SeriesStats *>(down) + B);
    if (!acf)
        Y.stats.assign(reinterpret_cast<SeriesStats *>(down + al(B * sizeof(SeriesStats))),
                       reinterpret_cast<SeriesStats *>(down + al(B * sizeof(SeriesStats))) + B);
    if ((rc = check_stats(ctx, X, B, acf ? "x" : "x"))) return rc;
    if (!acf && (rc = check_stats(ctx, Y, B, "y"))) return rc;
    const std::vector<double> lagv(h_lags, h_lags + K);  // the staging buffer is reused below
    double max_tau = 0.0;
    for (int64_t k = 0; k < K; ++k) {
        if (!std::isfinite(lagv[k])) return fail(ctx, NCF_ENONFINITE, "lag %lld is not finite", (long long)k);
        max_tau = std::max(max_tau, std::fabs(lagv[k]));
    }
    double t_abs = 0.0;
    for (int64_t b = 0; b < B; ++b) {
        t_abs = std::max({t_abs, std::fabs(X.stats[b].t_first), std::fabs(X.stats[b].t_last)});
        if (!acf) t_abs = std::max({t_abs, std::fabs(Y.stats[b].t_first), std::fabs(Y.stats[b].t_last)});
    }
    const bool lag0 = opt->norm == NCF_NORM_LAG0;

    if (opt->kernel == NCF_RECTANGLE) {
        // ---- exact rectangle scan on fixed-point keys ----
        const FixedScales fs = choose_scales(t_abs + max_tau + opt->h + 1.0, std::max(X.n_max, O.n_max));
        auto key_bytes = [&](const Side &sd) {
            return al(sd.n_total * 8) * 2 + al((sd.n_total + 1) * 8) + al((sd.n_chunks + 1) * 8);
        };
        const int rtile = rect_tile_points();
        auto ntiles = [&](const std::vector<int64_t> &o) {
            int64_t n = 0;
            for (int64_t b = 0; b < B; ++b) n += (o[b + 1] - o[b] + rtile - 1) / rtile;
            return n;
        };
        // independent device and staging regions for the main scan and the two lag-0 scans
        const size_t rw_main = rect_workspace_bytes(ntiles(O.offs), K);
        const size_t rw_x = lag0 ? rect_workspace_bytes(ntiles(X.offs), 1) : 0;
        const size_t rw_y = (lag0 && !acf) ? rect_workspace_bytes(ntiles(Y.offs), 1) : 0;
        const size_t rs_main = rect_staging_bytes(ntiles(O.offs), K);
        const size_t rs_x = lag0 ? rect_staging_bytes(ntiles(X.offs), 1) : 0;
        const size_t rs_y = (lag0 && !acf) ? rect_staging_bytes(ntiles(Y.offs), 1) : 0;
        size_t need2 = key_bytes(X) + (acf ? 0 : key_bytes(Y)) + al(B * K * 8) * 3 + al(B * 8) * 8 + 1024 +
                       rw_main + rw_x + rw_y;
        if ((rc = grow(ctx, &ctx->ws2, &ctx->ws2_cap, need2, st))) return rc;
        if ((rc = grow_pinned(ctx, rs_main + rs_x + rs_y, st))) return rc;
        Arena a2{ctx->ws2, ctx->ws2_cap, 0};
        struct Keys { int64_t *T, *Xq, *P, *cs; };
        auto keys = [&](Side &sd) {
            Keys kk{a2.take<int64_t>(sd.n_total), a2.take<int64_t>(sd.n_total),
                    a2.take<int64_t>(sd.n_total + 1), a2.take<int64_t>(sd.n_chunks + 1)};
            launch_keys_prefix(sd.t, sd.v, sd.d_offs, sd.d_chunk_base, sd.d_cs, sd.n_chunks, kPrepChunk,
                               sd.d_stats, fs, kk.T, kk.Xq, kk.P, kk.cs, sd.n_total, st);
            return kk;
        };
        Keys kx = keys(X);
        Keys ky = acf ? kx : keys(Y);
        auto *cnt = a2.take<unsigned long long>(B * K);
        auto *num = a2.take<unsigned long long>(2 * B * K);
        auto *cnt0 = a2.take<unsigned long long>(2 * B);
        auto *num0 = a2.take<unsigned long long>(4 * B);
        auto *scale = a2.take<double>(B);
        char *rws_main = a2.take<char>(rw_main);
        char *rws_x = lag0 ? a2.take<char>(rw_x) : nullptr;
        char *rws_y = (lag0 && !acf) ? a2.take<char>(rw_y) : nullptr;
        if (!kx.cs || !ky.cs || !scale || !rws_main || (lag0 && !rws_x) || (lag0 && !acf && !rws_y))
            return fail(ctx, NCF_ENOMEM, "internal: workspace estimate too small");
        NCF_CUDA(cudaMemsetAsync(cnt, 0, B * K * 8, st));
        NCF_CUDA(cudaMemsetAsync(num, 0, 2 * B * K * 8, st));
        const int eps = acf ? +1 : -1;
        std::string msg;
        RectArgs ra{kx.T, kx.P, X.t, X.d_offs, ky.T, ky.Xq, O.t, &O.offs, B, K, lagv.data(), eps,
                    opt->h, fs, cnt, num};
        if ((rc = run_rect_scan(ra, rws_main, rw_main, ctx->pinned, rs_main, st, &msg)))
            return fail(ctx, rc, "%s", msg.c_str());
        const double inv_v2 = std::ldexp(1.0, -2 * fs.p);
        if (lag0) {
            // ACF of each side at lag 0 (Algorithms 4 and 10): scale = c_xx(0) or sqrt(c_xx(0) c_yy(0))
            static const double zero = 0.0;
            NCF_CUDA(cudaMemsetAsync(cnt0, 0, 2 * B * 8, st));
            NCF_CUDA(cudaMemsetAsync(num0, 0, 4 * B * 8, st));
            RectArgs rx{kx.T, kx.P, X.t, X.d_offs, kx.T, kx.Xq, X.t, &X.offs, B, 1, &zero, +1, opt->h, fs,
                        cnt0, num0};
            if ((rc = run_rect_scan(rx, rws_x, rw_x, ctx->pinned + rs_main, rs_x, st, &msg)))
                return fail(ctx, rc, "%s", msg.c_str());
            if (!acf) {
                RectArgs ry{ky.T, ky.P, Y.t, Y.d_offs, ky.T, ky.Xq, Y.t, &Y.offs, B, 1, &zero, +1, opt->h,
                            fs, cnt0 + B, num0 + 2 * B};
                if ((rc = run_rect_scan(ry, rws_y, rw_y, ctx->pinned + rs_main + rs_x, rs_y, st, &msg)))
                    return fail(ctx, rc, "%s", msg.c_str());
            }
            launch_lag0_scale_rect(cnt0, num0, acf ? nullptr : cnt0 + B, acf ? nullptr : num0 + 2 * B,
                                   B, inv_v2, scale, st);
        }
        NCF_CUDA(cudaEventRecord(ctx->staged, st));
        launch_finish_rect(cnt, num, B, K, inv_v2, lag0 ? scale : nullptr, c_out, b_out, count_out, st);
        NCF_CUDA(cudaGetLastError());
        return NCF_OK;
    }

    if (path == NCF_PATH_WINDOWED) {
        // ---- Gaussian windowed FP64 scan ----
        const double R = opt->trunc_R > 0.0 ? opt->trunc_R : 8.0;
        const double Rh = R * opt->h;
        size_t need2 = al(B * K * 8) * 3 + al(B * 8) * 8 + 1024;
        if (lag0) need2 += al((X.n_total / tileJ + B) * sizeof(ScanTile)) + 256;
        if ((rc = grow(ctx, &ctx->ws2, &ctx->ws2_cap, need2, st))) return rc;
        Arena a2{ctx->ws2, ctx->ws2_cap, 0};
        auto *num = a2.take<double>(B * K);
        auto *den = a2.take<double>(B * K);
        auto *cnt = a2.take<unsigned long long>(B * K);
        auto *zero_lag = a2.take<double>(1);
        auto *n0 = a2.take<double>(2 * B);
        auto *d0 = a2.take<double>(2 * B);
        auto *c0 = a2.take<unsigned long long>(2 * B);
        auto *scale = a2.take<double>(B);
        if (!scale) return fail(ctx, NCF_ENOMEM, "internal: workspace estimate too small");
        NCF_CUDA(cudaMemsetAsync(num, 0, B * K * 8, st));
        NCF_CUDA(cudaMemsetAsync(den, 0, B * K * 8, st));
        NCF_CUDA(cudaMemsetAsync(cnt, 0, B * K * 8, st));
        const int eps = acf ? +1 : -1;
        launch_gauss_window(X.t, X.v, X.d_offs, X.d_stats, O.t, O.v, O.d_stats, d_tiles, n_tiles, lags, K,
                            eps, opt->h, Rh, num, den, cnt, st);
        if (lag0) {
            NCF_CUDA(cudaMemsetAsync(zero_lag, 0, 8, st));
            NCF_CUDA(cudaMemsetAsync(n0, 0, 2 * B * 8, st));
            NCF_CUDA(cudaMemsetAsync(d0, 0, 2 * B * 8, st));
            NCF_CUDA(cudaMemsetAsync(c0, 0, 2 * B * 8, st));
            ScanTile *tx_tiles = d_tiles;
            int64_t ntx = n_tiles;
            if (!acf) {
                std::vector<ScanTile> tt = make_tiles(X.offs, B, tileJ);
                ntx = (int64_t)tt.size();
                tx_tiles = a2.take<ScanTile>(ntx);
                if (!tx_tiles) return fail(ctx, NCF_ENOMEM, "internal: workspace estimate too small");
                if ((rc = grow_pinned(ctx, ntx * sizeof(ScanTile), st))) return rc;
                std::memcpy(ctx->pinned, tt.data(), ntx * sizeof(ScanTile));
                NCF_CUDA(cudaMemcpyAsync(tx_tiles, ctx->pinned, ntx * sizeof(ScanTile),
                                         cudaMemcpyHostToDevice, st));
                NCF_CUDA(cudaEventRecord(ctx->staged, st));
            }
            launch_gauss_window(X.t, X.v, X.d_offs, X.d_stats, X.t, X.v, X.d_stats, tx_tiles, ntx, zero_lag,
                                1, +1, opt->h, Rh, n0, d0, c0, st);
            if (!acf)
                launch_gauss_window(Y.t, Y.v, Y.d_offs, Y.d_stats, Y.t, Y.v, Y.d_stats, d_tiles, n_tiles,
                                    zero_lag, 1, +1, opt->h, Rh, n0 + B, d0 + B, c0 + B, st);
            launch_lag0_scale_gauss(n0, d0, acf ? nullptr : n0 + B, acf ? nullptr : d0 + B, B, scale, st);
        }
        launch_finish_gauss(num, den, cnt, B, K, lag0 ? scale : nullptr, c_out, b_out, count_out, st);
        NCF_CUDA(cudaGetLastError());
        return NCF_OK;
    }

    // ---- Gaussian spectral path ----
    SpectralArgs sa;
    sa.acf = acf;
    sa.B = B;
    sa.K = K;
    sa.h = opt->h;
    sa.fp32 = opt->precision == NCF_FP32;
    sa.tol = opt->tol > 0.0 ? opt->tol : (sa.fp32 ? 1e-7 : 1e-14);
    sa.max_tau = max_tau;
    sa.lag0 = lag0;
    sa.lags = lags;
    sa.h_lags = lagv.data();
    sa.x = {X.t, X.v, X.d_offs, X.d_stats, X.offs.data(), X.stats.data(), X.n_total, X.n_max,
            X.d_chunk_base, X.n_chunks, X.d_cs};
    if (!acf)
        sa.y = {Y.t, Y.v, Y.d_offs, Y.d_stats, Y.offs.data(), Y.stats.data(), Y.n_total, Y.n_max,
                Y.d_chunk_base, Y.n_chunks, Y.d_cs};
    sa.c_out = c_out;
    sa.b_out = b_out;
    sa.count_out = count_out;
    sa.sm_count = ctx->sm_count;
    std::string msg;
    SpectralGeometry geom{0.0, 0, 0, 0};
    rc = run_spectral(sa, &ctx->ws2, &ctx->ws2_cap, &ctx->pinned, &ctx->pinned_cap, st, &msg, &geom);
    if (rc) return fail(ctx, rc, "%s", msg.c_str());
    ctx->plan = ncf_plan_info{geom.L, geom.M, geom.nf, geom.W, B, K};
    NCF_CUDA(cudaEventRecord(ctx->staged, st));
    NCF_CUDA(cudaGetLastError());
    return NCF_OK;
}

}  // namespace ncf

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
    if (ctx->staged) cudaEventDestroy(ctx->staged);
    for (cudaEvent_t e : ctx->prof.pool) cudaEventDestroy(e);
    delete ctx;
}

ncf_status ncf_last_plan(const ncf_ctx *ctx, ncf_plan_info *out) {
    if (!ctx || !out) return NCF_EINVAL;
    *out = ctx->plan;
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

ncf_status ncf_corr_batch(ncf_ctx *ctx, const int64_t *offs_x, const double *t, const double *x,
                          const int64_t *offs_y, const double *s, const double *y, int64_t B,
                          const double *lags, int64_t K, const ncf_options *opt, double *c_out,
                          double *b_out, int64_t *count_out, void *stream) {
    if (!ctx) return NCF_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return NCF_ECUDA;
    return ncf::corr_batch_impl(ctx, offs_x, t, x, offs_y, s, y, B, lags, K, opt, c_out, b_out, count_out,
                                (cudaStream_t)stream);
}

ncf_status ncf_corr_batch_host(ncf_ctx *ctx, const int64_t *offs_x, const double *t, const double *x,
                               const int64_t *offs_y, const double *s, const double *y, int64_t B,
                               const double *lags, int64_t K, const ncf_options *opt, double *c_out,
                               double *b_out, int64_t *count_out, void *stream) {
    using ncf::al;
    if (!ctx) return NCF_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return NCF_ECUDA;
    if (!offs_x || B < 1 || K < 1 || !t || !x || !lags || !c_out) {
        ctx->err = "ncf_corr_batch_host: NULL pointer or empty batch";
        return NCF_EINVAL;
    }
    const bool acf = (s == nullptr && y == nullptr);
    if (!acf && (!s || !y || !offs_y)) {
        ctx->err = "ncf_corr_batch_host: CCF needs s, y and offs_y";
        return NCF_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nx = offs_x[B], ny = acf ? 0 : offs_y[B];
    const size_t need = al(nx * 8) * 2 + al(ny * 8) * 2 + al(K * 8) + al(B * K * 8) * 3;
    ncf_status rc = ncf::grow(ctx, &ctx->hbuf, &ctx->hbuf_cap, need, st);
    if (rc) return rc;
    ncf::Arena ar{ctx->hbuf, ctx->hbuf_cap, 0};
    double *dt = ar.take<double>(nx), *dx = ar.take<double>(nx);
    double *ds = acf ? nullptr : ar.take<double>(ny), *dy = acf ? nullptr : ar.take<double>(ny);
    double *dl = ar.take<double>(K);
    double *dc = ar.take<double>(B * K), *db = ar.take<double>(B * K);
    int64_t *dn = ar.take<int64_t>(B * K);
    auto h2d = [&](void *d, const void *h, size_t n) {
        return cudaMemcpyAsync(d, h, n, cudaMemcpyHostToDevice, st) == cudaSuccess;
    };
    if (!h2d(dt, t, nx * 8) || !h2d(dx, x, nx * 8) || !h2d(dl, lags, K * 8) ||
        (!acf && (!h2d(ds, s, ny * 8) || !h2d(dy, y, ny * 8)))) {
        ctx->err = std::string("host-to-device copy failed: ") + cudaGetErrorString(cudaGetLastError());
        return NCF_ECUDA;
    }
    rc = ncf::corr_batch_impl(ctx, offs_x, dt, dx, offs_y, ds, dy, B, dl, K, opt, dc, b_out ? db : nullptr,
                              count_out ? dn : nullptr, st);
    if (rc) return rc;
    auto d2h = [&](void *h, const void *d, size_t n) {
        return cudaMemcpyAsync(h, d, n, cudaMemcpyDeviceToHost, st) == cudaSuccess;
    };
    if (!d2h(c_out, dc, B * K * 8) || (b_out && !d2h(b_out, db, B * K * 8)) ||
        (count_out && !d2h(count_out, dn, B * K * 8)) || cudaStreamSynchronize(st) != cudaSuccess) {
        ctx->err = std::string("device-to-host copy failed: ") + cudaGetErrorString(cudaGetLastError());
        return NCF_ECUDA;
    }
    return NCF_OK;
}

}  // extern "C"
