// k_static.cu -- ncf_corr_window_static: the Gaussian windowed estimator for
// one series (or one pair) with no device allocation at all.
//
// Who needs it: programs that may not call cudaMalloc once they are running,
// e.g. a real-time or embedded pipeline whose device memory is planned at
// start-up, or a plug-in living inside a framework whose own caching
// allocator owns the device memory.  The regular entry points keep a
// per-context workspace that grows with cudaMalloc; this one instead uses a
// fixed scratch array compiled into the library (kStaticScratchBytes bytes
// on every GPU that loads the library, held until the process exits).
//
// The scratch array's name, used in host code, is only a host-side stand-in
// for the device variable: handing it to a kernel would fault, or on systems
// where the GPU can reach host memory silently use the wrong memory.  Its
// device address is therefore fetched with cudaGetSymbolAddress, once per
// device, by the first call made while that device is current.  Every call shares the same
// array and the array keeps the last call's contents: the accumulators are
// cleared at the start of each call, and calls that overlap on the GPU (two
// streams, two threads) race on it.
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace ncf {
namespace {

constexpr int64_t kStaticMaxPoints = 262144;   // per series
constexpr int64_t kStaticMaxLags = 1024;
constexpr size_t kStaticScratchBytes = 64 * 1024;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// scratch layout (byte offsets)
constexpr size_t al256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr int64_t kMaxChunks = (kStaticMaxPoints + kPrepChunk - 1) / kPrepChunk;
constexpr int64_t kMaxTiles = kStaticMaxPoints / 512 + 1;
constexpr size_t kOffOffs = 0;                                               // 4 x int64: offs x, offs y
constexpr size_t kOffChunkBase = kOffOffs + al256(4 * 8);                    // 4 x int64
constexpr size_t kOffPart = kOffChunkBase + al256(4 * 8);                    // 2 x kMaxChunks partials
constexpr size_t kOffStats = kOffPart + al256(2 * kMaxChunks * sizeof(ChunkPartial));
constexpr size_t kOffTiles = kOffStats + al256(2 * sizeof(SeriesStats));
constexpr size_t kOffNum = kOffTiles + al256(kMaxTiles * sizeof(ScanTile));
constexpr size_t kOffDen = kOffNum + al256(kStaticMaxLags * 8);
constexpr size_t kOffCnt = kOffDen + al256(kStaticMaxLags * 8);
constexpr size_t kOffCs = kOffCnt + al256(kStaticMaxLags * 8);                // 2 x kMaxChunks int32
constexpr size_t kOffEnd = kOffCs + al256(2 * kMaxChunks * 4);
static_assert(kOffEnd <= kStaticScratchBytes, "static scratch layout exceeds its array");

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_dev_ptr[kMaxDevices] = {};

// Writes the CSR offsets, chunk tables and scan tiles of one series (or
// pair) into the scratch array, so no host-built table has to be copied.
__global__ void static_setup_kernel(unsigned char *scratch, int64_t nx, int64_t ny, int tileJ) {
    auto *offs = reinterpret_cast<int64_t *>(scratch + kOffOffs);
    auto *cb = reinterpret_cast<int64_t *>(scratch + kOffChunkBase);
    auto *tiles = reinterpret_cast<ScanTile *>(scratch + kOffTiles);
    auto *cs = reinterpret_cast<int32_t *>(scratch + kOffCs);
    for (int64_t i = threadIdx.x; i < 2 * kMaxChunks; i += blockDim.x) cs[i] = 0;  // one series
    const int64_t n_out = ny > 0 ? ny : nx;
    const int64_t nt = (n_out + tileJ - 1) / tileJ;
    for (int64_t i = threadIdx.x; i < nt; i += blockDim.x)
        tiles[i] = ScanTile{0, 0, i * tileJ, min((i + 1) * tileJ, n_out)};
    if (threadIdx.x == 0) {
        offs[0] = 0; offs[1] = nx; offs[2] = 0; offs[3] = ny;
        cb[0] = 0; cb[1] = (nx + kPrepChunk - 1) / kPrepChunk;
        cb[2] = 0; cb[3] = (ny + kPrepChunk - 1) / kPrepChunk;
    }
}

ncf_status scratch_for_current_device(unsigned char **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return NCF_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return NCF_ECUDA;
        }
        g_dev_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_dev_ptr[dev];
    return NCF_OK;
}

}  // namespace
}  // namespace ncf

extern "C" ncf_status ncf_corr_window_static(const double *t, const double *x, int64_t nx,
                                             const double *s, const double *y, int64_t ny,
                                             const double *lags, int64_t K, double h, double trunc_R,
                                             double *c_out, double *b_out, void *stream) {
    using namespace ncf;
    const bool acf = (s == nullptr && y == nullptr);
    if (!t || !x || !lags || !c_out || (!acf && (!s || !y))) return NCF_EINVAL;
    if (nx < 2 || (!acf && ny < 2) || K < 1 || !(h > 0.0) || !(trunc_R >= 0.0)) return NCF_EINVAL;
    if (nx > kStaticMaxPoints || (!acf && ny > kStaticMaxPoints) || K > kStaticMaxLags)
        return NCF_EUNSUPPORTED;  // beyond the fixed scratch: use ncf_corr
    unsigned char *sc = nullptr;
    ncf_status rc = scratch_for_current_device(&sc);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    auto *offs = reinterpret_cast<int64_t *>(sc + kOffOffs);
    auto *cb = reinterpret_cast<int64_t *>(sc + kOffChunkBase);
    auto *part = reinterpret_cast<ChunkPartial *>(sc + kOffPart);
    auto *stats = reinterpret_cast<SeriesStats *>(sc + kOffStats);
    auto *tiles = reinterpret_cast<ScanTile *>(sc + kOffTiles);
    auto *num = reinterpret_cast<double *>(sc + kOffNum);
    auto *den = reinterpret_cast<double *>(sc + kOffDen);
    auto *cnt = reinterpret_cast<unsigned long long *>(sc + kOffCnt);
    auto *cs = reinterpret_cast<int32_t *>(sc + kOffCs);
    const int tileJ = scan_tile_points();
    const int64_t n_out = acf ? nx : ny;
    NCF_LAUNCH("static_setup_kernel", st, static_setup_kernel<<<1, 256, 0, st>>>(sc, nx, acf ? 0 : ny, tileJ));
    const int64_t chx = (nx + kPrepChunk - 1) / kPrepChunk, chy = (ny + kPrepChunk - 1) / kPrepChunk;
    launch_stats_chunks(t, x, offs, cb, cs, chx, kPrepChunk, part, st);
    launch_stats_finish(t, x, offs, cb, 1, part, stats, st);
    if (!acf) {
        launch_stats_chunks(s, y, offs + 2, cb + 2, cs + kMaxChunks, chy, kPrepChunk, part + kMaxChunks, st);
        launch_stats_finish(s, y, offs + 2, cb + 2, 1, part + kMaxChunks, stats + 1, st);
    }
    // validation: read the two statistics records back into host stack memory
    SeriesStats hs[2];
    std::memset(hs, 0, sizeof hs);
    if (cudaMemcpyAsync(hs, stats, (acf ? 1 : 2) * sizeof(SeriesStats), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return NCF_ECUDA;
    }
    for (int q = 0; q < (acf ? 1 : 2); ++q) {
        if (hs[q].flags & STAT_NONFINITE) return NCF_ENONFINITE;
        if (hs[q].flags & STAT_UNSORTED) return NCF_ENOTSORTED;
        if (hs[q].flags & STAT_DEGENERATE) return NCF_EDEGENERATE;
    }
    // the accumulators keep the previous call's sums: clear them
    if (cudaMemsetAsync(num, 0, K * 8, st) != cudaSuccess || cudaMemsetAsync(den, 0, K * 8, st) != cudaSuccess ||
        cudaMemsetAsync(cnt, 0, K * 8, st) != cudaSuccess) {
        cudaGetLastError();
        return NCF_ECUDA;
    }
    const double R = trunc_R > 0.0 ? trunc_R : 8.0;
    const int64_t n_tiles = (n_out + tileJ - 1) / tileJ;
    launch_gauss_window(t, x, offs, stats, acf ? t : s, acf ? x : y, acf ? stats : stats + 1, tiles,
                        n_tiles, lags, K, acf ? +1 : -1, h, R * h, 0, num, den, cnt, st);
    launch_finish_gauss(num, den, cnt, 1, K, nullptr, nullptr, c_out, b_out, nullptr, st);
    if (cudaGetLastError() != cudaSuccess) return NCF_ECUDA;
    return NCF_OK;
}
