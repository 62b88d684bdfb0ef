// k_rect.cu -- exact rectangle pair counts and numerators (Algorithms 6 and 8).
//
// For every outer point s_j and lag tau_k the window is
//     lo_jk = #{i : t_i <  fl(c - h)},   hi_jk = #{i : t_i <= fl(c + h)},   c = fl(s_j + e tau_k),
// count_k = sum_j (hi_jk - lo_jk) and N_k = sum_j y_j (P[hi_jk] - P[lo_jk]) with P the prefix
// sums of x (Algorithm 8).  Both are computed exactly:
//
//  * keys.  T = floor(t 2^q) (int64) is monotone in t.  The integer bound
//    S_j + e Tau_k - H differs from the scaled FP64 bound by less than eta
//    units, so a key more than eta below / at least eta above decides the
//    comparison; a key inside the band is decided by the FP64 predicate itself.
//  * numerators.  X = round(x_std 2^p), P = int64 prefix sums (wrap-around; a
//    window sum is exact whenever its value fits in 63 bits), N accumulated in
//    128-bit integers: order-independent and identical on every run.
//
// Work decomposition (B300): one CTA = one tile of 2048 consecutive outer
// points x 32 consecutive lags of the sorted lag list.  Lane l of every warp
// owns lag l of the group; warp w owns 64 consecutive outer points of the
// tile, so the 32 lanes of a warp walk the same outer points (one broadcast
// load each) with their own window pointers, which move together across
// observing gaps.  The union of the 32 windows over the tile is staged in
// shared memory as 32-bit coarse keys (T - base) >> sh plus int64 prefix
// sums; coarse comparisons are exact away from a 2-unit band, and the band
// falls back to the full keys and then to FP64.  Per-lag sums are reduced
// across warps in shared memory and added to the output with integer
// atomics.  A CTA whose union does not fit runs the same scan on global keys.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>

#include "common.cuh"

namespace ncf {

namespace {

constexpr int kRectWarps = 32;                      // outer runs per CTA
// outer points per warp run: a template parameter, chosen by the autotuner
// (rect_variant_run); 16, 32 or 64
constexpr int kRectTile = 2048;                     // outer points per CTA
constexpr int kLagGroup = 32;                       // lags per CTA (one per lane)
constexpr int kKeyCap = 10240;                      // staged window entries
constexpr int32_t kSentinel = 0x7fffffff;

struct RectRange { int64_t ia, ib; };               // staged key range [ia, ib]

struct __align__(16) RectSmem {
    int64_t sY[kRectTile];
    int64_t sP[kKeyCap + 1];
    int32_t sSc[kRectTile];
    int32_t sK[kKeyCap + 8];
    unsigned int pc[kRectWarps][32];
    unsigned long long pl[kRectWarps][32], ph[kRectWarps][32];
    int next_run;
};

__device__ __forceinline__ int64_t lower_bound64(const int64_t *__restrict__ T, int64_t lo,
                                                 int64_t hi, int64_t v) {
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (T[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ int lower_bound32(const int32_t *__restrict__ K, int lo, int hi, int32_t v) {
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (K[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// One thread per (tile, lag group): the staged key range of the CTA.
__global__ void rect_range_kernel(const int64_t *__restrict__ Tx, const int64_t *__restrict__ offs_x,
                                  const int64_t *__restrict__ Sy, const ScanTile *__restrict__ tiles,
                                  int64_t n_tiles, int G, const int64_t *__restrict__ gmin,
                                  const int64_t *__restrict__ gmax, int64_t eta,
                                  RectRange *__restrict__ ranges) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n_tiles * G) return;
    const int64_t tI = id / G;
    const int g = (int)(id - tI * G);
    const ScanTile tile = tiles[tI];
    const int64_t xa = offs_x[tile.b], xb = offs_x[tile.b + 1];
    const int64_t lo_b = Sy[tile.j0] + gmin[g] - eta;
    const int64_t hi_b = Sy[tile.j1 - 1] + gmax[g] + eta;
    const int64_t ia = lower_bound64(Tx, xa, xb, lo_b);
    const int64_t ib = lower_bound64(Tx, ia, xb, hi_b);
    ranges[id] = RectRange{ia, ib};
}

struct U128 { unsigned long long lo, hi; };
__device__ __forceinline__ void add128(U128 &a, unsigned long long lo, unsigned long long hi) {
    const unsigned long long n = a.lo + lo;
    a.hi += hi + (n < a.lo ? 1ull : 0ull);
    a.lo = n;
}
__device__ __forceinline__ void mac128(U128 &a, long long w, long long y) {
    add128(a, (unsigned long long)w * (unsigned long long)y, (unsigned long long)__mul64hi(w, y));
}

// Coarse pointer advance in shared memory: the first index >= p whose key is
// not below `bound`.  Two keys per step for the common short move; a long
// move (the outer point crossed an observing gap) gallops, then bisects.
// sK holds sentinels at nK .. nK + 7, and the answer is <= nK.
__device__ __forceinline__ int advance32(const int32_t *__restrict__ sK, int p, int nK, int32_t bound,
                                         int32_t &key) {
    const int32_t k0 = sK[p], k1 = sK[p + 1];
    const int a = k0 < bound, b = k1 < bound;
    p += a + (a & b);
    key = a ? k1 : k0;  // the key at the returned position (short move)
    if (a & b) {
        int step = 4;
        for (;;) {
            const int idx = min(p + step - 1, nK);
            if (sK[idx] < bound) {
                p = idx + 1;
                step <<= 1;
            } else {
                p = lower_bound32(sK, p, idx, bound);
                key = sK[p];
                return p;
            }
        }
    }
    return p;
}

// FP64 predicates of Algorithm 6 on the caller's own values.
__device__ __forceinline__ double centre(double s, double tau, int eps) {
    return __dadd_rn(s, eps > 0 ? tau : -tau);
}

template <int kRun>
__global__ void __launch_bounds__(kRectWarps * 32, 1)
rect_scan_kernel(const int64_t *__restrict__ Tx, const int64_t *__restrict__ P,
                 const double *__restrict__ tx, const int64_t *__restrict__ offs_x,
                 const int64_t *__restrict__ Sy, const int64_t *__restrict__ Yq,
                 const double *__restrict__ sy, const ScanTile *__restrict__ tiles, int G,
                 const RectRange *__restrict__ ranges, const double *__restrict__ slags,
                 const int32_t *__restrict__ perm, const int64_t *__restrict__ dls,
                 const int64_t *__restrict__ dus, const int64_t *__restrict__ gmin,
                 const int64_t *__restrict__ gmax, int64_t K, int eps,
                 double h, int64_t eta, unsigned long long *__restrict__ cnt,
                 unsigned long long *__restrict__ num128) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RectSmem &sm = *reinterpret_cast<RectSmem *>(smem_raw);
    const int64_t tI = blockIdx.x / G;
    const int g = (int)(blockIdx.x - tI * G);
    const ScanTile tile = tiles[tI];
    const RectRange rg = ranges[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tid = threadIdx.x;
    const int64_t xa = offs_x[tile.b], xb = offs_x[tile.b + 1];
    (void)xa;
    const int tn = (int)(tile.j1 - tile.j0);
    const int64_t S0 = Sy[tile.j0];
    const int64_t base = S0 + gmin[g] - eta;      // <= every lower band edge of the CTA
    const int64_t ia = rg.ia, ib = min(rg.ib, xb);
    const int64_t lim = min(rg.ib + 1, xb);       // every pointer stays < lim (or == xb)
    const int64_t t_last = min(rg.ib, xb - 1);
    const int nK = (int)(t_last - ia + 1);
    const bool staged = nK + 0 <= kKeyCap && (ib - ia + 1) <= kKeyCap + 1;
    // coarse shift: all coarse values of the CTA below 2^29
    const int64_t span = (Sy[tile.j1 - 1] - S0) + (gmax[g] - gmin[g]) + 4 * eta + 16;
    int sh = 0;
    {
        const int64_t mag = max(span, (int64_t)1);
        const int bits = 64 - __clzll((unsigned long long)mag);
        sh = max(0, bits - 28);
    }
#pragma unroll 2
    for (int i = tid; i < tn; i += blockDim.x) {
        sm.sY[i] = Yq[tile.j0 + i];
        sm.sSc[i] = (int32_t)((Sy[tile.j0 + i] - S0) >> sh);
    }
    if (staged) {
#pragma unroll 4
        for (int i = tid; i < nK; i += blockDim.x) {
            const int64_t v = (Tx[ia + i] - base) >> sh;
            sm.sK[i] = (int32_t)min(v, (int64_t)(1 << 30));
        }
        if (tid < 8) sm.sK[nK + tid] = kSentinel;
    }
    if (tid == 0) sm.next_run = 0;
    if (staged) {
#pragma unroll 4
        for (int i = tid; i <= (int)(ib - ia); i += blockDim.x) sm.sP[i] = P[ia + i];
    }
    __syncthreads();

    const int64_t k = (int64_t)g * kLagGroup + lane;
    const bool active = k < K;
    const int64_t kk = active ? k : (int64_t)g * kLagGroup;
    const double tau = slags[kk];
    const int64_t dl = dls[kk], du = dus[kk];
    // per-lane coarse offsets (see the header): L - eta - base = (sSc + dlc) 2^sh + [0, 2^(sh+1))
    const int32_t dlc = (int32_t)((S0 + dl - eta - base) >> sh);
    const int32_t dlc2 = (int32_t)((S0 + dl + eta - base) >> sh) + 2;
    const int32_t duc = (int32_t)((S0 + du - eta - base) >> sh);
    const int32_t duc2 = (int32_t)((S0 + du + eta - base) >> sh) + 2;
    unsigned int c = 0;
    U128 acc{0ull, 0ull};
    // runs of kRun outer points are handed out dynamically, so warps whose
    // runs cross observing gaps do not hold the others at the barrier
    for (;;) {
        int r0 = 0;
        if (lane == 0) r0 = atomicAdd(&sm.next_run, 1) * kRun;
        r0 = __shfl_sync(0xffffffffu, r0, 0);
        if (r0 >= tn) break;
        const int r1 = min(r0 + kRun, tn);
        if (!active) continue;
        if (staged) {
            const int32_t *sK = sm.sK;
            int lo = lower_bound32(sK, 0, nK, sm.sSc[r0] + dlc);
            int hi = lower_bound32(sK, lo, nK, sm.sSc[r0] + duc);
            for (int r = r0; r < r1; ++r) {
                const int32_t sc = sm.sSc[r];
                const int32_t La = sc + dlc, Ua = sc + duc;
                int32_t klo, khi;
                lo = advance32(sK, lo, nK, La, klo);
                if (klo < sc + dlc2) {  // inside the coarse band: full keys, then FP64
                    const int64_t j = tile.j0 + r;
                    const int64_t Lf = Sy[j] + dl;
                    const double lb = __dsub_rn(centre(sy[j], tau, eps), h);
                    int64_t p = ia + lo;
                    while (p < lim && Tx[p] < Lf + eta && (Tx[p] < Lf - eta || tx[p] < lb)) ++p;
                    lo = (int)(p - ia);
                }
                if (hi < lo) hi = lo;
                hi = advance32(sK, hi, nK, Ua, khi);
                if (khi < sc + duc2) {
                    const int64_t j = tile.j0 + r;
                    const int64_t Uf = Sy[j] + du;
                    const double ub = __dadd_rn(centre(sy[j], tau, eps), h);
                    int64_t p = ia + hi;
                    while (p < lim && Tx[p] < Uf + eta && (Tx[p] < Uf - eta || tx[p] <= ub)) ++p;
                    hi = (int)(p - ia);
                }
                c += (unsigned int)(hi - lo);
                const long long w = (long long)((unsigned long long)sm.sP[hi] - (unsigned long long)sm.sP[lo]);
                mac128(acc, w, sm.sY[r]);
            }
        } else {
            // the union does not fit: the same scan on the global full keys
            const int64_t j0 = tile.j0 + r0;
            int64_t lo = lower_bound64(Tx, ia, lim, Sy[j0] + dl - eta);
            int64_t hi = lo;
            for (int r = r0; r < r1; ++r) {
                const int64_t j = tile.j0 + r;
                const int64_t Lf = Sy[j] + dl, Uf = Sy[j] + du;
                while (lo < lim && Tx[lo] < Lf - eta) ++lo;
                if (lo < lim && Tx[lo] < Lf + eta) {
                    const double lb = __dsub_rn(centre(sy[j], tau, eps), h);
                    while (lo < lim && Tx[lo] < Lf + eta && tx[lo] < lb) ++lo;
                }
                if (hi < lo) hi = lo;
                while (hi < lim && Tx[hi] < Uf - eta) ++hi;
                if (hi < lim && Tx[hi] < Uf + eta) {
                    const double ub = __dadd_rn(centre(sy[j], tau, eps), h);
                    while (hi < lim && Tx[hi] < Uf + eta && tx[hi] <= ub) ++hi;
                }
                c += (unsigned int)(hi - lo);
                const long long w = (long long)((unsigned long long)P[hi] - (unsigned long long)P[lo]);
                mac128(acc, w, sm.sY[r]);
            }
        }
    }
    sm.pc[warp][lane] = c;
    sm.pl[warp][lane] = acc.lo;
    sm.ph[warp][lane] = acc.hi;
    __syncthreads();
    if (warp == 0 && active) {
        unsigned long long cs = 0;
        U128 a{0ull, 0ull};
        for (int w = 0; w < kRectWarps; ++w) {
            cs += sm.pc[w][lane];
            add128(a, sm.pl[w][lane], sm.ph[w][lane]);
        }
        const int64_t slot = (int64_t)tile.b * K + (perm ? perm[k] : k);
        atomicAdd(cnt + slot, cs);
        const unsigned long long old = atomicAdd(num128 + 2 * slot, a.lo);
        const unsigned long long carry = (old + a.lo < old) ? 1ull : 0ull;
        atomicAdd(num128 + 2 * slot + 1, a.hi + carry);
    }
}

size_t al(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

int rect_tile_points() { return kRectTile; }

size_t rect_workspace_bytes(int64_t n_tiles, int64_t K) {
    const int64_t G = (K + kLagGroup - 1) / kLagGroup;
    return al(n_tiles * sizeof(ScanTile)) + al(n_tiles * G * sizeof(RectRange)) + al(K * 8) * 3 +
           al(K * 4) + al(G * 8) * 2 + 1024;
}

size_t rect_staging_bytes(int64_t n_tiles, int64_t K) {
    const int64_t G = (K + kLagGroup - 1) / kLagGroup;
    return al(n_tiles * sizeof(ScanTile)) + al(K * 8) * 3 + al(K * 4) + al(G * 8) * 2 + 1024;
}

int64_t rect_tiles_of(const std::vector<int64_t> &offs, int64_t B) {
    int64_t n = 0;
    for (int64_t b = 0; b < B; ++b) n += (offs[b + 1] - offs[b] + kRectTile - 1) / kRectTile;
    return n;
}

// Host tables of one rectangle scan -> device region `ws`: tiles of outer
// points, the sorted lags with their integer offsets, and the lag groups.
ncf_status rect_prepare(const RectArgs &a, char *ws, size_t ws_cap, char *pinned, size_t pinned_cap,
                        cudaStream_t st, RectPrepared *out, std::string *msg) {
    const int64_t B = a.B, K = a.K;
    const int64_t G = (K + kLagGroup - 1) / kLagGroup;
    std::vector<ScanTile> tiles;
    for (int64_t b = 0; b < B; ++b)
        for (int64_t j = (*a.outer_offs)[b]; j < (*a.outer_offs)[b + 1]; j += kRectTile)
            tiles.push_back(ScanTile{(int32_t)b, 0, j, std::min(j + kRectTile, (*a.outer_offs)[b + 1])});
    const int64_t n_tiles = (int64_t)tiles.size();
    // lags sorted ascending so a group's windows form one compact union
    std::vector<int32_t> perm(K);
    std::iota(perm.begin(), perm.end(), 0);
    std::stable_sort(perm.begin(), perm.end(), [&](int32_t p, int32_t q) { return a.h_lags[p] < a.h_lags[q]; });
    std::vector<double> slags(K);
    std::vector<int64_t> dls(K), dus(K), gmin(G), gmax(G);
    const int64_t H = (int64_t)std::floor(a.h * a.fs.tscale);
    for (int64_t k = 0; k < K; ++k) {
        slags[k] = a.h_lags[perm[k]];
        const int64_t Tau = (int64_t)std::floor(slags[k] * a.fs.tscale);
        const int64_t e = a.eps > 0 ? Tau : -Tau;
        dls[k] = e - H;
        dus[k] = e + H;
    }
    for (int64_t g = 0; g < G; ++g) {
        int64_t lo = INT64_MAX, hi = INT64_MIN;
        for (int64_t k = g * kLagGroup; k < std::min(K, (g + 1) * kLagGroup); ++k) {
            lo = std::min(lo, dls[k]);
            hi = std::max(hi, dus[k]);
        }
        gmin[g] = lo;
        gmax[g] = hi;
    }
    if (rect_workspace_bytes(n_tiles, K) > ws_cap || rect_staging_bytes(n_tiles, K) > pinned_cap) {
        *msg = "internal: rectangle workspace estimate too small";
        return NCF_ENOMEM;
    }
    size_t used = 0, off = 0;
    auto take = [&](size_t bytes) { char *p = ws + used; used += al(bytes); return p; };
    auto up = [&](void *dst, const void *src, size_t bytes) {
        std::memcpy(pinned + off, src, bytes);
        cudaMemcpyAsync(dst, pinned + off, bytes, cudaMemcpyHostToDevice, st);
        off += al(bytes);
    };
    RectPrepared r;
    r.n_tiles = n_tiles;
    r.G = G;
    r.tiles = take(n_tiles * sizeof(ScanTile));
    r.ranges = take(n_tiles * G * sizeof(RectRange));
    r.slags = reinterpret_cast<double *>(take(K * 8));
    r.dls = reinterpret_cast<int64_t *>(take(K * 8));
    r.dus = reinterpret_cast<int64_t *>(take(K * 8));
    r.perm = reinterpret_cast<int32_t *>(take(K * 4));
    r.gmin = reinterpret_cast<int64_t *>(take(G * 8));
    r.gmax = reinterpret_cast<int64_t *>(take(G * 8));
    up(r.tiles, tiles.data(), n_tiles * sizeof(ScanTile));
    up(r.slags, slags.data(), K * 8);
    up(r.dls, dls.data(), K * 8);
    up(r.dus, dus.data(), K * 8);
    up(r.perm, perm.data(), K * 4);
    up(r.gmin, gmin.data(), G * 8);
    up(r.gmax, gmax.data(), G * 8);
    *out = r;
    return NCF_OK;
}

// The data-dependent part: key ranges of every (tile, lag group), then the scan.
ncf_status rect_launch(const RectArgs &a, const RectPrepared &r, cudaStream_t st, std::string *msg) {
    const int64_t nr = r.n_tiles * r.G;
    auto *tiles = reinterpret_cast<const ScanTile *>(r.tiles);
    auto *ranges = reinterpret_cast<RectRange *>(r.ranges);
    NCF_LAUNCH("rect_range_kernel", st,
               rect_range_kernel<<<(unsigned)((nr + 255) / 256), 256, 0, st>>>(
                   a.Tx, a.offs_x, a.Sy, tiles, r.n_tiles, (int)r.G, r.gmin, r.gmax, a.fs.eta, ranges));
    static bool attr_set = false;
    const size_t smem = sizeof(RectSmem);
    if (!attr_set) {
        cudaFuncSetAttribute(rect_scan_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(rect_scan_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(rect_scan_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr_set = true;
    }
#define NCF_RECT_SCAN(RUN)                                                                              \
    NCF_LAUNCH("rect_scan_kernel", st,                                                                 \
               rect_scan_kernel<RUN><<<(unsigned)nr, kRectWarps * 32, smem, st>>>(                     \
                   a.Tx, a.P, a.tx, a.offs_x, a.Sy, a.Yq, a.sy, tiles, (int)r.G, ranges, r.slags, r.perm, \
                   r.dls, r.dus, r.gmin, r.gmax, a.K, a.eps, a.h, a.fs.eta, a.cnt, a.num128))
    switch (r.variant) {
        case 0: NCF_RECT_SCAN(16); break;
        case 2: NCF_RECT_SCAN(64); break;
        default: NCF_RECT_SCAN(32); break;
    }
#undef NCF_RECT_SCAN
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        *msg = std::string("rectangle scan launch failed: ") + cudaGetErrorString(e);
        return NCF_ECUDA;
    }
    return NCF_OK;
}

}  // namespace ncf
