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
//  * numerators.  X = round(x_std 2^p) with p the value bits of the series side
//    (value_bits of its length), P = int64 prefix sums (wrap-around; a
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
#include <climits>
#include <cstddef>
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

// ---------------------------------------------------------------------------
// Points-on-lanes scan.  Lane l of warp w owns the outer points
// ((b 8 + w) 4 + i) 32 + l (b < 2, i < 4) of the tile, so at every step the 32 lanes
// of a warp hold 32 consecutive outer points: their window edges sit at neighbouring
// positions of the staged keys (conflict-free shared-memory access) and the
// loop over the lags of the group is warp-uniform.  A window edge is found in
// O(1): a rank table over uniform bins of the coarse key range gives the first
// key of the edge's bin, and a short walk inside the bin finishes.  The group's
// lags are split into sub-groups whose key union fits the staging area.  When a
// single lag's union does not fit, the tile's outer points are split into
// segments (at the widest time gap, else in the middle) and each segment is
// planned again; a lag whose single-point window fills half the staging area
// runs on the global keys.
//
// Staged entries.  Entry i of a sub-group holds the coarse key of window point
// ia + i (relative to the segment's smallest query) and the prefix sum
// P[ia + i] as three limbs p0, p1 (21 bits, unsigned) and p2 = P >> 42 (22 bits,
// signed), so one 16-byte load at a window edge yields both the key the edge
// search compares and the prefix sum the numerator needs.
//
// Numerators.  With p <= 61 - 1.5 log2(n) for each series side and |x_std| <= sqrt(n) the
// quantised values satisfy |Y| < 2^61 and every window sum |w| < 2^62.  The
// limb differences of w = P[hi] - P[lo] are d0, d1 in (-2^21, 2^21) and d2 (the
// top-limb difference taken modulo 2^22, exact because |w| < 2^62), and
// Y = y1 2^31 + y0 (y0 in [0, 2^31), |y1| < 2^30), so the six 32 x 32 -> 64-bit
// products y_a d_b are below 2^52 each; they are accumulated in six int64 sums
// (2^11 items of headroom, 8 are used) and combined to 128 bits once per
// (lane, lag), then reduced across the warp.  Lane k of each warp keeps lag k's
// running sum.
// ---------------------------------------------------------------------------
constexpr int kPtWarps = 8;
constexpr int kPtM = kRectTile / (kPtWarps * 32);  // outer points per lane
constexpr int kPtBatch = 2;                         // points of a lane handled together (load ILP)
// Lane l of warp w owns point ((b kPtWarps + w) kPtBatch + i) 32 + l of the tile for
// slot q = b kPtBatch + i: the kPtBatch slots of a batch are 32 kPtBatch consecutive
// points (their windows tend to be empty together, so the batch is skipped whole),
// and each warp's batches are spread over the tile.
__device__ __forceinline__ constexpr int pt_off(int q) {
    return (q / kPtBatch) * (kPtWarps * kPtBatch * 32) + (q % kPtBatch) * 32;
}
__device__ __forceinline__ constexpr int pt_base(int warp, int lane) { return warp * kPtBatch * 32 + lane; }
constexpr int kPtCap = 4915;                        // staged entries per sub-group
constexpr int kPtSamples = 1024;                    // planning samples of a lag group's key range
constexpr int kPtExact = 16;                        // sample stride up to which the bounds stay coarse
// rank-table bins; with the staging area, the shared memory of two CTAs per SM.
// On the bench batch's rectangle plan (histogram-built table): 10240 bins and
// 5430 entries 78.5 ms, 12288 and 5170 77.9 ms, 14336 and 4915 77.1 ms, 16384 and
// 4650 84.1 ms (finer bins shorten the walks; a smaller staging area means more
// sub-groups, and below about 4900 entries more split segments)
constexpr int kPtBins = 14336;
constexpr int kPtWords = kPtBins / 2 / (kPtWarps * 32);  // 32-bit words of the rank table per thread
static_assert(kPtWords * 2 * kPtWarps * 32 == kPtBins && kPtWords % 4 == 0, "whole 16-byte rows per thread");
static_assert(kPtBins % (kPtWarps * 32) == 0, "bins split evenly over the threads");
static_assert(kPtCap + 1 <= 65535, "rank-table entries are 16-bit entry indices");
static_assert(kPtM % kPtBatch == 0, "whole batches");
static_assert(8 * kPtSamples <= 16 * (kPtCap + 1), "planning samples fit the staging area");

struct PtSub {
    int ka, kb, global, pad;
    int64_t ia, ib, dmin, dmax;
};

struct __align__(16) PtSmem {
    int4 sE[kPtCap + 1];                // {key, p0, p1, p2}; entry nK carries the sentinel key
    uint16_t sT[kPtBins];               // index in sE of the bin's first entry
    int4 lc[kLagGroup];                 // lag offsets relative to vmin: dlc, dlc2, duc, duc2
    int64_t klo[kLagGroup], khi[kLagGroup];
    int64_t kdl[kLagGroup], kdu[kLagGroup];
    PtSub sub[kLagGroup];
    int2 seg[16];                       // stack of outer-point segments [pa, pb) still to do
    int n_sub, n_seg;
    unsigned int pc[kPtWarps][32];
    unsigned long long pl[kPtWarps][32], ph[kPtWarps][32];
};
constexpr unsigned kOffE = offsetof(PtSmem, sE);
constexpr unsigned kOffT = offsetof(PtSmem, sT);
// two CTAs per SM: 228 KB of shared memory, 1 KB of it reserved per CTA
static_assert(2 * (sizeof(PtSmem) + 1024) <= 228 * 1024, "two CTAs per SM");

// Loads at 32-bit addresses of the shared window.  Indexing shared memory
// through a generic byte pointer makes the compiler form 64-bit addresses (an
// add with carry per access); the lag loop addresses its staged entries and
// rank table this way instead.  volatile keeps them in program order, after the
// barrier that publishes the staged data.
__device__ __forceinline__ int4 lds_v4(uint32_t a) {
    int4 v;
    asm volatile("ld.shared.v4.s32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    return v;
}
__device__ __forceinline__ int32_t lds_s32(uint32_t a) {
    int32_t v;
    asm volatile("ld.shared.s32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t lds_u16(uint32_t a) {
    unsigned short v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(a));
    return v;
}
// Bin of a value v in [0, R] of a sub-group's query range: floor(v mult / 2^32),
// with mult chosen so that the kPtBins bins span [0, R] exactly (a power-of-two
// shift would leave up to half of them unused).  Monotone in v, so every key in
// a lower bin than a query's is below the query.
__device__ __forceinline__ uint32_t pt_bin(int32_t v, uint32_t mult) {
    return __umulhi((uint32_t)max(v, 0), mult);
}
__host__ __device__ __forceinline__ uint32_t pt_bin_mult(int32_t R) {
    return R + 1 <= kPtBins ? 0xffffffffu : (uint32_t)(((uint64_t)kPtBins << 32) / (uint64_t)(R + 1));
}
// shared address of the rank-table entry of query v (v >= 0)
__device__ __forceinline__ uint32_t pt_bin_addr(uint32_t aT, int32_t v, uint32_t mult) {
    return aT + (__umulhi((uint32_t)v, mult) << 1);
}

// Bounds of lower_bound(Tx, ia, ib, v) from the planning samples samp[m] =
// Tx[ia + m stride], m < ns: lo <= answer <= hi with hi - lo < stride.  Past
// kPtExact the bracket is closed by a binary search on the global keys.
__device__ __forceinline__ void pt_bracket(const int64_t *samp, int ns, int64_t stride,
                                           const int64_t *__restrict__ Tx, int64_t ia, int64_t ib,
                                           int64_t v, int64_t &lo, int64_t &hi) {
    int a = 0, b = ns;
    while (a < b) {
        const int mid = (a + b) >> 1;
        if (samp[mid] < v) a = mid + 1; else b = mid;
    }
    lo = a == 0 ? ia : ia + (int64_t)(a - 1) * stride + 1;
    hi = min(ia + (int64_t)a * stride, ib);
    if (stride > kPtExact) lo = hi = lower_bound64(Tx, lo, hi, v);
}

// Window edges inside the coarse band: full keys, then the FP64 predicate of
// Algorithm 6 on the caller's own values.  Out of line, so that none of its
// loads are hoisted into the common path.  lo, hi are staged indices.
__device__ __noinline__ int2 pt_band(const int64_t *__restrict__ Tx, const double *__restrict__ tx,
                                     const int64_t *__restrict__ Sy, const double *__restrict__ sy,
                                     const int64_t *__restrict__ dls, const int64_t *__restrict__ dus,
                                     const double *__restrict__ slags, int64_t j, int64_t k, int eps,
                                     double h, int64_t eta, int64_t ia_s, int64_t lim, int lo, int hi,
                                     int fix_lo, int fix_hi) {
    const int64_t Sj = Sy[j];
    const double cj = centre(sy[j], slags[k], eps);
    if (fix_lo) {
        const int64_t Lf = Sj + dls[k];
        const double lb = __dsub_rn(cj, h);
        int64_t p = ia_s + lo;
        while (p < lim && Tx[p] < Lf + eta && (Tx[p] < Lf - eta || tx[p] < lb)) ++p;
        lo = (int)(p - ia_s);
    }
    if (hi < lo) hi = lo;
    if (fix_hi || hi == lo) {
        const int64_t Uf = Sj + dus[k];
        const double ub = __dadd_rn(cj, h);
        int64_t p = ia_s + hi;
        while (p < lim && Tx[p] < Uf + eta && (Tx[p] < Uf - eta || tx[p] <= ub)) ++p;
        hi = (int)(p - ia_s);
    }
    return make_int2(lo, hi);
}

struct PtAcc { long long a00, a01, a02, a10, a11, a12; };

// sum_i a[i] b[i] over the points of a batch as one chain of 32 x 32 -> 64-bit
// multiply-adds (each product below 2^52, the chain below 2^54), then one 64-bit
// add into the accumulator: a chain lets the multiply-adds accumulate in place
// instead of taking a 64-bit add each.
__device__ __forceinline__ long long pt_dot(const int32_t (&a)[kPtBatch], const int32_t (&b)[kPtBatch]) {
    long long t;
    asm("mul.wide.s32 %0, %1, %2;" : "=l"(t) : "r"(a[0]), "r"(b[0]));
#pragma unroll
    for (int i = 1; i < kPtBatch; ++i) asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(t) : "r"(a[i]), "r"(b[i]));
    return t;
}

// The six limb products y_a d_b of a batch's points into the accumulators.
__device__ __forceinline__ void pt_mac_batch(PtAcc &A, const int32_t (&d0)[kPtBatch], const int32_t (&d1)[kPtBatch],
                                             const int32_t (&d2)[kPtBatch], const int32_t (&y0)[kPtM],
                                             const int32_t (&y1)[kPtM], int q0) {
    int32_t ya[kPtBatch], yb[kPtBatch];
#pragma unroll
    for (int i = 0; i < kPtBatch; ++i) {
        ya[i] = y0[q0 + i];
        yb[i] = y1[q0 + i];
    }
    A.a00 += pt_dot(ya, d0);
    A.a01 += pt_dot(ya, d1);
    A.a02 += pt_dot(ya, d2);
    A.a10 += pt_dot(yb, d0);
    A.a11 += pt_dot(yb, d1);
    A.a12 += pt_dot(yb, d2);
}

// a 2^e added to the 128-bit two's-complement value (lo, hi), 0 < e < 64
template <int e>
__device__ __forceinline__ void pt_add_shifted(unsigned long long &lo, unsigned long long &hi, long long a) {
    const unsigned long long l = (unsigned long long)a << e;
    const unsigned long long h = (unsigned long long)(a >> (64 - e));
    asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(lo), "+l"(hi) : "l"(l), "l"(h));
}

__device__ __forceinline__ U128 pt_combine(const PtAcc &A) {
    unsigned long long lo = (unsigned long long)A.a00;
    unsigned long long hi = (unsigned long long)(A.a00 >> 63) + ((unsigned long long)A.a12 << 9);  // a12 2^73
    pt_add_shifted<21>(lo, hi, A.a01);
    pt_add_shifted<31>(lo, hi, A.a10);
    pt_add_shifted<42>(lo, hi, A.a02);
    pt_add_shifted<52>(lo, hi, A.a11);
    return U128{lo, hi};
}

__device__ __forceinline__ void add128x(U128 &a, const U128 &b) {
    asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(a.lo), "+l"(a.hi) : "l"(b.lo), "l"(b.hi));
}
__device__ __forceinline__ U128 shfl_xor128(const U128 &v, int o) {
    return U128{__shfl_xor_sync(0xffffffffu, v.lo, o), __shfl_xor_sync(0xffffffffu, v.hi, o)};
}
__device__ __forceinline__ void warp_sum128(U128 &a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long lo = __shfl_xor_sync(0xffffffffu, a.lo, o);
        const unsigned long long hi = __shfl_xor_sync(0xffffffffu, a.hi, o);
        add128(a, lo, hi);
    }
}

struct PtLagArgs {
    const int64_t *Tx, *Sy, *dls, *dus;
    const double *tx, *sy, *slags;
    int64_t j0, k, ia_s, lim, eta;
    double h;
    int eps, pa, pb;
    uint32_t mult;
};

// One lag over this lane's outer points of the segment [pa, pb) (the whole
// full tile when kFull).  Bit q of m (warp-uniform) is clear when no window of
// slot q's points at this lag can hold a key; a batch whose slots are all clear
// is skipped.  Points are handled kPtBatch at a time: the rank-table
// and entry loads of a batch are issued together; an edge whose bin holds keys
// below its query steps forward in one warp-uniform loop over the batch (about
// 0.25 keys per query on the light-curve batch, but over a warp's 32 lanes the
// loop runs to the largest count), then the rarely entered band test's FP64
// fix-up, then the counts and the numerators.  Edge positions are
// shared-window byte addresses of staged entries (16 bytes each).
template <bool kFull>
__device__ __forceinline__ void pt_lag(uint32_t aE, uint32_t aT, const int32_t (&sc)[kPtM],
                                       const int32_t (&y0)[kPtM], const int32_t (&y1)[kPtM], int pbase,
                                       int32_t sca, int4 L, uint32_t m, const PtLagArgs &g, unsigned &c,
                                       PtAcc &A) {
#pragma unroll
    for (int q0 = 0; q0 < kPtM; q0 += kPtBatch) {
        if (((m >> q0) & ((1u << kPtBatch) - 1u)) == 0u) continue;
        int32_t s[kPtBatch];
        bool ok[kPtBatch];
#pragma unroll
        for (int i = 0; i < kPtBatch; ++i) {
            const int pt = pbase + pt_off(q0 + i);
            ok[i] = kFull || (pt >= g.pa && pt < g.pb);
            s[i] = ok[i] ? sc[q0 + i] : sca;  // a point outside the segment queries in range, counts nothing
        }
        uint32_t ol[kPtBatch], oh[kPtBatch];
        int4 el[kPtBatch], eh[kPtBatch];
#pragma unroll
        for (int i = 0; i < kPtBatch; ++i) {
            ol[i] = lds_u16(pt_bin_addr(aT, s[i] + L.x, g.mult));
            oh[i] = lds_u16(pt_bin_addr(aT, s[i] + L.z, g.mult));
        }
#pragma unroll
        for (int i = 0; i < kPtBatch; ++i) {
            ol[i] = aE + (ol[i] << 4);
            oh[i] = aE + (oh[i] << 4);
            el[i] = lds_v4(ol[i]);
            eh[i] = lds_v4(oh[i]);
        }
        // one warp-uniform walk loop over the batch's slots, two predicated steps
        // per iteration: the slots' loads are in flight together and the loop
        // control (a vote) is shared by all the batch's edges and two steps.  With
        // four-slot batches on the bench batch's rectangle call: 102.7 ms, against
        // 103.9 ms with one step and 103.7 ms with three per iteration, 104.8 ms for
        // a loop per pair of slots, 105.7 ms for a loop per slot; with two-slot
        // batches one step per iteration is 1 % slower than two
        static_assert(kPtBatch == 2 || kPtBatch == 4, "the walk below spells out two or four slots");
        const auto pend = [&](int u) { return (el[u].x < s[u] + L.x) | (eh[u].x < s[u] + L.z); };
        bool step = kPtBatch == 4 ? pend(0) | pend(1) | pend(2) | pend(3) : pend(0) | pend(1);
        while (__any_sync(0xffffffffu, step)) {
#pragma unroll
            for (int r = 0; r < 2; ++r) {
#pragma unroll
                for (int u = 0; u < kPtBatch; ++u) {
                    if (el[u].x < s[u] + L.x) {
                        ol[u] += 16u;
                        el[u] = lds_v4(ol[u]);
                    }
                    if (eh[u].x < s[u] + L.z) {
                        oh[u] += 16u;
                        eh[u] = lds_v4(oh[u]);
                    }
                }
            }
            step = kPtBatch == 4 ? pend(0) | pend(1) | pend(2) | pend(3) : pend(0) | pend(1);
        }
        bool band = false;
#pragma unroll
        for (int i = 0; i < kPtBatch; ++i) band |= ok[i] & ((el[i].x < s[i] + L.y) | (eh[i].x < s[i] + L.w));
        if (__any_sync(0xffffffffu, band)) {
#pragma unroll
            for (int i = 0; i < kPtBatch; ++i) {
                const bool fl = el[i].x < s[i] + L.y, fh = eh[i].x < s[i] + L.w;
                if (ok[i] && (fl || fh)) {
                    const int2 r = pt_band(g.Tx, g.tx, g.Sy, g.sy, g.dls, g.dus, g.slags,
                                           g.j0 + pbase + pt_off(q0 + i), g.k, g.eps, g.h, g.eta, g.ia_s, g.lim,
                                           (int)((ol[i] - aE) >> 4), (int)((oh[i] - aE) >> 4), fl, fh);
                    ol[i] = aE + 16u * (unsigned)r.x;
                    oh[i] = aE + 16u * (unsigned)r.y;
                    el[i] = lds_v4(ol[i]);
                    eh[i] = lds_v4(oh[i]);
                }
            }
        }
        // off the band, oh >= ol: the upper query is not below the lower one
        int32_t d0[kPtBatch], d1[kPtBatch], d2[kPtBatch];
#pragma unroll
        for (int i = 0; i < kPtBatch; ++i) {
            const bool use = kFull || ok[i];
            c += use ? oh[i] - ol[i] : 0u;
            // limbs of prefix sums rebased to the sub-group's first entry: |P| < 2^61,
            // so the top limbs (P >> 42) differ by less than 2^20 and every
            // difference is exact
            d0[i] = use ? eh[i].y - el[i].y : 0;
            d1[i] = use ? eh[i].z - el[i].z : 0;
            d2[i] = use ? eh[i].w - el[i].w : 0;
        }
        pt_mac_batch(A, d0, d1, d2, y0, y1, q0);
    }
}

__global__ void __launch_bounds__(kPtWarps * 32, 2)
rect_scan_pt_kernel(const int64_t *__restrict__ Tx, const int64_t *__restrict__ P,
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
    PtSmem &sm = *reinterpret_cast<PtSmem *>(smem_raw);
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem_raw);
    const uint32_t aE = sbase + kOffE, aT = sbase + kOffT;
    const int64_t tI = blockIdx.x / G;
    const int g = (int)(blockIdx.x - tI * G);
    const ScanTile tile = tiles[tI];
    const RectRange rg = ranges[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tid = threadIdx.x;
    const int64_t xb = offs_x[tile.b + 1];
    const int tn = (int)(tile.j1 - tile.j0);
    const int64_t S0 = Sy[tile.j0], Slast = Sy[tile.j1 - 1];
    const int64_t k0 = (int64_t)g * kLagGroup;
    const int nk = (int)min((int64_t)kLagGroup, K - k0);
    const int64_t ia = rg.ia, ib = min(rg.ib, xb);
    // coarse shift: every coarse value of the CTA below 2^29 (as in the lags-on-lanes scan)
    int sh = 0;
    {
        const int64_t span = (Slast - S0) + (gmax[g] - gmin[g]) + 4 * eta + 16;
        const int bits = 64 - __clzll((unsigned long long)max(span, (int64_t)1));
        sh = max(0, bits - 28);
    }
    // this lane's outer points: coarse offsets and the two limbs of Y
    int32_t sc[kPtM], y0[kPtM], y1[kPtM];
    const int pbase = pt_base(warp, lane);
#pragma unroll
    for (int q = 0; q < kPtM; ++q) {
        const int pt = pbase + pt_off(q);
        const int64_t Y = pt < tn ? Yq[tile.j0 + pt] : 0;
        sc[q] = pt < tn ? (int32_t)((Sy[tile.j0 + pt] - S0) >> sh) : 0;
        y0[q] = (int32_t)(Y & 0x7fffffffll);
        y1[q] = (int32_t)(Y >> 31);
    }
    if (tid == 0) {
        sm.seg[0] = make_int2(0, tn);
        sm.n_seg = 1;
    }
    unsigned int my_c = 0;
    U128 my{0ull, 0ull};
    for (;;) {
        __syncthreads();
        const int n_seg = sm.n_seg;
        if (n_seg == 0) break;
        const int2 seg = sm.seg[n_seg - 1];
        const int pa = seg.x, pb = seg.y;
        __syncthreads();  // every thread has read the segment before warp 0 edits the stack
        // plan the segment: lag sub-groups whose key unions fit the staging area,
        // or a split of the segment when one lag's union does not fit
        const bool whole = pa == 0 && pb == tn && ib - ia + 1 <= kPtCap;
        // planning samples of the group's keys [ia, ib), one round of independent
        // loads by the whole CTA into the (idle) staging area; the searches below
        // run on them in shared memory
        const int64_t *samp = reinterpret_cast<const int64_t *>(sm.sE);
        int64_t stride = 1;
        int ns = 0;
        if (!whole) {
            const int64_t nr = ib - ia;
            stride = max((int64_t)1, (nr + kPtSamples - 1) / kPtSamples);
            ns = (int)((nr + stride - 1) / stride);
            int64_t *w = reinterpret_cast<int64_t *>(sm.sE);
            for (int m = tid; m < ns; m += blockDim.x) w[m] = Tx[ia + (int64_t)m * stride];
            __syncthreads();
        }
        if (warp == 0) {
            if (whole) {
                if (lane == 0) {
                    sm.sub[0] = PtSub{0, nk, 0, 0, ia, ib, gmin[g], gmax[g]};
                    sm.n_sub = 1;
                    sm.n_seg = n_seg - 1;
                }
            } else {
                const int64_t Sa = Sy[tile.j0 + pa], Sb = Sy[tile.j0 + pb - 1];
                int big = 0, wide = 0;
                if (lane < nk) {
                    // bracketed ranks: the lower end of the first query, the upper
                    // end of the last; the staged range may grow by < 2 stride keys
                    const int64_t dl = dls[k0 + lane], du = dus[k0 + lane];
                    int64_t lo, hi, x0, x1;
                    pt_bracket(samp, ns, stride, Tx, ia, ib, Sa + dl - eta, lo, x1);
                    pt_bracket(samp, ns, stride, Tx, ia, ib, Sb + du + eta, x0, hi);
                    hi = max(hi, lo);
                    sm.klo[lane] = lo;
                    sm.khi[lane] = hi;
                    sm.kdl[lane] = dl;
                    sm.kdu[lane] = du;
                    big = hi - lo + 1 > kPtCap;
                    // a single outer point's window already fills half the area:
                    // splitting would not help, the lag runs on the global keys
                    if (big) {
                        pt_bracket(samp, ns, stride, Tx, ia, ib, Sa + du + eta, x0, x1);
                        wide = x1 - lo + 1 > kPtCap / 2;
                    }
                }
                // Split point: at the widest time gap between consecutive outer points
                // when it spans a quarter of the segment or more (a tile across a
                // seasonal gap, whose windows at some lags cover a whole observing
                // season), else in the middle.  Gap splits stop at 8 pending segments
                // and middle splits at 15, so the stack of 16 never overflows.
                const bool need = __any_sync(0xffffffffu, big && !wide);
                int cut = -1;
                if (need && pb - pa > 1 && n_seg < 8) {
                    int64_t best = -1;
                    int at = -1;
                    for (int p = pa + lane; p + 1 < pb; p += 32) {
                        const int64_t gp = Sy[tile.j0 + p + 1] - Sy[tile.j0 + p];
                        if (gp > best) {
                            best = gp;
                            at = p;
                        }
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const int64_t b2 = __shfl_xor_sync(0xffffffffu, best, o);
                        const int a2 = __shfl_xor_sync(0xffffffffu, at, o);
                        if (b2 > best || (b2 == best && a2 >= 0 && (at < 0 || a2 < at))) {
                            best = b2;
                            at = a2;
                        }
                    }
                    if (at >= 0 && 4 * best >= Sb - Sa) cut = at + 1;
                }
                if (cut < 0 && need && pb - pa > 32 && n_seg < 15) cut = pa + ((((pb - pa) >> 1) + 31) & ~31);
                const bool split = cut > pa && cut < pb;
                __syncwarp();
                if (lane == 0) {
                    if (split) {
                        sm.seg[n_seg - 1] = make_int2(cut, pb);
                        sm.seg[n_seg] = make_int2(pa, cut);
                        sm.n_seg = n_seg + 1;
                        sm.n_sub = 0;
                    } else {
                        int n = 0, a = 0;
                        while (a < nk) {
                            int64_t lo = sm.klo[a], hi = sm.khi[a];
                            int64_t dmn = sm.kdl[a], dmx = sm.kdu[a];
                            int b = a + 1;
                            const int gl = (hi - lo + 1 > kPtCap) ? 1 : 0;
                            while (!gl && b < nk) {
                                const int64_t nlo = min(lo, sm.klo[b]), nhi = max(hi, sm.khi[b]);
                                if (nhi - nlo + 1 > kPtCap) break;
                                lo = nlo;
                                hi = nhi;
                                dmn = min(dmn, sm.kdl[b]);
                                dmx = max(dmx, sm.kdu[b]);
                                ++b;
                            }
                            sm.sub[n++] = PtSub{a, b, gl, 0, lo, hi, dmn, dmx};
                            a = b;
                        }
                        sm.n_sub = n;
                        sm.n_seg = n_seg - 1;
                    }
                }
            }
        }
        __syncthreads();
        const int n_sub = sm.n_sub;
        const bool full = pa == 0 && pb == kRectTile;
        // coarse offsets of the segment's first and last outer points
        const int32_t sca = (int32_t)((Sy[tile.j0 + pa] - S0) >> sh);
        const int32_t scb = (int32_t)((Sy[tile.j0 + pb - 1] - S0) >> sh);
        for (int s = 0; s < n_sub; ++s) {
            const PtSub sb = sm.sub[s];
            const int64_t lim = min(sb.ib + 1, xb);
            if (!sb.global) {
                const int64_t base = S0 + sb.dmin - eta;
                const int64_t t_last = min(sb.ib, xb - 1);
                const int nK = (int)(t_last - sb.ia + 1);
                // queries of the segment lie in [vmin, vmax]; keys and lag offsets
                // are stored relative to vmin, the bins cover [0, vmax - vmin]
                const int32_t vmin = sca + (int32_t)((S0 + sb.dmin - eta - base) >> sh);
                const int32_t vmax = scb + (int32_t)((S0 + sb.dmax + eta - base) >> sh) + 2;
                const uint32_t mult = pt_bin_mult(max(vmax - vmin, 1));
                // entries 0 .. nK: keys (nK: the sentinel) and the limbs of P[ia + i].
                // Tx and P of entry i are copied asynchronously into its own 16-byte
                // slot (all copies in flight at once), then each thread rewrites its
                // own slots in place as {key, p0, p1, p2}.
                for (int i = tid; i <= max(nK, 0); i += blockDim.x) {
                    const unsigned slot = (unsigned)__cvta_generic_to_shared(&sm.sE[i]);
                    if (i < nK)
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(slot), "l"(Tx + sb.ia + i)
                                     : "memory");
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(slot + 8u), "l"(P + sb.ia + i)
                                 : "memory");
                }
                // the rank table is built as a histogram of the keys' bins (two 16-bit
                // counters per word) and then scanned: cleared while the copies fly
                uint32_t *const T32 = reinterpret_cast<uint32_t *>(sm.sT);
                for (int i = tid; i < kPtBins / 8; i += blockDim.x)
                    reinterpret_cast<uint4 *>(T32)[i] = make_uint4(0u, 0u, 0u, 0u);
                asm volatile("cp.async.wait_all;" ::: "memory");
                __syncthreads();
                // prefix sums rebased to the first entry's: |P[ia + i] - P[ia]| is a sum
                // of |X| within one series, below n 2^p + n/2 < 2^61 (sum |x_std| <= n for
                // ddof 0 and p <= 61 - 1.5 log2 n), so the three limbs never wrap
                const int64_t P0 = P[sb.ia];
                for (int i = tid; i <= max(nK, 0); i += blockDim.x) {
                    const longlong2 raw = *reinterpret_cast<const longlong2 *>(&sm.sE[i]);
                    int32_t key = kSentinel;
                    if (i < nK) {
                        const int64_t v = ((raw.x - base) >> sh) - vmin;
                        key = (int32_t)max(min(v, (int64_t)(1 << 30)), (int64_t)-1);
                        const uint32_t bk = pt_bin(key, mult);
                        if (bk < (uint32_t)kPtBins) atomicAdd(T32 + (bk >> 1), (bk & 1u) ? 0x10000u : 1u);
                    }
                    const int64_t pv = (int64_t)((unsigned long long)raw.y - (unsigned long long)P0);
                    sm.sE[i] = make_int4(key, (int32_t)(pv & 0x1fffff), (int32_t)((pv >> 21) & 0x1fffff),
                                         (int32_t)(pv >> 42));
                }
                if (tid < sb.kb - sb.ka) {
                    const int k = (int)k0 + sb.ka + tid;
                    const int64_t dl = dls[k], du = dus[k];
                    sm.lc[sb.ka + tid] = make_int4((int32_t)((S0 + dl - eta - base) >> sh) - vmin,
                                                   (int32_t)((S0 + dl + eta - base) >> sh) + 2 - vmin,
                                                   (int32_t)((S0 + du - eta - base) >> sh) - vmin,
                                                   (int32_t)((S0 + du + eta - base) >> sh) + 2 - vmin);
                }
                __syncthreads();
                // rank table: sT[b] = the first index whose key's bin is >= b, which for
                // sorted keys (bins non-decreasing) is the number of keys in bins below b:
                // the exclusive prefix sum of the histogram.  Entry nK, the sentinel, is
                // after every bin.  Each thread scans 2 kPtWords consecutive bins, the
                // warps' totals are combined through shared memory (the per-warp sums
                // of the lag loop's results are written only at the end of the CTA).
                {
                    uint32_t w[kPtWords];
                    const uint4 *src = reinterpret_cast<const uint4 *>(T32 + tid * kPtWords);
#pragma unroll
                    for (int q = 0; q < kPtWords / 4; ++q) {
                        const uint4 u = src[q];
                        w[4 * q] = u.x;
                        w[4 * q + 1] = u.y;
                        w[4 * q + 2] = u.z;
                        w[4 * q + 3] = u.w;
                    }
                    uint32_t run = 0;  // below 2^16: at most kPtCap keys
#pragma unroll
                    for (int q = 0; q < kPtWords; ++q) {
                        const uint32_t lo = w[q] & 0xffffu, hi = w[q] >> 16;
                        w[q] = run | ((run + lo) << 16);
                        run += lo + hi;
                    }
                    uint32_t inc = run;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                        if (lane >= o) inc += y;
                    }
                    if (lane == 31) sm.pc[0][warp] = inc;
                    __syncthreads();
                    uint32_t off = inc - run;
                    for (int v = 0; v < warp; ++v) off += sm.pc[0][v];
                    off *= 0x10001u;
                    uint4 *dst = reinterpret_cast<uint4 *>(T32 + tid * kPtWords);
#pragma unroll
                    for (int q = 0; q < kPtWords / 4; ++q)
                        dst[q] = make_uint4(w[4 * q] + off, w[4 * q + 1] + off, w[4 * q + 2] + off, w[4 * q + 3] + off);
                }
                __syncthreads();
                // Slots whose windows are empty at a lag.  Slot q of this warp holds 32
                // consecutive outer points with query offsets in [lo_q, hi_q] (points
                // of the segment only).  At lag kl, keys below lo_q + L.x are certainly
                // below every lower bound of the slot (the walk's test) and keys at or
                // above hi_q + L.w certainly above every upper bound (the band test's),
                // so when the first key at or above lo_q + L.x is at or above
                // hi_q + L.w, every window of the slot is empty: count 0, window sum 0.
                // Lane kl - ka keeps lag kl's mask of the other slots.  Windows that
                // fall in a seasonal gap or on nights without data are skipped.
                uint32_t act = 0;
                {
                    const int4 Lm = sm.lc[sb.ka + min(lane, sb.kb - sb.ka - 1)];
#pragma unroll
                    for (int q = 0; q < kPtM; ++q) {
                        const int pt = pbase + pt_off(q);
                        const bool in = full || (pt >= pa && pt < pb);
                        const int32_t lo_q = __reduce_min_sync(0xffffffffu, in ? sc[q] : INT_MAX);
                        const int32_t hi_q = __reduce_max_sync(0xffffffffu, in ? sc[q] : INT_MIN);
                        if (lo_q <= hi_q) {
                            const int32_t v = lo_q + Lm.x;
                            uint32_t a = aE + (lds_u16(pt_bin_addr(aT, v, mult)) << 4);
                            int32_t key = lds_s32(a);
                            while (key < v) {
                                a += 16u;
                                key = lds_s32(a);
                            }
                            act |= (key < hi_q + Lm.w ? 1u : 0u) << q;
                        }
                    }
                }
                PtLagArgs ga{Tx, Sy, dls, dus, tx, sy, slags, tile.j0, 0, sb.ia, lim, eta, h, eps, pa, pb, mult};
                for (int kl = sb.ka; kl < sb.kb; ++kl) {
                    const uint32_t m = __shfl_sync(0xffffffffu, act, kl - sb.ka);
                    if (m == 0u) continue;  // every window of the warp's points is empty
                    const int4 L = sm.lc[kl];
                    ga.k = k0 + kl;
                    unsigned int c = 0;
                    PtAcc A{0, 0, 0, 0, 0, 0};
                    if (full)
                        pt_lag<true>(aE, aT, sc, y0, y1, pbase, sca, L, m, ga, c, A);
                    else
                        pt_lag<false>(aE, aT, sc, y0, y1, pbase, sca, L, m, ga, c, A);
                    c = __reduce_add_sync(0xffffffffu, c >> 4);
                    U128 acc = pt_combine(A);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) add128x(acc, shfl_xor128(acc, o));
                    if (lane == kl) {
                        my_c += c;
                        add128x(my, acc);
                    }
                }
                __syncthreads();  // the staging area is rewritten next
            } else {
                // one lag whose union does not fit: binary searches on the global keys
                for (int kl = sb.ka; kl < sb.kb; ++kl) {
                    const int64_t dl = dls[k0 + kl], du = dus[k0 + kl];
                    const double tau = slags[k0 + kl];
                    unsigned int c = 0;
                    U128 acc{0ull, 0ull};
                    for (int q = 0; q < kPtM; ++q) {
                        const int pt = pbase + pt_off(q);
                        if (pt < pa || pt >= pb) continue;
                        const int64_t j = tile.j0 + pt;
                        const int64_t Lf = Sy[j] + dl, Uf = Sy[j] + du;
                        int64_t lo = lower_bound64(Tx, sb.ia, sb.ib, Lf - eta);
                        if (lo < lim && Tx[lo] < Lf + eta) {
                            const double lb = __dsub_rn(centre(sy[j], tau, eps), h);
                            while (lo < lim && Tx[lo] < Lf + eta && tx[lo] < lb) ++lo;
                        }
                        int64_t hi = max(lo, lower_bound64(Tx, lo, sb.ib, Uf - eta));
                        if (hi < lim && Tx[hi] < Uf + eta) {
                            const double ub = __dadd_rn(centre(sy[j], tau, eps), h);
                            while (hi < lim && Tx[hi] < Uf + eta && tx[hi] <= ub) ++hi;
                        }
                        c += (unsigned int)(hi - lo);
                        const long long w = (long long)((unsigned long long)P[hi] - (unsigned long long)P[lo]);
                        mac128(acc, w, Yq[j]);
                    }
                    c = __reduce_add_sync(0xffffffffu, c);
                    warp_sum128(acc);
                    if (lane == kl) {
                        my_c += c;
                        add128(my, acc.lo, acc.hi);
                    }
                }
            }
        }
    }
    sm.pc[warp][lane] = my_c;
    sm.pl[warp][lane] = my.lo;
    sm.ph[warp][lane] = my.hi;
    __syncthreads();
    if (warp == 0 && lane < nk) {
        unsigned long long cs = 0;
        U128 a{0ull, 0ull};
        for (int w = 0; w < kPtWarps; ++w) {
            cs += sm.pc[w][lane];
            add128(a, sm.pl[w][lane], sm.ph[w][lane]);
        }
        const int64_t k = k0 + lane;
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
        copy_pinned(dst, pinned + off, bytes, st);
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
    static std::atomic<unsigned long long> attr_done{0};
    const size_t smem = sizeof(RectSmem);
    once_per_device(attr_done, [&] {
        return set_smem_limit(rect_scan_kernel<16>, smem) & set_smem_limit(rect_scan_kernel<32>, smem) &
               set_smem_limit(rect_scan_kernel<64>, smem) & set_smem_limit(rect_scan_pt_kernel, sizeof(PtSmem));
    });
#define NCF_RECT_SCAN(RUN)                                                                              \
    NCF_LAUNCH("rect_scan_kernel", st,                                                                 \
               rect_scan_kernel<RUN><<<(unsigned)nr, kRectWarps * 32, smem, st>>>(                     \
                   a.Tx, a.P, a.tx, a.offs_x, a.Sy, a.Yq, a.sy, tiles, (int)r.G, ranges, r.slags, r.perm, \
                   r.dls, r.dus, r.gmin, r.gmax, a.K, a.eps, a.h, a.fs.eta, a.cnt, a.num128))
    switch (r.variant) {
        case 0: NCF_RECT_SCAN(16); break;
        case 2: NCF_RECT_SCAN(64); break;
        case 3:
            NCF_LAUNCH("rect_scan_pt_kernel", st,
                       rect_scan_pt_kernel<<<(unsigned)nr, kPtWarps * 32, sizeof(PtSmem), st>>>(
                           a.Tx, a.P, a.tx, a.offs_x, a.Sy, a.Yq, a.sy, tiles, (int)r.G, ranges, r.slags,
                           r.perm, r.dls, r.dus, r.gmin, r.gmax, a.K, a.eps, a.h, a.fs.eta, a.cnt, a.num128));
            break;
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
