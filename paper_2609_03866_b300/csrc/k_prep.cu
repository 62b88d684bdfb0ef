// k_prep.cu -- per-series statistics, validation flags, fixed-point keys and
// exact integer prefix sums.
//
// Standardisation (Appendix, "Prior standardization"; step 1 of Algorithms
// 2, 4, 9, 10): mean and population variance (ddof 0).  The pass is chunked --
// one CTA per `chunk` points of one series -- so a single series of 1e7 points
// spreads over the whole GPU; sums are shifted by the series' first value
// (d = x - x_ref, one FP64 subtraction) so that the one-pass variance
// S2/n - (S1/n)^2 does not cancel.  Each thread sums its 16 points' d and d^2
// in double-float (about 47 bits; the FP64 pipe would bound the pass), the
// partials are combined in FP64 in a fixed order (deterministic).
//
// The exact rectangle scan works on fixed-point images of the inputs:
//   T_i = floor(t_i * 2^q)  -- monotone, so comparisons against window bounds
//                              are decided in integer arithmetic except inside
//                              a narrow ambiguity band that falls back to FP64;
//   X_i = round(x_std,i * 2^p) and P = exclusive prefix sums of X in int64
//   with wrap-around: a window sum P[hi] - P[lo] is exact whenever its true
//   value fits in 63 bits, whatever the prefix values themselves do.
#include <algorithm>

#include "common.cuh"

namespace ncf {

namespace {

constexpr int kThreads = 256;

// cs[g] = series of chunk g (one thread per series writes its chunk range)
__global__ void chunk_series_kernel(const int64_t *__restrict__ chunk_base, int64_t B,
                                    int32_t *__restrict__ cs) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    for (int64_t g = chunk_base[b]; g < chunk_base[b + 1]; ++g) cs[g] = (int32_t)b;
}

// floor(v * 2^q) as int64 from the bit pattern of v (exact: the product is a
// power-of-two scaling).  Requires |v| 2^q < 2^62.  Integer operations only:
// FP64 conversion instructions are slow on this GPU.
__device__ __forceinline__ long long fixed_floor(double v, int q) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const bool neg = (u >> 63) != 0;
    const int e = (int)((u >> 52) & 0x7FF);
    if (e == 0) return (neg && (u << 1) != 0) ? -1 : 0;  // zero or subnormal
    const unsigned long long m = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = e - 1075 + q;
    unsigned long long mag;
    bool rem;
    if (sh >= 0) {
        mag = m << sh;
        rem = false;
    } else if (sh > -64) {
        mag = m >> -sh;
        rem = (m << (64 + sh)) != 0;
    } else {
        mag = 0;
        rem = true;
    }
    return neg ? -(long long)(mag + (rem ? 1 : 0)) : (long long)mag;
}

// Double-float arithmetic (an unevaluated sum h + l of two floats, about 47
// significant bits): the statistics pass accumulates each thread's points this
// way on the FP32 pipe, which runs many times the FP64 rate here.
struct DF {
    float h, l;
};
// sum of two double-float values (two-sum of the high parts, low parts added)
__device__ __forceinline__ DF df_add(DF a, DF b) {
    const float s = a.h + b.h;
    const float v = s - a.h;
    float e = (a.h - (s - v)) + (b.h - v);
    e += a.l + b.l;
    const float h = s + e;
    return DF{h, e - (h - s)};
}
// square of a double-float value (exact product of the high parts by FMA)
__device__ __forceinline__ DF df_sqr(DF a) {
    const float p = a.h * a.h;
    float e = fmaf(a.h, a.h, -p);
    e = fmaf(2.0f * a.h, a.l, e);
    const float h = p + e;
    return DF{h, e - (h - p)};
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kThreads)
stats_chunks_kernel(const double *__restrict__ t, const double *__restrict__ x,
                    const int64_t *__restrict__ offs, const int64_t *__restrict__ chunk_base,
                    const int32_t *__restrict__ cs, int chunk, ChunkPartial *__restrict__ part) {
    const int64_t g = blockIdx.x;
    const int64_t b = cs[g];
    const int64_t a0 = offs[b], a1 = offs[b + 1];
    const int64_t start = a0 + (g - chunk_base[b]) * (int64_t)chunk;
    const int64_t end = min(start + (int64_t)chunk, a1);
    const double xref = x[a0];
    DF f1{0.0f, 0.0f}, f2{0.0f, 0.0f};  // this thread's sums of d and d^2
    int flags = 0;
    // largest exponent field of the thread's values (bits 20..30 of the high
    // words), tested for 0x7FF once at the end: written as a per-value test of
    // the exponent, the compiler turned it into two FP64 compares per point, on
    // this GPU's slow FP64 pipe
    unsigned emax = 0u;
    constexpr int kPer = kPrepChunk / kThreads;
    const int lane = threadIdx.x & 31;
    // order-preserving integer image of a time
    auto okey = [](double v) {
        const unsigned long long u = (unsigned long long)__double_as_longlong(v);
        return (long long)(u ^ ((u >> 63) ? 0x7FFFFFFFFFFFFFFFull : 0ull));
    };
#pragma unroll 4
    for (int r = 0; r < kPer; ++r) {
        const int64_t i = start + threadIdx.x + (int64_t)r * kThreads;
        const bool in = i < end;
        const double xi = in ? x[i] : xref, ti = in ? t[i] : 0.0;
        // the point before i is lane - 1's point of the same round (lane 0: a load)
        const double tprev_l = __shfl_up_sync(0xffffffffu, ti, 1);
        if (in) {
            emax = max(emax, max((unsigned)__double2hiint(xi) & 0x7FF00000u,
                                 (unsigned)__double2hiint(ti) & 0x7FF00000u));
            if (i > a0) {
                const double tprev = lane ? tprev_l : t[i - 1];
                if (okey(tprev) > okey(ti)) flags |= STAT_UNSORTED;
            }
            // one FP64 subtraction (as rounded as before), then double-float sums
            float dh, dl;
            split_df(xi - xref, dh, dl);
            const DF d{dh, dl};
            f1 = df_add(f1, d);
            f2 = df_add(f2, df_sqr(d));
        }
    }
    if (emax == 0x7FF00000u) flags |= STAT_NONFINITE;
    double s1 = (double)f1.h + (double)f1.l, s2 = (double)f2.h + (double)f2.l;
    __shared__ double sh1[kThreads / 32], sh2[kThreads / 32];
    __shared__ int shf[kThreads / 32];
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    flags = __reduce_or_sync(0xffffffffu, flags);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sh1[w] = s1; sh2[w] = s2; shf[w] = flags; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0;
        int f = 0;
        for (int q = 0; q < kThreads / 32; ++q) { a += sh1[q]; c += sh2[q]; f |= shf[q]; }
        part[g] = ChunkPartial{a, c, f, 0};
    }
}

__global__ void stats_finish_kernel(const double *__restrict__ t, const double *__restrict__ x,
                                    const int64_t *__restrict__ offs,
                                    const int64_t *__restrict__ chunk_base, int64_t B,
                                    const ChunkPartial *__restrict__ part,
                                    SeriesStats *__restrict__ stats) {
    // one warp per series: lane l sums chunks l, l + 32, ..., then a butterfly over
    // the lanes (a fixed order: the same sums on every run)
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= B) return;
    double s1 = 0.0, s2 = 0.0;
    int flags = 0;
    for (int64_t g = chunk_base[b] + lane; g < chunk_base[b + 1]; g += 32) {
        s1 += part[g].s1;
        s2 += part[g].s2;
        flags |= part[g].flags;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        flags |= __shfl_xor_sync(0xffffffffu, flags, o);
    }
    if (lane != 0) return;
    const int64_t a0 = offs[b], a1 = offs[b + 1];
    const double n = (double)(a1 - a0);
    const double m1 = s1 / n;
    const double var = s2 / n - m1 * m1;
    SeriesStats st;
    st.mean = x[a0] + m1;
    st.n = a1 - a0;
    if (var > 0.0 && isfinite(var)) {
        st.inv_std = 1.0 / sqrt(var);
    } else {
        st.inv_std = 0.0;
        flags |= STAT_DEGENERATE;
    }
    st.t_first = t[a0];
    st.t_last = t[a1 - 1];
    st.flags = flags;
    st.pad = 0;
    stats[b] = st;
}

constexpr int kItems = 16;  // elements per thread in the keys/prefix kernels
static_assert(kThreads * kItems == kPrepChunk, "one chunk per CTA of the prefix pass");

__global__ void __launch_bounds__(kThreads)
keys_chunks_kernel(const double *__restrict__ t, const double *__restrict__ x,
                   const int64_t *__restrict__ offs, const int64_t *__restrict__ chunk_base,
                   const int32_t *__restrict__ cs, int chunk, const SeriesStats *__restrict__ stats,
                   FixedScales fs, int64_t n_force, int64_t *__restrict__ Tk, int64_t *__restrict__ Xq,
                   unsigned long long *__restrict__ chunk_sums) {
    const int64_t g = blockIdx.x;
    const int64_t b = cs[g];
    const int64_t a0 = offs[b], a1 = offs[b + 1];
    const int64_t start = a0 + (g - chunk_base[b]) * (int64_t)chunk;
    const int64_t end = min(start + (int64_t)chunk, a1);
    const double mean = stats[b].mean, inv = stats[b].inv_std;
    const int p = value_bits(n_force > 0 ? n_force : a1 - a0);
    unsigned long long acc = 0;
#pragma unroll 4
    for (int r = 0; r < kPrepChunk / kThreads; ++r) {
        const int64_t i = start + threadIdx.x + (int64_t)r * kThreads;
        if (i < end) {
            Tk[i] = fixed_floor(t[i], fs.q);
            // round(x_std 2^p) = floor(x_std 2^(p+1) + 1) >> 1, half up
            const long long q2 = fixed_floor((x[i] - mean) * inv, p + 1);
            const long long q = (q2 + 1) >> 1;
            Xq[i] = q;
            acc += (unsigned long long)q;
        }
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ unsigned long long sh[kThreads / 32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int q = 0; q < kThreads / 32; ++q) s += sh[q];
        chunk_sums[g] = s;
    }
}

// Exclusive scan of the chunk sums in place (single CTA, wrap-around int64).
__global__ void __launch_bounds__(1024)
scan_chunk_sums_kernel(unsigned long long *__restrict__ v, int64_t n,
                       unsigned long long *__restrict__ total) {
    const int tid = threadIdx.x;
    const int64_t per = (n + blockDim.x - 1) / blockDim.x;
    const int64_t a = min((int64_t)tid * per, n), e = min(a + per, n);
    unsigned long long s = 0;
    for (int64_t i = a; i < e; ++i) s += v[i];
    __shared__ unsigned long long sh[1024];
    sh[tid] = s;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        unsigned long long add = tid >= o ? sh[tid - o] : 0ull;
        __syncthreads();
        sh[tid] += add;
        __syncthreads();
    }
    unsigned long long run = sh[tid] - s;  // exclusive prefix of this thread's segment
    for (int64_t i = a; i < e; ++i) {
        unsigned long long c = v[i];
        v[i] = run;
        run += c;
    }
    if (tid == (int)blockDim.x - 1) *total = sh[tid];
}

// Per chunk: P[i] = chunk prefix + exclusive scan of Xq inside the chunk.
__global__ void __launch_bounds__(kThreads)
prefix_apply_kernel(const int64_t *__restrict__ offs, const int64_t *__restrict__ chunk_base,
                    const int32_t *__restrict__ cs, int chunk, const int64_t *__restrict__ Xq,
                    const unsigned long long *__restrict__ chunk_pref,
                    const unsigned long long *__restrict__ total, int64_t n_total,
                    int64_t *__restrict__ P) {
    const int64_t g = blockIdx.x;
    const int64_t b = cs[g];
    const int64_t a0 = offs[b], a1 = offs[b + 1];
    const int64_t start = a0 + (g - chunk_base[b]) * (int64_t)chunk;
    const int64_t end = min(start + (int64_t)chunk, a1);
    // the chunk goes through shared memory so that global loads and stores are
    // coalesced (lane-consecutive) while each thread scans 16 consecutive values;
    // one pad slot per 16 keeps the per-thread reads free of bank conflicts
    __shared__ unsigned long long sx[kPrepChunk + kPrepChunk / kItems];
    auto pad = [](int i) { return i + i / kItems; };
    const int n = (int)(end - start);
#pragma unroll
    for (int i = threadIdx.x; i < kPrepChunk; i += kThreads)  // all 16 loads in flight
        sx[pad(i)] = i < n ? (unsigned long long)Xq[start + i] : 0ull;
    __syncthreads();
    const int my0 = threadIdx.x * kItems;
    unsigned long long loc[kItems];
    unsigned long long s = 0;
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
        loc[q] = sx[pad(my0 + q)];
        s += loc[q];
    }
    // block exclusive scan of the per-thread sums
    const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long inc = s;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long u = __shfl_up_sync(0xffffffffu, inc, o);
        if (l >= o) inc += u;
    }
    __shared__ unsigned long long wsum[kThreads / 32];
    if (l == 31) wsum[w] = inc;
    __syncthreads();
    unsigned long long wpre = 0;
    for (int q = 0; q < w; ++q) wpre += wsum[q];
    unsigned long long run = chunk_pref[g] + wpre + inc - s;
#pragma unroll
    for (int q = 0; q < kItems; ++q) {  // each thread rewrites the slots it alone read
        sx[pad(my0 + q)] = run;
        run += loc[q];
    }
    __syncthreads();
#pragma unroll 4
    for (int i = threadIdx.x; i < n; i += kThreads) P[start + i] = (int64_t)sx[pad(i)];
    if (g == (int64_t)gridDim.x - 1 && threadIdx.x == 0) P[n_total] = (int64_t)*total;
}

__global__ void stats_guard_kernel(const SeriesStats *__restrict__ sx, const SeriesStats *__restrict__ sy,
                                   int64_t B, int *__restrict__ status) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    if (sx[b].flags != 0 || (sy && sy[b].flags != 0)) atomicOr(status, STATUS_INPUT);
}

__global__ void keys_guard_kernel(const SeriesStats *__restrict__ sx, const SeriesStats *__restrict__ sy,
                                  int64_t B, double t_abs, int *__restrict__ status) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    double m = fmax(fabs(sx[b].t_first), fabs(sx[b].t_last));
    if (sy) m = fmax(m, fmax(fabs(sy[b].t_first), fabs(sy[b].t_last)));
    if (!(m <= t_abs)) atomicOr(status, STATUS_RANGE);
}

// dst[0 .. bytes) = src[0 .. bytes) in 8-byte words, then the tail bytes
__global__ void copy_pinned_kernel(unsigned char *__restrict__ dst, const unsigned char *__restrict__ src,
                                   size_t bytes) {
    const size_t nw = bytes / 8;
    const size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = i0; i < nw; i += stride)
        reinterpret_cast<unsigned long long *>(dst)[i] = reinterpret_cast<const unsigned long long *>(src)[i];
    for (size_t i = nw * 8 + i0; i < bytes; i += stride) dst[i] = src[i];
}

}  // namespace

void copy_pinned(void *dst, const void *src, size_t bytes, cudaStream_t st) {
    if (bytes == 0) return;
    const size_t words = (bytes + 7) / 8;
    const unsigned blocks = (unsigned)std::min<size_t>((words + 255) / 256, 592);
    NCF_LAUNCH("copy_pinned_kernel", st,
               copy_pinned_kernel<<<blocks, 256, 0, st>>>(static_cast<unsigned char *>(dst),
                                                          static_cast<const unsigned char *>(src), bytes));
}

void launch_stats_guard(const SeriesStats *sx, const SeriesStats *sy, int64_t B, int *status,
                        cudaStream_t st) {
    NCF_LAUNCH("stats_guard_kernel", st,
               stats_guard_kernel<<<(unsigned)((B + 127) / 128), 128, 0, st>>>(sx, sy, B, status));
}

void launch_keys_guard(const SeriesStats *sx, const SeriesStats *sy, int64_t B, double t_abs, int *status,
                       cudaStream_t st) {
    NCF_LAUNCH("keys_guard_kernel", st,
               keys_guard_kernel<<<(unsigned)((B + 127) / 128), 128, 0, st>>>(sx, sy, B, t_abs, status));
}

void launch_chunk_series(const int64_t *chunk_base, int64_t B, int32_t *cs, cudaStream_t st) {
    NCF_LAUNCH("chunk_series_kernel", st,
               chunk_series_kernel<<<(unsigned)((B + 255) / 256), 256, 0, st>>>(chunk_base, B, cs));
}

void launch_stats_chunks(const double *t, const double *x, const int64_t *offs,
                         const int64_t *chunk_base, const int32_t *cs, int64_t n_chunks, int chunk,
                         ChunkPartial *part, cudaStream_t st) {
    NCF_LAUNCH("stats_chunks_kernel", st,
    stats_chunks_kernel<<<(unsigned)n_chunks, kThreads, 0, st>>>(t, x, offs, chunk_base, cs, chunk, part));
}

void launch_stats_finish(const double *t, const double *x, const int64_t *offs,
                         const int64_t *chunk_base, int64_t B, const ChunkPartial *part,
                         SeriesStats *stats, cudaStream_t st) {
    NCF_LAUNCH("stats_finish_kernel", st,
    stats_finish_kernel<<<(unsigned)((B * 32 + 127) / 128), 128, 0, st>>>(t, x, offs, chunk_base, B, part, stats));
}

void launch_keys_prefix(const double *t, const double *x, const int64_t *offs,
                        const int64_t *chunk_base, const int32_t *cs, int64_t n_chunks, int chunk,
                        const SeriesStats *stats, FixedScales fs, int64_t n_force, int64_t *Tk, int64_t *Xq,
                        int64_t *P, int64_t *chunk_sums, int64_t n_total, cudaStream_t st) {
    // chunk must equal kThreads * kItems (= kPrepChunk) for prefix_apply_kernel
    auto *csum = reinterpret_cast<unsigned long long *>(chunk_sums);
    NCF_LAUNCH("keys_chunks_kernel", st,
               keys_chunks_kernel<<<(unsigned)n_chunks, kThreads, 0, st>>>(t, x, offs, chunk_base, cs, chunk,
                                                                            stats, fs, n_force, Tk, Xq, csum));
    NCF_LAUNCH("scan_chunk_sums_kernel", st,
               scan_chunk_sums_kernel<<<1, 1024, 0, st>>>(csum, n_chunks, csum + n_chunks));
    NCF_LAUNCH("prefix_apply_kernel", st,
               prefix_apply_kernel<<<(unsigned)n_chunks, kThreads, 0, st>>>(offs, chunk_base, cs, chunk, Xq,
                                                                             csum, csum + n_chunks, n_total, P));
}

}  // namespace ncf
