// k_boot.cu -- bootstrap replicates of a series, drawn on the device.
//
// The paper recommends resampling (bootstrap or Monte-Carlo over realisations)
// to weigh an estimate against its sampling variance (Sec. 4, "Monte-Carlo over
// independent realizations", and the discussion of Sec. 6), without providing
// it.  Replicate r of a series of n points draws n indices with replacement,
//     i_j = floor(n u_j / 2^64),  u_j = SplitMix64 output number c = 2^32 r + j
// of the stream started at `seed` (output c is mix(seed + (c + 1) gamma), the
// generator of Steele, Lea and Flood with Vigna's constants; the range
// reduction is Lemire's multiply-high), and keeps the drawn points in time
// order.  Drawing is done by counting: one atomic increment per draw on the
// replicate's multiplicity array, then one CTA per replicate scans the
// multiplicities and writes every point as many times as it was drawn, so the
// replicate comes out sorted without a sort.
#include <algorithm>

#include "common.cuh"

namespace ncf {
namespace {

constexpr int kBootThreads = 256;
constexpr int kBootItems = 8;

__device__ __forceinline__ uint64_t splitmix64_out(uint64_t seed, uint64_t c) {
    uint64_t z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void boot_count_kernel(uint64_t seed, int64_t n, int64_t n_boot, int32_t *__restrict__ cnt) {
    const int64_t total = n * n_boot;
    for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < total;
         id += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = id / n, j = id - r * n;
        const uint64_t u = splitmix64_out(seed, ((uint64_t)r << 32) | (uint64_t)j);
        const int64_t i = (int64_t)__umul64hi(u, (uint64_t)n);
        atomicAdd(cnt + r * n + i, 1);
    }
}

// One CTA per replicate: exclusive scan of the multiplicities, chunk by chunk,
// and the expansion of every point into its drawn copies.
__global__ void __launch_bounds__(kBootThreads)
boot_expand_kernel(const double *__restrict__ t, const double *__restrict__ x, int64_t n,
                   const int32_t *__restrict__ cnt, double *__restrict__ bt, double *__restrict__ bx) {
    __shared__ int64_t wsum[kBootThreads / 32];
    const int64_t r = blockIdx.x;
    const int32_t *c = cnt + r * n;
    double *ot = bt + r * n, *ox = bx + r * n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t carry = 0;
    for (int64_t c0 = 0; c0 < n; c0 += (int64_t)kBootThreads * kBootItems) {
        const int64_t my0 = c0 + (int64_t)threadIdx.x * kBootItems;
        int32_t v[kBootItems];
        int64_t s = 0;
#pragma unroll
        for (int q = 0; q < kBootItems; ++q) {
            v[q] = my0 + q < n ? c[my0 + q] : 0;
            s += v[q];
        }
        int64_t inc = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += u;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        int64_t wpre = 0, total = 0;
        for (int w = 0; w < kBootThreads / 32; ++w) {
            if (w < warp) wpre += wsum[w];
            total += wsum[w];
        }
        int64_t pos = carry + wpre + inc - s;
#pragma unroll
        for (int q = 0; q < kBootItems; ++q) {
            const int64_t i = my0 + q;
            if (v[q] > 0) {
                const double ti = t[i], xi = x[i];
                for (int k = 0; k < v[q]; ++k) {
                    ot[pos + k] = ti;
                    ox[pos + k] = xi;
                }
            }
            pos += v[q];
        }
        carry += total;
        __syncthreads();  // wsum is rewritten by the next chunk
    }
}

}  // namespace

void launch_bootstrap(const double *t, const double *x, int64_t n, int64_t n_boot, uint64_t seed, int32_t *cnt,
                      double *bt, double *bx, int sm_count, cudaStream_t st) {
    cudaMemsetAsync(cnt, 0, (size_t)(n * n_boot) * sizeof(int32_t), st);
    const int64_t total = n * n_boot;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, (int64_t)std::max(sm_count, 1) * 16);
    NCF_LAUNCH("boot_count_kernel", st,
               boot_count_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(seed, n, n_boot, cnt));
    NCF_LAUNCH("boot_expand_kernel", st,
               boot_expand_kernel<<<(unsigned)n_boot, kBootThreads, 0, st>>>(t, x, n, cnt, bt, bx));
}

}  // namespace ncf
