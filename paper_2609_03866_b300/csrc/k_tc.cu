// k_tc.cu -- the mode-to-lag contraction of the batched FP32 form on the
// 5th-generation tensor cores (tcgen05, accumulators in tensor memory).
//
// For every channel c (numerator, Gaussian denominator):
//     acc_c[b][k] += sum_m A_c[b][m] E[m][k]
// where A_c holds the weighted cross/power spectra (one row of modes per
// series) and E = cos/sin(2 pi m tau_k / L) is shared by the batch
// (replacing the type-2 NUFFT of Algorithms 2 and 4).
//
// Precision: FP32 operands are split into TF32 pairs, x = hi + lo, both halves
// rounded to nearest TF32, and each product is formed as
// A_hi E_hi + A_hi E_lo + A_lo E_hi + A_lo E_lo (four tcgen05.mma kind::tf32,
// FP32 accumulation in TMEM), which keeps about 22 significant bits -- the
// FP32 SIMT product's accuracy at tensor-core rate.  Each CTA accumulates one chunk
// of kChunkModes modes in TMEM and adds its partial sums to FP64 accumulators
// in HBM, so long mode sums are combined in FP64.
//
// CTA: 128 series (MMA M) x 128 lags (MMA N) x kChunkModes modes, 128 threads.
// Per K-block of 32 modes the threads load A and E from HBM, split them and
// store them in shared memory in the K-major 128-byte-swizzled layout the MMA
// descriptors describe; thread 0 issues 32 MMAs (4 K-steps x 4 products x 2
// channels) and commits them to an mbarrier that every thread waits on
// (bounded) before the buffers are overwritten.  The two accumulators occupy
// 256 TMEM columns; the epilogue reads them with tcgen05.ld (warp w owns TMEM
// lanes 32w..32w+31, i.e. series b0+32w..) and adds them in FP64.
#include <cstdint>

#include "spectral.cuh"

namespace ncf {
namespace {

constexpr int kTcM = 128;          // series per CTA (MMA M)
constexpr int kTcN = 128;          // lags per CTA (MMA N)
constexpr int kTcKB = 32;          // modes per K-block (128 bytes of FP32 per row)
constexpr int kChunkModes = 128;   // modes per CTA (FP32 accumulation span)
constexpr int kTileBytes = kTcM * kTcKB * 4;   // 16 KiB, one operand tile
constexpr uint32_t kTmemCols = 256;
constexpr long long kSpinLimit = 1ll << 26;    // bounded mbarrier wait

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (r, kk) in a 128-row x 32-col FP32 tile, K-major,
// 128-byte swizzle: 16-byte chunk index XOR (row mod 8) inside each 8-row atom
__device__ __forceinline__ uint32_t sw128(int r, int kk) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((kk >> 2) ^ (r & 7)) << 4) | ((kk & 3) << 2)));
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), Blackwell descriptor version 1
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// instruction descriptor: D FP32, A and B TF32, both K-major, M = 128, N = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                            ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long long limit = kSpinLimit) {
    for (long long it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity));
        if (done) return true;
    }
    return false;
}

// round to the nearest TF32 value (10 stored mantissa bits); the MMA reads only
// those bits, so x = rna(x) + rna(x - rna(x)) is exact to about 2^-22 and its
// error has no sign bias (truncation would bias every product toward zero)
__device__ __forceinline__ float tf32_rn(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__global__ void __launch_bounds__(128, 1)
contract_tc_kernel(const float *__restrict__ Anum, const float *__restrict__ Aden,
                   const float *__restrict__ E, int64_t B, int64_t M2, int64_t Kp,
                   double *__restrict__ acc_num, double *__restrict__ acc_den, int *__restrict__ status) {
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte aligned operand tiles: An_hi An_lo Ad_hi Ad_lo E_hi E_lo
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *tiles = base;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int fail_sh;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t b0 = (int64_t)blockIdx.x * kTcM;
    const int64_t k0 = (int64_t)blockIdx.y * kTcN;
    const int64_t m_lo = (int64_t)blockIdx.z * kChunkModes;
    const int64_t m_hi = min(m_lo + (int64_t)kChunkModes, M2);
    const uint32_t mb = smem_u32(&mbar);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_sh)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb));
        asm volatile("fence.mbarrier_init.release.cluster;");
        fail_sh = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base_sh;
    const uint32_t d_num = tmem, d_den = tmem + kTcN;

    uint32_t parity = 0;
    bool first = true;
    for (int64_t m0 = m_lo; m0 < m_hi; m0 += kTcKB) {
        // ---- load, split and stage the K-block ----
        // A: 128 rows x 32 modes per channel; 4 consecutive modes per thread step
        for (int i = tid; i < kTcM * (kTcKB / 4); i += blockDim.x) {
            const int r = i / (kTcKB / 4), c4 = (i % (kTcKB / 4)) * 4;
            const int64_t gb = b0 + r;
            float4 vn = make_float4(0.f, 0.f, 0.f, 0.f), vd = vn;
            if (gb < B) {
                vn = *reinterpret_cast<const float4 *>(Anum + gb * M2 + m0 + c4);
                vd = *reinterpret_cast<const float4 *>(Aden + gb * M2 + m0 + c4);
            }
            float xn[4] = {vn.x, vn.y, vn.z, vn.w}, xd[4] = {vd.x, vd.y, vd.z, vd.w};
            if (m0 + c4 == 0) {  // the m = 0 term is added exactly in FP64 by the finish kernel
                xn[0] = 0.f;
                xd[0] = 0.f;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t off = sw128(r, c4 + q);
                const float nh = tf32_rn(xn[q]), dh = tf32_rn(xd[q]);
                *reinterpret_cast<float *>(tiles + 0 * kTileBytes + off) = nh;
                *reinterpret_cast<float *>(tiles + 1 * kTileBytes + off) = tf32_rn(xn[q] - nh);
                *reinterpret_cast<float *>(tiles + 2 * kTileBytes + off) = dh;
                *reinterpret_cast<float *>(tiles + 3 * kTileBytes + off) = tf32_rn(xd[q] - dh);
            }
        }
        // E: stored [mode][lag]; the B operand wants lag rows with modes along K
        for (int i = tid; i < kTcKB * kTcN; i += blockDim.x) {
            const int mm = i / kTcN, n = i % kTcN;
            const int64_t gk = k0 + n;
            const float v = gk < Kp ? E[(m0 + mm) * Kp + gk] : 0.f;
            const float vh = tf32_rn(v);
            const uint32_t off = sw128(n, mm);
            *reinterpret_cast<float *>(tiles + 4 * kTileBytes + off) = vh;
            *reinterpret_cast<float *>(tiles + 5 * kTileBytes + off) = tf32_rn(v - vh);
        }
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t t0 = smem_u32(tiles);
#pragma unroll
            for (int ks = 0; ks < kTcKB / 8; ++ks) {
                const uint32_t koff = (uint32_t)ks * 32;  // 8 TF32 = 32 bytes along K
                const uint64_t anh = sdesc(t0 + 0 * kTileBytes + koff), anl = sdesc(t0 + 1 * kTileBytes + koff);
                const uint64_t adh = sdesc(t0 + 2 * kTileBytes + koff), adl = sdesc(t0 + 3 * kTileBytes + koff);
                const uint64_t eh = sdesc(t0 + 4 * kTileBytes + koff), el = sdesc(t0 + 5 * kTileBytes + koff);
                const uint32_t acc0 = (first && ks == 0) ? 0u : 1u;
                mma_tf32(d_num, anh, eh, acc0);
                mma_tf32(d_num, anh, el, 1u);
                mma_tf32(d_num, anl, eh, 1u);
                mma_tf32(d_num, anl, el, 1u);
                mma_tf32(d_den, adh, eh, acc0);
                mma_tf32(d_den, adh, el, 1u);
                mma_tf32(d_den, adl, eh, 1u);
                mma_tf32(d_den, adl, el, 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb));
        }
        // every thread waits before the tiles are rewritten (bounded)
        if (!mbar_wait(mb, parity)) {
            if (tid == 0) atomicOr(status, STATUS_TIMEOUT);
            fail_sh = 1;
        }
        parity ^= 1u;
        first = false;
        __syncthreads();
        if (fail_sh) break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");

    // ---- epilogue: TMEM -> registers -> FP64 atomics ----
    if (!fail_sh && !first) {
        const int64_t gb = b0 + warp * 32 + lane;
        const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
#pragma unroll 1
        for (int ch = 0; ch < 2; ++ch) {
            double *acc = ch == 0 ? acc_num : acc_den;
            const uint32_t dcol = ch == 0 ? d_num : d_den;
#pragma unroll 1
            for (int c0 = 0; c0 < kTcN; c0 += 16) {
                uint32_t v[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
                    "%11, %12, %13, %14, %15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
                      "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                    : "r"(dcol + lane_off + (uint32_t)c0));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                if (gb < B) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int64_t gk = k0 + c0 + q;
                        if (gk < Kp) atomicAdd(acc + gb * Kp + gk, (double)__uint_as_float(v[q]));
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

// Self-test of the bounded wait: an mbarrier phase that nothing completes must
// end in STATUS_TIMEOUT after `limit` polls, with the kernel returning normally.
__global__ void bounded_wait_selftest_kernel(int *status, long long limit) {
    __shared__ __align__(8) unsigned long long mb;
    const uint32_t a = smem_u32(&mb);
    if (threadIdx.x == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(1));
    __syncthreads();
    if (!mbar_wait(a, 0u, limit) && threadIdx.x == 0) atomicOr(status, STATUS_TIMEOUT);
}

}  // namespace

void launch_bounded_wait_selftest(int *status, cudaStream_t st) {
    NCF_LAUNCH("bounded_wait_selftest_kernel", st, bounded_wait_selftest_kernel<<<1, 32, 0, st>>>(status, 4096));
}

size_t contract_tc_smem_bytes() { return 6 * (size_t)kTileBytes + 1024; }

bool contract_tc_supported(int64_t M2) { return M2 % kTcKB == 0; }

void launch_contract_tc(const float *Anum, const float *Aden, const float *E, int64_t B, int64_t M2,
                        int64_t Kp, double *acc_num, double *acc_den, int *status, cudaStream_t st) {
    static std::atomic<unsigned long long> attr_done{0};
    const size_t smem = contract_tc_smem_bytes();
    once_per_device(attr_done, [&] { return set_smem_limit(contract_tc_kernel, smem); });
    dim3 grid((unsigned)((B + kTcM - 1) / kTcM), (unsigned)((Kp + kTcN - 1) / kTcN),
              (unsigned)((M2 + kChunkModes - 1) / kChunkModes));
    NCF_LAUNCH("contract_tc_kernel", st,
               contract_tc_kernel<<<grid, 128, smem, st>>>(Anum, Aden, E, B, M2, Kp, acc_num, acc_den, status));
}

}  // namespace ncf
