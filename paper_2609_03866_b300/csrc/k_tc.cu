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
// A_hi E_hi + A_hi E_lo + A_lo E_hi (three tcgen05.mma kind::tf32, FP32
// accumulation in TMEM; the dropped A_lo E_lo is below 2^-44 of the product),
// which keeps about 22 significant bits -- the FP32 SIMT product's accuracy at
// tensor-core rate.  The FP32 accumulation runs over spans of 128 modes (4
// K-blocks), whose sums are added to FP64 accumulators in HBM, so long mode sums
// are combined in FP64 (longer FP32 spans raise the error in proportion).
//
// Operands are split once, outside the contraction, into the exact shared-memory
// image the MMA descriptors describe (K-major, 128-byte swizzle, 16 KiB per
// 128-row x 32-mode tile): tc_pack_a_kernel for the spectra of each execution,
// tc_pack_e_kernel for the lag table when a plan is prepared.  A K-block of the
// contraction is then two contiguous bulk copies (cp.async.bulk, completing on
// an mbarrier): 64 KiB of A (numerator hi/lo, denominator hi/lo) and 32 KiB of
// E (hi/lo).
//
// CTA: 128 series (MMA M) x up to 128 lags (MMA N, the last lag tile cut to its
// live lags rounded up to 16) x a run of 128-mode spans; two 96 KiB operand
// stages and two TMEM accumulator sets (2 channels x 128 columns each), warp
// specialised:
//   thread 0       bulk copies of K-block i + 1 while the MMAs of K-block i run;
//   thread 32      24 MMAs per K-block (4 K-steps x 3 products x 2 channels)
//                  into the span's accumulator set, tcgen05.commit releasing the
//                  stage ("empty") and, after a span's last K-block, the set
//                  ("full");
//   warps 2..9     drain a full set while the MMAs fill the other: tcgen05.ld of
//                  16 columns (warp w owns TMEM lanes 32 (w % 4).., one half of
//                  the columns), a transpose through shared memory, FP64 atomics
//                  that each cover 2 series x 16 consecutive lags.
// Every wait has an iteration limit (timeout -> status word; copies in flight
// and issued MMAs awaited, TMEM freed before exit).
#include <cstdint>

#include "spectral.cuh"

namespace ncf {
namespace {

constexpr int kTcM = 128;          // series per CTA (MMA M)
constexpr int kTcN = 128;          // lags per lag tile (largest MMA N used)
constexpr int kTcKB = 32;          // modes per K-block (128 bytes of FP32 per row)
constexpr int kTileBytes = kTcM * kTcKB * 4;   // 16 KiB, one operand tile
constexpr int kAStage = 4 * kTileBytes;        // numerator hi, lo; denominator hi, lo
constexpr int kEStage = 2 * kTileBytes;        // lag table hi, lo
constexpr int kStage = kAStage + kEStage;      // one K-block, 96 KiB
constexpr int kStages = 2;
constexpr uint32_t kTmemCols = 512;        // two accumulator sets x 2 channels x 128
constexpr int kChunkKB = 4;                    // K-blocks per FP32 accumulation span (128 modes)
constexpr int kEpiWarps = 8;                   // two per TMEM lane quadrant
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

// instruction descriptor: D FP32, A and B TF32, both K-major, M = 128, N = n
__device__ __forceinline__ uint32_t idesc_tf32(int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
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

// Spectra rows -> split tiles.  Tile (bt, kb) of A holds series bt*128 + r,
// modes kb*32 + kk at sw128(r, kk) in four 16 KiB parts: numerator hi, lo,
// denominator hi, lo.  Rows past B are zero; so is the m = 0 column (its term
// is added exactly in FP64 by the finish kernel).
__global__ void tc_pack_a_kernel(const float *__restrict__ Anum, const float *__restrict__ Aden, int64_t B,
                                 int64_t M2, unsigned char *__restrict__ At) {
    const int64_t nkb = M2 / kTcKB;
    const int64_t kb = blockIdx.x, bt = blockIdx.y;
    unsigned char *tile = At + ((size_t)bt * nkb + kb) * kAStage;
    for (int i = threadIdx.x; i < kTcM * (kTcKB / 4); i += blockDim.x) {
        const int r = i / (kTcKB / 4), c4 = (i % (kTcKB / 4)) * 4;
        const int64_t gb = bt * kTcM + r, m0 = kb * kTcKB + c4;
        float4 vn = make_float4(0.f, 0.f, 0.f, 0.f), vd = vn;
        if (gb < B) {
            vn = *reinterpret_cast<const float4 *>(Anum + gb * M2 + m0);
            vd = *reinterpret_cast<const float4 *>(Aden + gb * M2 + m0);
        }
        float xn[4] = {vn.x, vn.y, vn.z, vn.w}, xd[4] = {vd.x, vd.y, vd.z, vd.w};
        if (m0 == 0) {
            xn[0] = 0.f;
            xd[0] = 0.f;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t off = sw128(r, c4 + q);
            const float nh = tf32_rn(xn[q]), dh = tf32_rn(xd[q]);
            *reinterpret_cast<float *>(tile + 0 * kTileBytes + off) = nh;
            *reinterpret_cast<float *>(tile + 1 * kTileBytes + off) = tf32_rn(xn[q] - nh);
            *reinterpret_cast<float *>(tile + 2 * kTileBytes + off) = dh;
            *reinterpret_cast<float *>(tile + 3 * kTileBytes + off) = tf32_rn(xd[q] - dh);
        }
    }
}

// Lag table [M2][Kp] -> split tiles.  Tile (nt, kb) holds lags nt*128 + n (the
// B operand's rows), modes kb*32 + mm at sw128(n, mm): hi, then lo.  Lags past
// Kp are zero.
__global__ void tc_pack_e_kernel(const float *__restrict__ E, int64_t M2, int64_t Kp,
                                 unsigned char *__restrict__ Et) {
    const int64_t nkb = M2 / kTcKB;
    const int64_t kb = blockIdx.x, nt = blockIdx.y;
    unsigned char *tile = Et + ((size_t)nt * nkb + kb) * kEStage;
    for (int i = threadIdx.x; i < kTcKB * kTcN; i += blockDim.x) {
        const int mm = i / kTcN, n = i % kTcN;
        const int64_t gk = nt * kTcN + n;
        const float v = gk < Kp ? E[(kb * kTcKB + mm) * Kp + gk] : 0.f;
        const float vh = tf32_rn(v);
        const uint32_t off = sw128(n, mm);
        *reinterpret_cast<float *>(tile + off) = vh;
        *reinterpret_cast<float *>(tile + kTileBytes + off) = tf32_rn(v - vh);
    }
}

// 32 TMEM lanes x 16 columns of 32 bits starting at taddr, one lane per thread
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(mbar)
        : "memory");
}

__global__ void __launch_bounds__(64 + 32 * kEpiWarps, 1)
contract_tc_kernel(const unsigned char *__restrict__ At, const unsigned char *__restrict__ Et, int64_t B,
                   int64_t nkb, int64_t Kp, int kb_per_cta, double *__restrict__ acc_num,
                   double *__restrict__ acc_den, int *__restrict__ status) {
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte aligned stages: [A: num hi, num lo, den hi, den lo][E: hi, lo]
    unsigned char *stages = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages], accf_bar[2], acce_bar[2], done_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int fail_sh, nfill_sh[kStages], ncons_sh[kStages];
    __shared__ float xpose[kEpiWarps * 32 * 17];  // per epilogue warp: 32 rows x 16 lags, padded

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t nt = blockIdx.x, bt = blockIdx.y;
    const int64_t kb0 = (int64_t)blockIdx.z * kb_per_cta;
    const int nk = (int)min((int64_t)kb_per_cta, nkb - kb0);
    const int nch = (nk + kChunkKB - 1) / kChunkKB;             // FP32 accumulation spans
    const int live = (int)min((int64_t)kTcN, Kp - nt * kTcN);  // lags of this tile
    const int n_mma = (live + 15) & ~15;
    const uint32_t idesc = idesc_tf32(n_mma);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_sh)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full_bar[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty_bar[s])));
            nfill_sh[s] = 0;
            ncons_sh[s] = 0;
        }
        for (int s = 0; s < 2; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&accf_bar[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&acce_bar[s])), "r"(kEpiWarps));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done_bar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
        fail_sh = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base_sh;
    const uint32_t sbase = smem_u32(stages);
    volatile int *failed = &fail_sh;

    if (tid == 0) {
        // producer: K-block i into stage i % 2 once the MMAs of K-block i - 2 are done
        for (int i = 0; i < nk && !*failed; ++i) {
            const int s = i & 1, u = i >> 1;
            if (u > 0 && !mbar_wait(smem_u32(&empty_bar[s]), (uint32_t)((u - 1) & 1))) {
                atomicOr(status, STATUS_TIMEOUT);
                atomicExch(&fail_sh, 1);
                break;
            }
            const uint32_t fb = smem_u32(&full_bar[s]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"((uint32_t)kStage)
                         : "memory");
            const uint32_t dst = sbase + (uint32_t)(s * kStage);
            bulk_copy(dst, At + ((size_t)bt * nkb + kb0 + i) * kAStage, kAStage, fb);
            bulk_copy(dst + kAStage, Et + ((size_t)nt * nkb + kb0 + i) * kEStage, kEStage, fb);
            nfill_sh[s] = u + 1;
        }
    } else if (tid == 32) {
        // MMA issuer: K-block i into accumulator set (i / kChunkKB) % 2
        for (int i = 0; i < nk && !*failed; ++i) {
            const int s = i & 1, u = i >> 1;
            const int j = i / kChunkKB, set = j & 1;
            const bool first = i % kChunkKB == 0;
            // a set is reused once the epilogue has drained the chunk two back
            if (first && j >= 2 && !mbar_wait(smem_u32(&acce_bar[set]), (uint32_t)(((j >> 1) - 1) & 1))) {
                atomicOr(status, STATUS_TIMEOUT);
                atomicExch(&fail_sh, 1);
                break;
            }
            if (!mbar_wait(smem_u32(&full_bar[s]), (uint32_t)(u & 1))) {
                atomicOr(status, STATUS_TIMEOUT);
                atomicExch(&fail_sh, 1);
                break;
            }
            ncons_sh[s] = u + 1;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t d_num = tmem + (uint32_t)(set * 2 * kTcN), d_den = d_num + kTcN;
            const uint32_t t0 = sbase + (uint32_t)(s * kStage);
#pragma unroll
            for (int ks = 0; ks < kTcKB / 8; ++ks) {
                const uint32_t koff = (uint32_t)ks * 32;  // 8 TF32 = 32 bytes along K
                const uint64_t anh = sdesc(t0 + 0 * kTileBytes + koff), anl = sdesc(t0 + 1 * kTileBytes + koff);
                const uint64_t adh = sdesc(t0 + 2 * kTileBytes + koff), adl = sdesc(t0 + 3 * kTileBytes + koff);
                const uint64_t eh = sdesc(t0 + 4 * kTileBytes + koff), el = sdesc(t0 + 5 * kTileBytes + koff);
                const uint32_t acc0 = (first && ks == 0) ? 0u : 1u;
                mma_tf32(d_num, anh, eh, idesc, acc0);
                mma_tf32(d_num, anh, el, idesc, 1u);
                mma_tf32(d_num, anl, eh, idesc, 1u);
                mma_tf32(d_den, adh, eh, idesc, acc0);
                mma_tf32(d_den, adh, el, idesc, 1u);
                mma_tf32(d_den, adl, eh, idesc, 1u);
            }
            // the stage is free once these MMAs have read it
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&empty_bar[s])));
            // the chunk's sums are complete once its last MMAs have finished
            if (i % kChunkKB == kChunkKB - 1 || i == nk - 1)
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&accf_bar[set])));
        }
        // completes when every MMA issued above has finished (also after a failure)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&done_bar)));
    } else if (warp >= 2) {
        // epilogue warps: warp w reads TMEM lanes 32 (w % 4) .. + 31, i.e. series
        // bt*128 + 32 (w % 4) + lane, over one half of the lag columns, and adds
        // each chunk's sums in FP64.  The next 16-column load is issued before the
        // current group's atomics.
        const int q = warp & 3, half = (warp - 2) >> 2;
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        float *xp = xpose + (warp - 2) * (32 * 17);
        const int c_lo = half * (kTcN / 2), c_hi = min(c_lo + kTcN / 2, n_mma);
        const int ngrp = c_hi > c_lo ? 2 * ((c_hi - c_lo) / 16) : 0;  // (channel, 16 columns) groups
        for (int j = 0; j < nch; ++j) {
            const int set = j & 1;
            if (!mbar_wait(smem_u32(&accf_bar[set]), (uint32_t)((j >> 1) & 1))) {
                if (lane == 0) atomicOr(status, STATUS_TIMEOUT);
                atomicExch(&fail_sh, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            auto col_of = [&](int g) { return c_lo + 16 * (g >> 1); };
            auto taddr = [&](int g) {
                return tmem + (uint32_t)((set * 2 + (g & 1)) * kTcN + col_of(g)) + lane_off;
            };
            uint32_t v[16];
            if (ngrp > 0) tmem_ld16(taddr(0), v);
#pragma unroll 1
            for (int g = 0; g < ngrp; ++g) {
                // v is read only after this wait (the clobber keeps the stores below it)
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                // transpose the warp's 32 rows x 16 lags through shared memory, so
                // that each atomic instruction covers 2 rows x 16 consecutive lags
                // (two 128-byte segments) instead of 32 rows x 1 lag
#pragma unroll
                for (int e = 0; e < 16; ++e) xp[lane * 17 + e] = __uint_as_float(v[e]);
                __syncwarp();
                if (g + 1 < ngrp) tmem_ld16(taddr(g + 1), v);
                double *acc = (g & 1) ? acc_den : acc_num;
                const int c0 = col_of(g), col = lane & 15;
#pragma unroll 4
                for (int rr = 0; rr < 16; ++rr) {
                    const int r = 2 * rr + (lane >> 4);
                    const int64_t b = bt * kTcM + q * 32 + r;
                    const float val = xp[r * 17 + col];
                    if (b < B && c0 + col < live) atomicAdd(acc + b * Kp + nt * kTcN + c0 + col, (double)val);
                }
                __syncwarp();
            }
            // the set may be overwritten once every epilogue warp has read it
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce_bar[set])) : "memory");
        }
    }
    __syncwarp();
    // before the CTA's shared and tensor memory are released: every MMA issued
    // has finished (done_bar) and, after a failure, every copy still in flight has
    // landed (each wait bounded)
    __syncthreads();
    if (fail_sh && tid == 0) {
        for (int s = 0; s < kStages; ++s)
            if (nfill_sh[s] > ncons_sh[s]) mbar_wait(smem_u32(&full_bar[s]), (uint32_t)((nfill_sh[s] - 1) & 1));
    }
    if (tid == 32) mbar_wait(smem_u32(&done_bar), 0u);  // every MMA issued has finished
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

size_t contract_tc_smem_bytes() { return (size_t)kStages * kStage + 1024; }

bool contract_tc_supported(int64_t M2) { return M2 % kTcKB == 0; }

size_t tc_a_tiles_bytes(int64_t B, int64_t M2) {
    return (size_t)((B + kTcM - 1) / kTcM) * (size_t)(M2 / kTcKB) * kAStage;
}
size_t tc_e_tiles_bytes(int64_t M2, int64_t Kp) {
    return (size_t)((Kp + kTcN - 1) / kTcN) * (size_t)(M2 / kTcKB) * kEStage;
}

void launch_tc_pack_a(const float *Anum, const float *Aden, int64_t B, int64_t M2, unsigned char *At,
                      cudaStream_t st) {
    dim3 grid((unsigned)(M2 / kTcKB), (unsigned)((B + kTcM - 1) / kTcM));
    NCF_LAUNCH("tc_pack_a_kernel", st, tc_pack_a_kernel<<<grid, 256, 0, st>>>(Anum, Aden, B, M2, At));
}

void launch_tc_pack_e(const float *E, int64_t M2, int64_t Kp, unsigned char *Et, cudaStream_t st) {
    dim3 grid((unsigned)(M2 / kTcKB), (unsigned)((Kp + kTcN - 1) / kTcN));
    NCF_LAUNCH("tc_pack_e_kernel", st, tc_pack_e_kernel<<<grid, 256, 0, st>>>(E, M2, Kp, Et));
}

// K-blocks per CTA, a whole number of 4-K-block accumulation spans: the split
// of each tile's spans over CTAs that minimises (waves of one CTA per SM) x
// (spans per CTA), the fewer CTAs on a tie.
int tc_kb_per_cta(int64_t B, int64_t M2, int64_t Kp, int sm_count) {
    const int64_t nkb = M2 / kTcKB;
    const int64_t nch = (nkb + kChunkKB - 1) / kChunkKB;
    const int64_t tiles = ((B + kTcM - 1) / kTcM) * ((Kp + kTcN - 1) / kTcN);
    const int64_t sms = std::max(sm_count, 1);
    int64_t best = 1, best_cost = -1;
    for (int64_t sp = 1; sp <= std::min<int64_t>(nch, 64); ++sp) {
        const int64_t per = (nch + sp - 1) / sp;
        const int64_t cost = ((tiles * sp + sms - 1) / sms) * per;
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = sp;
        }
    }
    return (int)(((nch + best - 1) / best) * kChunkKB);
}

void launch_contract_tc(const unsigned char *At, const unsigned char *Et, int64_t B, int64_t M2, int64_t Kp,
                        int sm_count, double *acc_num, double *acc_den, int *status, cudaStream_t st) {
    static std::atomic<unsigned long long> attr_done{0};
    const size_t smem = contract_tc_smem_bytes();
    once_per_device(attr_done, [&] { return set_smem_limit(contract_tc_kernel, smem); });
    const int64_t nkb = M2 / kTcKB;
    const int per = tc_kb_per_cta(B, M2, Kp, sm_count);
    dim3 grid((unsigned)((Kp + kTcN - 1) / kTcN), (unsigned)((B + kTcM - 1) / kTcM),
              (unsigned)((nkb + per - 1) / per));
    NCF_LAUNCH("contract_tc_kernel", st,
               contract_tc_kernel<<<grid, 64 + 32 * kEpiWarps, smem, st>>>(At, Et, B, nkb, Kp, per, acc_num, acc_den, status));
}

}  // namespace ncf
