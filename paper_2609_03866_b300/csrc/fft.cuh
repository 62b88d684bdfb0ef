// fft.cuh -- complex helpers and the Stockham radix-2/4/8 butterflies of the
// global-memory FFT passes (one launch per pass over every grid of a batch).
//
// Convention: G_k = sum_l g_l exp(+2 pi i k l / n) (the sign that maps spread
// samples at phase u to sum_j z_j exp(+2 pi i m u_j), Eq. nufft_type1).
//
// Stockham autosort pass of radix R at sub-length Ns (Ns = 1, R1, R1 R2, ...):
// for j in [0, n/R), with k = j mod Ns,
//     v_r = a[j + r n/R] * w_{Ns R}^{r k},   v = DFT_R(v),
//     a'[(j / Ns) Ns R + k + r Ns] = v_r,
// where w_M = exp(2 pi i / M).  After the last pass a' is in natural order.
#pragma once

#include <cuda_runtime.h>

namespace ncf {

template <typename R> struct CT;
template <> struct CT<float> { using V = float2; };
template <> struct CT<double> { using V = double2; };

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmul_i(float2 a) { return make_float2(-a.y, a.x); }  // i * a
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmul_i(double2 a) { return make_double2(-a.y, a.x); }

template <typename V> __device__ __forceinline__ V cscale(V a, decltype(a.x) s) {
    V r; r.x = a.x * s; r.y = a.y * s; return r;
}

// In-register DFT of size R with the +i sign.
template <typename V> __device__ __forceinline__ void dft2(V &a, V &b) {
    V t = a; a = cadd(t, b); b = csub(t, b);
}
template <typename V> __device__ __forceinline__ void dft4(V *v) {
    V a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
    V a2 = cadd(v[1], v[3]), a3 = cmul_i(csub(v[1], v[3]));
    v[0] = cadd(a0, a2); v[2] = csub(a0, a2);
    v[1] = cadd(a1, a3); v[3] = csub(a1, a3);
}
template <typename V> __device__ __forceinline__ void dft8(V *v) {
    using Rr = decltype(v[0].x);
    const Rr h = (Rr)0.707106781186547524400844362104849039;
    V e[4] = {v[0], v[2], v[4], v[6]};
    V o[4] = {v[1], v[3], v[5], v[7]};
    dft4(e);
    dft4(o);
    // o_k *= exp(+2 pi i k / 8)
    V o1; o1.x = h * (o[1].x - o[1].y); o1.y = h * (o[1].x + o[1].y);
    V o2 = cmul_i(o[2]);
    V o3; o3.x = -h * (o[3].x + o[3].y); o3.y = h * (o[3].x - o[3].y);
    v[0] = cadd(e[0], o[0]); v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);   v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);   v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);   v[7] = csub(e[3], o3);
}
template <int RAD, typename V> __device__ __forceinline__ void dft(V *v) {
    if constexpr (RAD == 2) dft2(v[0], v[1]);
    else if constexpr (RAD == 4) dft4(v);
    else dft8(v);
}

// Radix plan for n = 2^lg: as many radix-8 passes as possible, then one 4 or 2.
struct RadixPlan {
    int n_pass;
    int radix[24];
};
inline RadixPlan radix_plan(int lg) {
    RadixPlan p{0, {}};
    while (lg >= 3) { p.radix[p.n_pass++] = 8; lg -= 3; }
    if (lg == 2) p.radix[p.n_pass++] = 4;
    if (lg == 1) p.radix[p.n_pass++] = 2;
    return p;
}

}  // namespace ncf
