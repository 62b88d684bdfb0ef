"""FP64 CPU oracle for the kernel-weighted ACF/CCF estimator.

TEST INFRASTRUCTURE ONLY: the plain, slow, obviously correct reference that the
CUDA library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with
the CUDA path and imports nothing from it.

What it computes (Sec. 2.3, Eq. kernel_estimator, with the real-space
algorithms of the appendix for the windowed variant):

    N_k = sum_i sum_j x_std,i * y_std,j * b(d),   B_k = sum_i sum_j b(d),
    c_k = N_k / max(B_k, 1e-16),

with d the deviation of the pair separation from lag tau_k, b the Gaussian
(Eq. Gaussian_kernel) or rectangle (Eq. rectangle_kernel, half-width h as in
Algorithms 6 and 8) kernel, and standardisation x_std = (x - mean) / std with
ddof = 0 (Sec. "Prior standardization").  Optional Pearson normalisation by the
lag-0 values follows Algorithms 4 and 10.

Three evaluators:
  * ``corr(method="direct")``   -- O1, the double sum (C, OpenMP over lags);
  * ``corr(method="windowed")`` -- O2, the two-pointer scan of Algorithms 5-8;
  * ``exact_rectangle`` / ``exact_gaussian`` -- O0, pure-Python enumeration in
    exact rational arithmetic (rectangle) or 50-digit mpmath (Gaussian) for
    inputs of a dozen points.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ncf_oracle.c")
_LIB = os.path.join(_HERE, "libncf_oracle.so")
_lib = None

GAUSSIAN = 0
RECTANGLE = 1
HANNING = 2
_KERNELS = {"gaussian": GAUSSIAN, "rectangle": RECTANGLE, "hanning": HANNING}


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int64)
        lib.oracle_stats.argtypes = [dp, ctypes.c_int64, dp, dp]
        lib.oracle_stats.restype = None
        for name in ("oracle_corr_direct", "oracle_corr_windowed"):
            fn = getattr(lib, name)
            fn.argtypes = [dp, dp, ctypes.c_int64, dp, dp, ctypes.c_int64, dp, ctypes.c_int64,
                           ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                           dp, dp, ip]
            fn.restype = None
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def stats(x):
    """Mean and ddof-0 standard deviation with compensated sums."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    m = ctypes.c_double()
    s = ctypes.c_double()
    _load().oracle_stats(_dp(x), x.size, ctypes.byref(m), ctypes.byref(s))
    return m.value, s.value


def standardise(x):
    """x_std = (x - mean) / std (step 1 of Algorithms 2, 4, 9, 10)."""
    m, s = stats(x)
    if not s > 0.0:
        raise ValueError("zero variance: the standardised series is undefined")
    return (np.asarray(x, dtype=np.float64) - m) / s


def _sums(method, t, x, s, y, lags, kernel, h, trunc_R, eps):
    lib = _load()
    K = lags.size
    num = np.zeros(K)
    den = np.zeros(K)
    cnt = np.zeros(K, dtype=np.int64)
    fn = lib.oracle_corr_direct if method == "direct" else lib.oracle_corr_windowed
    fn(_dp(t), _dp(x), t.size, _dp(s), _dp(y), s.size, _dp(lags), K, kernel, float(h),
       float(trunc_R), int(eps), _dp(num), _dp(den),
       cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return num, den, cnt


def corr(t, x, lags, kernel="gaussian", h=1.0, s=None, y=None, norm="none",
         method="direct", trunc_R=0.0):
    """Kernel-weighted ACF (s, y omitted) or CCF of x at t with y at s.

    Returns a dict with ``c`` (estimate), ``b`` (effective pair count, the
    unclamped denominator), ``count`` (pairs inside the window; the exact
    integer pair count for the rectangle) and ``num`` (the numerator).

    kernel  "gaussian" (sigma = h), "rectangle" (half-width h) or "hanning"
            (the Hann window cos^2(pi d / 2h) / h on |d| <= h: the kernel Sec. 2.3
            names without defining; the rectangle's closed window, Hann weights).
    norm    "none": c = N / max(B, 1e-16) (Eq. kernel_estimator);
            "lag0": Pearson -- ACF divided by its lag-0 value (Algorithm 4),
            CCF divided by sqrt(ACF_x(0) ACF_y(0)) (Algorithm 10).
    method  "direct" (O1) or "windowed" (O2, Algorithms 5-8).
    trunc_R Gaussian window half-width in units of h (0 = untruncated; the
            paper's real-space algorithms use 6).
    """
    kern = _KERNELS[kernel]
    t = np.ascontiguousarray(t, dtype=np.float64)
    lags = np.ascontiguousarray(lags, dtype=np.float64)
    xs = np.ascontiguousarray(standardise(x))
    acf = s is None
    if acf:
        s_, ys, eps = t, xs, +1
    else:
        s_ = np.ascontiguousarray(s, dtype=np.float64)
        ys = np.ascontiguousarray(standardise(y))
        eps = -1
    num, den, cnt = _sums(method, t, xs, s_, ys, lags, kern, h, trunc_R, eps)
    c = num / np.maximum(den, 1e-16)
    if norm == "lag0":
        zero = np.zeros(1)

        def lag0(tt, vv):
            n0, d0, _ = _sums(method, tt, vv, tt, vv, zero, kern, h, trunc_R, +1)
            return n0[0] / max(d0[0], 1e-16)

        if acf:
            c = c / lag0(t, xs)
        else:
            c = c / np.sqrt(lag0(t, xs) * lag0(s_, ys))
    elif norm != "none":
        raise ValueError(f"unknown norm {norm!r}")
    return {"c": c, "b": den, "count": cnt, "num": num}


# --------------------------------------------------------------------------
# O0: exact enumeration for a dozen points.
# --------------------------------------------------------------------------

def _exact_centered(v):
    fr = [Fraction(float(a)) for a in v]
    m = sum(fr, Fraction(0)) / len(fr)
    d = [a - m for a in fr]
    var = sum((a * a for a in d), Fraction(0)) / len(fr)
    return d, var


def exact_rectangle(t, x, lags, h, s=None, y=None):
    """Rectangle estimator by exhaustive enumeration in exact rationals.

    Valid when every centre s_j + eps tau_k and bound centre -/+ h is exactly
    representable in FP64 (dyadic inputs of modest size), so that the FP64
    window predicate of Algorithm 6 and the exact one coincide.  Returns
    (count list of ints, numerator list of mpmath values, c list).
    """
    import mpmath as mp
    mp.mp.dps = 50
    acf = s is None
    tq = [Fraction(float(a)) for a in t]
    xd, vx = _exact_centered(x)
    if acf:
        sq, yd, vy, eps = tq, xd, vx, 1
    else:
        sq = [Fraction(float(a)) for a in s]
        yd, vy = _exact_centered(y)
        eps = -1
    hq = Fraction(float(h))
    scale = mp.sqrt(mp.mpf(vx.numerator) / vx.denominator) * mp.sqrt(mp.mpf(vy.numerator) / vy.denominator)
    counts, nums, cs = [], [], []
    for tau in lags:
        tk = Fraction(float(tau))
        cnt = 0
        acc = Fraction(0)
        for j in range(len(sq)):
            c = sq[j] + eps * tk
            for i in range(len(tq)):
                if c - hq <= tq[i] <= c + hq:
                    cnt += 1
                    acc += xd[i] * yd[j]
        n = mp.mpf(acc.numerator) / acc.denominator / scale
        counts.append(cnt)
        nums.append(n)
        cs.append(n / max(cnt, mp.mpf("1e-16")))
    return counts, nums, cs


def exact_gaussian(t, x, lags, h, s=None, y=None):
    """Untruncated Gaussian estimator summed pair by pair in 50-digit mpmath."""
    import mpmath as mp
    mp.mp.dps = 50
    acf = s is None

    def cen(v):
        vv = [mp.mpf(float(a)) for a in v]
        m = mp.fsum(vv) / len(vv)
        d = [a - m for a in vv]
        sd = mp.sqrt(mp.fsum(a * a for a in d) / len(vv))
        return [a / sd for a in d]

    tm = [mp.mpf(float(a)) for a in t]
    xs = cen(x)
    if acf:
        sm, ys, eps = tm, xs, 1
    else:
        sm = [mp.mpf(float(a)) for a in s]
        ys = cen(y)
        eps = -1
    hm = mp.mpf(float(h))
    norm = 1 / (mp.sqrt(2 * mp.pi) * hm)
    nums, dens, cs = [], [], []
    for tau in lags:
        tk = mp.mpf(float(tau))
        N = []
        B = []
        for j in range(len(sm)):
            c = sm[j] + eps * tk
            for i in range(len(tm)):
                w = norm * mp.exp(-((tm[i] - c) ** 2) / (2 * hm * hm))
                B.append(w)
                N.append(w * xs[i] * ys[j])
        n, d = mp.fsum(N), mp.fsum(B)
        nums.append(n)
        dens.append(d)
        cs.append(n / max(d, mp.mpf("1e-16")))
    return nums, dens, cs



def exact_hanning(t, x, lags, h, s=None, y=None):
    """Hanning estimator summed pair by pair in 50-digit mpmath: weight
    cos^2(pi d / 2h) / h for |d| <= h, d = t_i - (s_j + eps tau), else 0."""
    import mpmath as mp
    mp.mp.dps = 50
    acf = s is None

    def cen(v):
        vv = [mp.mpf(float(a)) for a in v]
        m = mp.fsum(vv) / len(vv)
        d = [a - m for a in vv]
        sd = mp.sqrt(mp.fsum(a * a for a in d) / len(vv))
        return [a / sd for a in d]

    tm = [mp.mpf(float(a)) for a in t]
    xs = cen(x)
    if acf:
        sm, ys, eps = tm, xs, 1
    else:
        sm = [mp.mpf(float(a)) for a in s]
        ys = cen(y)
        eps = -1
    hm = mp.mpf(float(h))
    nums, dens, cs = [], [], []
    for tau in lags:
        tk = mp.mpf(float(tau))
        N, B = [], []
        for j in range(len(sm)):
            c = sm[j] + eps * tk
            for i in range(len(tm)):
                d = tm[i] - c
                if abs(d) <= hm:
                    w = mp.cos(mp.pi * d / (2 * hm)) ** 2 / hm
                    B.append(w)
                    N.append(w * xs[i] * ys[j])
        n, dd = mp.fsum(N), mp.fsum(B)
        nums.append(n)
        dens.append(dd)
        cs.append(n / max(dd, mp.mpf("1e-16")))
    return nums, dens, cs

# ---------------------------------------------------------------------------
# Bootstrap replicates (the resampling the paper recommends for sampling
# uncertainties, Sec. 4 "Monte-Carlo over independent realizations" and
# Sec. 6).  Own implementation of the counter-based generator from its
# published definition: SplitMix64 (Steele, Lea and Flood, "Fast splittable
# pseudorandom number generators", OOPSLA 2014; constants of Vigna's reference
# code), output number c of the stream started at `seed` being
# mix(seed + (c + 1) * 0x9E3779B97F4A7C15 mod 2^64); an index in [0, n) is the
# high word of u * n (Lemire's multiply-high reduction).  Pure Python integers.
# ---------------------------------------------------------------------------
_M64 = (1 << 64) - 1


def splitmix64(seed: int, c: int) -> int:
    """Output number c (0-based) of the SplitMix64 stream started at seed."""
    z = (seed + (c + 1) * 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def bootstrap_indices(n: int, seed: int, r: int) -> np.ndarray:
    """The n point indices of bootstrap replicate r, drawn with replacement
    (draw j = floor(n u / 2^64), u = output 2^32 r + j) and sorted, so the
    replicate keeps time order."""
    idx = [(splitmix64(seed & _M64, (r << 32) | j) * n) >> 64 for j in range(n)]
    return np.sort(np.asarray(idx, dtype=np.int64), kind="stable")


def bootstrap_corr(t, x, lags, r, seed, kernel="gaussian", h=1.0, s=None, y=None, method="windowed",
                   trunc_R=0.0, norm="none"):
    """The estimator on bootstrap replicate r: x side from the stream `seed`,
    y side (a CCF) from the stream ~seed."""
    t, x = np.asarray(t, dtype=np.float64), np.asarray(x, dtype=np.float64)
    ix = bootstrap_indices(t.size, seed, r)
    if s is None:
        return corr(t[ix], x[ix], lags, kernel, h, norm=norm, method=method, trunc_R=trunc_R)
    s, y = np.asarray(s, dtype=np.float64), np.asarray(y, dtype=np.float64)
    iy = bootstrap_indices(s.size, ~seed & _M64, r)
    return corr(t[ix], x[ix], lags, kernel, h, s=s[iy], y=y[iy], norm=norm, method=method, trunc_R=trunc_R)
