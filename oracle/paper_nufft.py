"""The paper's own NUFFT estimators, with the smoothing step S_h.

TEST INFRASTRUCTURE ONLY.  This module is the plain reference that the CUDA
implementation of the paper's NUFFT variant is checked against.  Only the test
suite, the smoke check and the benchmark's CPU legs may import it; the product
path never does.  It shares no code with the CUDA library.

What it computes (Appendix "NUFFT-based ACF/CCF algorithms"):
  Algorithm 1  PaddedDomain: L = span + 2 max|tau|, t_c = t_min + span / 2,
               N1 = round(32 n_max L / span) (Eq. N1_default);
  Algorithm 2  CCF: type-1 transforms of both standardised series on the map
               t -> pi + 2 pi (t - t_c) / L, cross-spectrum conj(F1) F2, type-2
               evaluation at the sorted lags (lag 0 prepended), S_h along the
               sorted lag array, division by the pair count, unsorting, division
               by sqrt(ACF_x(0) ACF_y(0)) from Algorithm 3;
  Algorithm 3  AcfScaleAtLag0: the same steps on the symmetric lag array
               -n_h .. n_h, n_h = max(ceil(4 h) + 2, 5), read at its centre;
  Algorithm 4  ACF: one transform, |F|^2, the same evaluation and smoothing,
               normalised by the entry of the prepended lag 0.

The transforms are written as their definitions (the tolerance -> 0 limit of a
NUFFT), with FINUFFT's conventions that the paper states (Sec. "Sign convention
and the non-Hermitian cross-spectrum"): type 1 uses exp(+i k t~), type 2
exp(-i k tau~), and the N1 modes are k = -floor(N1/2) .. ceil(N1/2) - 1.

Readings where the paper is not explicit, each with its reason:
  - S_h, Gaussian: weights exp(-j^2 / (2 h^2)) for |j| <= r, r = int(4 h + 0.5),
    normalised to unit sum; S_h, rectangle: the mean over round(2 h) consecutive
    entries j = i - size//2 .. i - size//2 + size - 1 (round half to even).
    Both treat the array edges by half-sample reflection (... c b a | a b c ...),
    repeated for windows longer than the array.  These are the defaults of
    scipy.ndimage's gaussian_filter1d / uniform_filter1d, which the paper's
    margin rule (n_h >= 4h + 2: "at least 4h on each side") and box size match.
  - PairCount (Algorithms 5 and 6) is the windowed oracle: the Gaussian summed
    in the half-open window [c - 6h, c + 6h), the rectangle counted in the
    closed window [c - h, c + h]; both clamped below at 1e-16.
"""
from __future__ import annotations

import math

import numpy as np

from . import _sums, standardise

GAUSSIAN, RECTANGLE = "gaussian", "rectangle"


def padded_domain(t_min: float, span: float, tau_srt, n_max: int, N1: int | None = None):
    """Algorithm 1: period L, frequency-grid size N1 and centre t_c."""
    if not span > 0.0:
        raise ValueError("the data must span a positive time interval")
    L = span + 2.0 * float(np.max(np.abs(tau_srt)))
    t_c = t_min + span / 2.0
    if N1 is None or N1 <= 0:
        N1 = int(round(32.0 * n_max * L / span))  # Eq. N1_default; Python rounds half to even
    return L, int(N1), t_c


def modes(N1: int) -> np.ndarray:
    """The N1 integer modes of a transform: -floor(N1/2) .. ceil(N1/2) - 1."""
    return np.arange(-(N1 // 2), (N1 + 1) // 2, dtype=np.int64)


def nufft1d1(tt, c, N1: int, block: int = 1 << 22) -> np.ndarray:
    """Type 1 (nonuniform -> modes): F_k = sum_j c_j exp(+i k tt_j), k in modes(N1)."""
    tt = np.asarray(tt, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    k = modes(N1).astype(np.float64)
    out = np.empty(N1, dtype=np.complex128)
    step = max(1, block // max(tt.size, 1))
    for a in range(0, N1, step):
        ph = np.outer(k[a:a + step], tt)
        out[a:a + step] = np.exp(1j * ph) @ c
    return out


def nufft1d2(taut, f, N1: int, block: int = 1 << 22) -> np.ndarray:
    """Type 2 (modes -> nonuniform): c(tau) = sum_k f_k exp(-i k tau~), k in modes(N1)."""
    taut = np.asarray(taut, dtype=np.float64)
    f = np.asarray(f, dtype=np.complex128)
    k = modes(N1).astype(np.float64)
    out = np.zeros(taut.size, dtype=np.complex128)
    step = max(1, block // max(taut.size, 1))
    for a in range(0, N1, step):
        ph = np.outer(taut, k[a:a + step])
        out += np.exp(-1j * ph) @ f[a:a + step]
    return out


def box_size(h: float) -> int:
    """Size round(2h) of the rectangle's box filter (round half to even)."""
    return int(round(2.0 * h))


def smooth(a, kernel: str, h: float) -> np.ndarray:
    """S_h along the array index (the smoothing step of Algorithms 2-4)."""
    a = np.asarray(a, dtype=np.float64)
    n = a.size
    if kernel == GAUSSIAN:
        r = int(4.0 * h + 0.5)
        j = np.arange(-r, r + 1, dtype=np.float64)
        w = np.exp(-0.5 / (h * h) * j * j)
        w = w / w.sum()
        offs = np.arange(-r, r + 1)
    elif kernel == RECTANGLE:
        size = box_size(h)
        if size < 1:
            raise ValueError(f"box filter size round(2h) = {size} for h = {h}")
        offs = np.arange(size) - size // 2
        w = np.full(size, 1.0 / size)
    else:
        raise ValueError(f"S_h is defined for the Gaussian and rectangle kernels, not {kernel!r}")
    out = np.zeros(n)
    for i in range(n):
        acc = 0.0
        for o, wj in zip(offs, w):
            q = (i + int(o)) % (2 * n)       # half-sample reflection, period 2n
            acc += wj * a[q if q < n else 2 * n - 1 - q]
        out[i] = acc
    return out


def pair_count(t_window, t_outer, taus, kernel: str, h: float, eps: int) -> np.ndarray:
    """PairCount (Algorithms 5 and 6): window array t^x, outer array t^y, centre
    c_j = t^y_j + eps tau; Gaussian truncated to [c - 6h, c + 6h); clamped at 1e-16."""
    tw = np.ascontiguousarray(t_window, dtype=np.float64)
    to = np.ascontiguousarray(t_outer, dtype=np.float64)
    taus = np.ascontiguousarray(taus, dtype=np.float64)
    kern = {GAUSSIAN: 0, RECTANGLE: 1}[kernel]
    _, den, _ = _sums("windowed", tw, np.zeros(tw.size), to, np.zeros(to.size), taus, kern, h,
                      6.0 if kernel == GAUSSIAN else 0.0, eps)
    return np.maximum(den, 1e-16)


def _eval_sorted(lags):
    tau_eval = np.concatenate([[0.0], np.asarray(lags, dtype=np.float64)])
    p = np.argsort(tau_eval, kind="stable")
    return tau_eval, p, tau_eval[p]


def raw_correlation(F1, F2, taus, L: float, N1: int) -> np.ndarray:
    """c_raw = Re[type-2 of conj(F1) F2 at 2 pi tau / L] (Algorithm 2)."""
    return np.real(nufft1d2(2.0 * np.pi * np.asarray(taus, dtype=np.float64) / L, np.conj(F1) * F2, N1))


def acf_scale_at_lag0(t, xs, t_c: float, L: float, N1: int, kernel: str, h: float) -> float:
    """Algorithm 3: ACF_x(0) with lag 0 at an interior position of the array."""
    tt = np.pi + 2.0 * np.pi * (np.asarray(t, dtype=np.float64) - t_c) / L
    F = nufft1d1(tt, xs, N1)
    n_h = max(math.ceil(4.0 * h) + 2, 5)
    tau_sym = np.arange(-n_h, n_h + 1, dtype=np.float64)
    c_sm = smooth(raw_correlation(F, F, tau_sym, L, N1), kernel, h)
    b_sym = pair_count(t, t, tau_sym, kernel, h, +1)
    return c_sm[n_h] / max(b_sym[n_h], 1e-16)


def ccf(t, x, s, y, lags, kernel: str = GAUSSIAN, h: float = 1.0, N1: int | None = None) -> dict:
    """Algorithm 2: CCF of x at t with y at s (positive lag: y lags x)."""
    t = np.asarray(t, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    xs, ys = standardise(x), standardise(y)
    _, p, tau_srt = _eval_sorted(lags)
    t_min = min(t.min(), s.min())
    span = max(t.max(), s.max()) - t_min
    L, N1, t_c = padded_domain(t_min, span, tau_srt, max(t.size, s.size), N1)
    F1 = nufft1d1(np.pi + 2.0 * np.pi * (t - t_c) / L, xs, N1)
    F2 = nufft1d1(np.pi + 2.0 * np.pi * (s - t_c) / L, ys, N1)
    c_raw = raw_correlation(F1, F2, tau_srt, L, N1)
    c_sm = smooth(c_raw, kernel, h)
    b_cross = pair_count(t, s, tau_srt, kernel, h, -1)
    c_norm = c_sm / b_cross
    inv = np.argsort(p, kind="stable")
    c_norm, b_cross = c_norm[inv], b_cross[inv]
    scale = math.sqrt(acf_scale_at_lag0(t, xs, t_c, L, N1, kernel, h) *
                      acf_scale_at_lag0(s, ys, t_c, L, N1, kernel, h))
    return {"c": c_norm[1:] / scale, "b": b_cross[1:], "L": L, "N1": N1, "t_c": t_c,
            "c_raw_sorted": c_raw, "tau_sorted": tau_srt}


def acf(t, x, lags, kernel: str = GAUSSIAN, h: float = 1.0, N1: int | None = None) -> dict:
    """Algorithm 4: ACF of x at t, normalised by its (prepended) lag-0 entry."""
    t = np.asarray(t, dtype=np.float64)
    xs = standardise(x)
    _, p, tau_srt = _eval_sorted(lags)
    t_min = t.min()
    span = t.max() - t_min
    L, N1, t_c = padded_domain(t_min, span, tau_srt, t.size, N1)
    F = nufft1d1(np.pi + 2.0 * np.pi * (t - t_c) / L, xs, N1)
    c_raw = raw_correlation(F, F, tau_srt, L, N1)
    c_sm = smooth(c_raw, kernel, h)
    b_eval = pair_count(t, t, tau_srt, kernel, h, +1)
    c_eval = c_sm / b_eval
    inv = np.argsort(p, kind="stable")
    c_eval, b_eval = c_eval[inv], b_eval[inv]
    return {"c": c_eval[1:] / c_eval[0], "b": b_eval[1:], "L": L, "N1": N1, "t_c": t_c,
            "c_raw_sorted": c_raw, "tau_sorted": tau_srt}
