"""Seeded synthetic workloads shaped like the paper's test series.

Generators only -- no part of the correlation estimator lives here, so both
the CUDA path and the CPU oracle can be fed from this module.  Each series
draws from its own stream keyed by (seed, workload, series id), so every
workload is reproducible bit for bit on any host.

Workloads (sizes are the defaults; tests pass smaller ones):

* ``ar1_acf``         -- n times uniform on [0, 1000] d, AR(1) values with
  phi = 0.9 in sample order plus N(0, 0.1^2) noise; 50 lags on [0, 100] d.
* ``ou_ccf``          -- two independently sampled series over 10 years with a
  120-day seasonal gap per year; B is A's latent OU signal (tau_c = 20 d)
  delayed by 15 d plus N(0, 0.2^2); 200 lags on [-100, 100] d.
* ``quasi_periodic``  -- one long series at MJD-scale times 60000 + U[0, 20000]
  d: OU-modulated sinusoid (P = 27 d) plus flicker noise; 1000 lags on
  [0, 200] d.
* ``light_curves``    -- B light curves with n log-uniform in [200, 2e5]:
  rotation signal with OU amplitude (Sec. 4.1, Eq. astro_model), flicker noise,
  heteroscedastic log-normal errors, nightly cadence with seasonal and weather
  gaps; shared 256-lag grid on [0, 200] d.

Flicker noise is a sum of 8 exact OU components with correlation times
log-spaced on [0.05, 500] d and equal variances -- a superposition of
Lorentzians whose spectrum is close to 1/f across that band.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 20260903
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libncf_synth.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"], check=True)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.synth_ou.argtypes = [_dp, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_uint64, ctypes.c_uint64, _dp, ctypes.c_int]
        lib.synth_normals.argtypes = [ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64, _dp]
        lib.synth_uniforms.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_uint64, ctypes.c_uint64, _dp]
        lib.synth_cadence.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64, _dp]
        lib.synth_cadence.restype = ctypes.c_int64
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(_dp)


def _stream(workload: int, series: int, part: int) -> int:
    return (workload << 48) ^ (series << 8) ^ part


def ou(t, tau, sigma, seed, stream, out=None):
    """Exact OU process (mean 0, std sigma, correlation time tau) at sorted t."""
    t = np.ascontiguousarray(t, dtype=np.float64)
    acc = out is not None
    if out is None:
        out = np.zeros_like(t)
    _load().synth_ou(_p(t), t.size, float(tau), float(sigma), seed, stream, _p(out), int(acc))
    return out


def normals(n, seed, stream):
    out = np.empty(n)
    _load().synth_normals(n, seed, stream, _p(out))
    return out


def uniforms(n, lo, hi, seed, stream):
    out = np.empty(n)
    _load().synth_uniforms(n, float(lo), float(hi), seed, stream, _p(out))
    return out


def flicker(t, sigma_total, seed, stream_base, n_comp=8, tau_lo=0.05, tau_hi=500.0):
    taus = np.geomspace(tau_lo, tau_hi, n_comp)
    sig = sigma_total / np.sqrt(n_comp)
    out = np.zeros(len(t))
    for c, tau in enumerate(taus):
        ou(t, tau, sig, seed, stream_base + c + 1, out=out)
    return out


@dataclass
class Workload:
    """One workload: CSR-packed series (x at t) and, for a CCF, partners (y at s)."""
    name: str
    t: np.ndarray
    x: np.ndarray
    offs: np.ndarray                      # int64[B+1]
    lags: np.ndarray
    s: np.ndarray | None = None
    y: np.ndarray | None = None
    offs_y: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def B(self) -> int:
        return len(self.offs) - 1

    def series(self, b: int):
        a, e = self.offs[b], self.offs[b + 1]
        if self.s is None:
            return self.t[a:e], self.x[a:e], None, None
        ay, ey = self.offs_y[b], self.offs_y[b + 1]
        return self.t[a:e], self.x[a:e], self.s[ay:ey], self.y[ay:ey]


def ar1_acf(n=2000, K=50, seed=BASE_SEED, series=0):
    """AR(1) (phi = 0.9, burn-in 200) in sample order plus N(0, 0.1^2) noise at
    n sorted uniform times on [0, 1000] d; K lags on [0, 100] d."""
    t = np.sort(uniforms(n, 0.0, 1000.0, seed, _stream(1, series, 0)))
    eta = normals(n + 200, seed, _stream(1, series, 1))
    v = np.empty(n + 200)
    acc = 0.0
    for k in range(n + 200):
        acc = 0.9 * acc + eta[k]
        v[k] = acc
    x = v[200:] + 0.1 * normals(n, seed, _stream(1, series, 2))
    return Workload("ar1_acf", t, x, np.array([0, n], dtype=np.int64), np.linspace(0.0, 100.0, K),
                    meta={"n": n, "K": K})


def _seasonal_times(n, years, gap, seed, stream):
    """n sorted times uniform over the observable part of `years` years of
    365 d, each year's last `gap` days unobserved."""
    obs = 365.0 - gap
    u = uniforms(n, 0.0, years * obs, seed, stream)
    yr = np.floor(u / obs)
    return np.sort(yr * 365.0 + (u - yr * obs))


def ou_ccf(nA=100_000, nB=80_000, K=200, delay=15.0, tau_c=20.0, noise=0.2, years=10, gap=120.0,
           seed=BASE_SEED, series=0):
    """A = OU(tau_c) at tA; B = the same latent OU at sB - delay plus noise."""
    tA = _seasonal_times(nA, years, gap, seed, _stream(2, series, 0))
    sB = _seasonal_times(nB, years, gap, seed, _stream(2, series, 1))
    merged = np.concatenate([tA, sB - delay])
    order = np.argsort(merged, kind="stable")
    lat = ou(merged[order], tau_c, 1.0, seed, _stream(2, series, 2))
    vals = np.empty_like(lat)
    vals[order] = lat
    xA = vals[:nA]
    yB = vals[nA:] + noise * normals(nB, seed, _stream(2, series, 3))
    return Workload("ou_ccf", tA, xA, np.array([0, nA], dtype=np.int64),
                    np.linspace(-100.0, 100.0, K), s=sB, y=yB,
                    offs_y=np.array([0, nB], dtype=np.int64),
                    meta={"nA": nA, "nB": nB, "K": K, "delay": delay})


def quasi_periodic(n=10_000_000, K=1000, t0=60000.0, span=20000.0, period=27.0,
                   seed=BASE_SEED, series=0):
    """OU-modulated sinusoid plus flicker at MJD-scale times t0 + U[0, span]."""
    t = np.sort(uniforms(n, t0, t0 + span, seed, _stream(3, series, 0)))
    amp = 1.0 + ou(t, 220.0, 0.35, seed, _stream(3, series, 1))
    phase = uniforms(1, 0.0, 2 * np.pi, seed, _stream(3, series, 2))[0]
    x = amp * np.cos(2 * np.pi * t / period + phase) + flicker(t, 0.55, seed, _stream(3, series, 16))
    return Workload("quasi_periodic", t, x, np.array([0, n], dtype=np.int64),
                    np.linspace(0.0, 200.0, K), meta={"n": n, "K": K})


def _light_curve(b, n, seed, years=4, season=243, p_weather=0.25, night=0.33):
    lib = _load()
    t = np.empty(n)
    lib.synth_cadence(n, years, season, p_weather, night, seed, _stream(4, b, 0), _p(t))
    par = uniforms(2, 0.0, 1.0, seed, _stream(4, b, 1))
    period = 2.0 + 48.0 * par[0]
    phase = 2 * np.pi * par[1]
    amp = 1.0 + ou(t, 220.0, 0.35, seed, _stream(4, b, 2))
    x = amp * np.cos(2 * np.pi * t / period + phase)
    x += flicker(t, 0.55, seed, _stream(4, b, 16))
    sig = np.exp(-3.0 + 0.5 * normals(n, seed, _stream(4, b, 3)))
    x += sig * normals(n, seed, _stream(4, b, 4))
    return t, x


def light_curve_sizes(B, n_lo=200, n_hi=200_000, seed=BASE_SEED):
    u = uniforms(B, np.log(n_lo), np.log(n_hi), seed, _stream(4, 0xFFFFFF, 9))
    return np.rint(np.exp(u)).astype(np.int64)


def light_curves(B=4096, n_lo=200, n_hi=200_000, K=256, max_lag=200.0, seed=BASE_SEED,
                 sizes=None, threads=None):
    """B light curves packed CSR (offsets int64[B+1]); shared K-lag grid."""
    _load()
    n = light_curve_sizes(B, n_lo, n_hi, seed) if sizes is None else np.asarray(sizes, np.int64)
    offs = np.zeros(B + 1, dtype=np.int64)
    np.cumsum(n, out=offs[1:])
    t = np.empty(int(offs[-1]))
    x = np.empty(int(offs[-1]))

    def one(b):
        tb, xb = _light_curve(b, int(n[b]), seed)
        t[offs[b]:offs[b + 1]] = tb
        x[offs[b]:offs[b + 1]] = xb

    with ThreadPoolExecutor(max_workers=threads or os.cpu_count()) as ex:
        list(ex.map(one, range(B)))
    return Workload("light_curves", t, x, offs, np.linspace(0.0, max_lag, K),
                    meta={"B": B, "K": K, "n_total": int(offs[-1])})
