"""Benchmark: batched kernel-weighted ACFs of 4096 irregularly sampled light
curves on one B300 (or N GPUs, weak scaling: every rank runs its own batch).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ncf|reference]

Workload: 4096 light curves, n log-uniform in [200, 2e5] (sum ~1.1e8 points),
rotation signal with OU amplitude, flicker noise, heteroscedastic errors,
nightly cadence with seasonal and weather gaps; shared 256-lag grid on
[0, 200] d; Gaussian kernel h = 0.5 d and rectangle half-width 0.5 d.

A step is the whole hot path over the batch: one statistics pass, the Gaussian
ACFs through the batched FP32 form (spreading, FFT, spectra, mode-to-lag
contraction on tensor cores) and the rectangle ACFs through the exact
pair-count scan, each with its normalisation.  Both estimators are one plan
(analysis done once, ncf_plan_create_multi) whose launches are captured in a
CUDA graph; a step replays it.  Series-lags per step = 2 * 4096 * 256 (one per
estimator).

One JSON line is printed (rank 0): the device-timed throughput (`value`) and
each estimator's own rate; the same metric end to end through the host-buffer
C call that evaluates both estimators from one upload of the batch (`e2e`);
the spec comparison of the FP32 form with the plain FP64 GPU path (the
faster of the FP64 spectral and FP64 windowed paths) on the Gaussian, with the
FP32 form's error on every value; accuracy against the FP64 oracle on sampled
series; the roofline of the dominant kernel; the single-series FP64 ACF and the
10^7-point MJD-offset precision workloads; serving; the library's device
memory high-water mark; and the oracle timed on this host's cores
(`cpu_baseline`).  `--impl reference` times only the oracle.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

B_SERIES = 4096
K_LAGS = 256
H = 0.5
METRIC = ("series*lags/s, batched FP32 form (Gaussian) + exact rectangle scan, 4096 light curves x 256 lags, "
          "one series*lag per estimator")
WORKLOAD = "light_curves: 4096 series, n log-uniform [200, 2e5], 256 lags on [0, 200] d, Gaussian h=0.5 + rectangle h=0.5"


# DRAM bytes per launch of a kernel at the default workload (4096 light curves x 256
# lags), dram__bytes_read.sum + dram__bytes_write.sum from one single-pass ncu capture of
# this command.  Reported as the roofline's traffic only for that workload; update or
# remove an entry whenever its kernel changes.
MEASURED_TRAFFIC = {("rect_scan_pt_kernel", 4096): 3.0136e9 + 30.24e6}


# Integer rates of this GPU measured by a probe of independent instruction chains
# (ops per clock per SM): IADD3 120 (full rate), LOP3 / SHF / IMAD / IMAD.WIDE 60
# (half rate).  The scan's 16 algorithmic int32 operations per item are 8 of each
# kind (the 64-bit adds and differences full rate; the compares and the limb
# multiply-adds half rate): 8/120 + 8/60 = 0.2 clock per item per SM, i.e. 80
# operations per clock per SM.
INT_OPS_PER_CLK_SM = 80.0


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    except Exception:
        return 6400.0, 1800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms, logged to
    $NCF_CLOCKS_DIR/clocks_gpu<index>.csv (default: the system temporary directory)."""

    def __init__(self, index: int):
        import tempfile
        self.index = index
        self.proc = None
        self.path = os.path.join(os.environ.get("NCF_CLOCKS_DIR", tempfile.gettempdir()), f"clocks_gpu{index}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [v.strip() for v in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_sample(w, n_series=64, n_lags=16, seed=7):
    """Bounded sample of the workload for the oracle: random series, a subset
    of the lags (the oracle's cost is linear in the number of lags)."""
    rng = np.random.default_rng(seed)
    series = np.sort(rng.choice(w.B, size=min(n_series, w.B), replace=False))
    lag_idx = np.sort(rng.choice(len(w.lags), size=min(n_lags, len(w.lags)), replace=False))
    return series, lag_idx


def time_oracle(w, series, lag_idx):
    """Oracle (windowed FP64 scan of the paper's real-space algorithms, OpenMP
    over lags) on the sample; both kernels.  Returns (series*lags/s, seconds,
    results)."""
    import oracle
    lags = w.lags[lag_idx]
    res = {}
    t0 = time.perf_counter()
    for b in series:
        tb, xb, _, _ = w.series(int(b))
        res[("gaussian", int(b))] = oracle.corr(tb, xb, lags, "gaussian", H, method="windowed", trunc_R=8)
        res[("rectangle", int(b))] = oracle.corr(tb, xb, lags, "rectangle", H, method="windowed")
    dt = time.perf_counter() - t0
    return 2 * len(series) * len(lags) / dt, dt, res


def reference_arm(args, rank, world):
    from paper_2609_03866_b300 import synth
    if rank != 0:
        return
    w = synth.light_curves(B=B_SERIES, K=K_LAGS)
    series, lag_idx = cpu_sample(w)
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state; its steps are independent
    rates, secs = [], []
    for s in range(args.steps):
        r, dt, _ = time_oracle(w, series, lag_idx)
        rates.append(r)
        secs.append(dt)
    value = float(np.median(rates))
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "series*lags/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * float(np.median(secs)), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "B": B_SERIES, "K": K_LAGS},
        "cpu_baseline": {"value": value, "unit": "series*lags/s", "cores": cores, "kind": "oracle",
                         "sample": f"{len(series)} random series x {len(lag_idx)} of 256 lags, both kernels, "
                                   "FP64 windowed scan (Gaussian window 8h)"},
        "e2e": {"value": value, "unit": "series*lags/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def bootstrap_run(api, device, n=20_000, K=256, n_boot=1024, seed=5):
    """Bootstrap replicates of one light curve, resampled and evaluated on the GPU
    (Gaussian FP32 form and rectangle exact scan), timed with CUDA events."""
    import torch
    from paper_2609_03866_b300 import synth
    w = synth.light_curves(B=1, K=K, sizes=[n], seed=synth.BASE_SEED + 2024)
    dev = torch.device("cuda", device)
    t, x, lags = (torch.from_numpy(a).to(dev) for a in (w.t, w.x, w.lags))
    ctx = api.Context(device)
    stream = torch.cuda.current_stream(dev)

    def step():
        api.corr_bootstrap(t, x, lags, n_boot, seed, kernel="gaussian", h=H, path="spectral", precision="fp32",
                           ctx=ctx, stream=stream)
        api.corr_bootstrap(t, x, lags, n_boot, seed, kernel="rectangle", h=H, ctx=ctx, stream=stream)

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(3):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 3
    ctx.close()
    return {"replicates": n_boot, "points": n, "K": K, "ms_per_step": ms,
            "value": 2.0 * n_boot * K / (ms / 1e3), "unit": "series*lags/s",
            "step": "Gaussian FP32 form + rectangle exact scan on every replicate, resampling included"}


def regular_run(api, device, n=256_000, K=366, h=1.0):
    """Classic-FFT path on a regular daily grid at the paper's regular-data benchmark size
    (n = 2.56e5, K = 366 lags), both kernels, inputs resident, timed with CUDA events."""
    import torch
    rng = np.random.default_rng(17)
    e = rng.normal(size=n)
    x = np.empty(n)
    acc = 0.0
    for i in range(n):           # AR(1), phi = 0.9
        acc = 0.9 * acc + e[i]
        x[i] = acc
    dev = torch.device("cuda", device)
    m = torch.arange(n, dtype=torch.int64, device=dev)
    xd = torch.from_numpy(x).to(dev)
    lags = torch.arange(K, dtype=torch.float64, device=dev)
    ctx = api.Context(device)
    stream = torch.cuda.current_stream(dev)
    out = {}
    for kernel in ("gaussian", "rectangle"):
        for _ in range(3):
            api.corr_regular(m, xd, 1.0, lags, kernel=kernel, h=h, ctx=ctx, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(5):
            api.corr_regular(m, xd, 1.0, lags, kernel=kernel, h=h, ctx=ctx, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        out[kernel + "_ms"] = e0.elapsed_time(e1) / 5
    ctx.close()
    out.update({"n": n, "K": K, "h": h, "unit": "ms per ACF (one call, host read-back of the lattice range included)",
                "paper": "fitted FFT-path times at n = 2.56e5: 70 ms (Gaussian), 40 ms (rectangle) on a "
                         "quad-core 2 GHz Intel Core i5 laptop (context, other hardware)"})
    return out


def spectral_k1024_run(api, device, B=1024, K=1024, h=0.5, reps=3):
    """The FP32 form on 1024 light curves x 1024 lags (the serving config's
    largest lag grid), Gaussian h = 0.5: a profiling workload for the
    contraction (9 lag tiles) and the spreading.  Per-kernel times from the
    context's profiler on the last of `reps` calls."""
    import torch
    from paper_2609_03866_b300 import synth
    w = synth.light_curves(B=B, K=K)
    dev = torch.device("cuda", device)
    t, x, lags = (torch.as_tensor(a, device=dev) for a in (w.t, w.x, w.lags))
    ctx = api.Context(device)
    for i in range(reps):
        if i == reps - 1:
            ctx.profile_reset()
            ctx.profile(True)
        api.corr_batch(w.offs, t, x, lags, kernel="gaussian", h=h, path="spectral", precision="fp32", ctx=ctx)
    torch.cuda.synchronize()
    rep = ctx.profile_report()
    ctx.close()
    return {"workload": f"{B} light curves ({w.t.size} points) x {K} lags on [0, 200] d, Gaussian h = {h}, FP32 form",
            "kernels_ms": {k: v[1] for k, v in sorted(rep.items(), key=lambda kv: -kv[1][1])}}


def mixed_spans_run(api, device, B=4096, K=128, h=0.5, seed=29):
    """Per-series grid sizing: 4096 series whose spans are log-uniform in
    [20, 1460] d (uniform times, n log-uniform in [200, 2e4], a sinusoid plus
    noise), 128 lags on [0, 10] d, Gaussian h = 0.5, FP32 form.  Two plans on
    the same inputs, one split into grid-size buckets and one on a common grid
    (NCF_SPEC_BUCKETS=0), each timed over 10 executions with CUDA events."""
    import os
    import torch
    rng = np.random.default_rng(seed)
    spans = np.exp(rng.uniform(np.log(20.0), np.log(1460.0), B))
    ns = np.rint(np.exp(rng.uniform(np.log(200.0), np.log(2e4), B))).astype(np.int64)
    offs = np.zeros(B + 1, dtype=np.int64)
    np.cumsum(ns, out=offs[1:])
    t = np.empty(int(offs[-1]))
    x = np.empty(int(offs[-1]))
    for b in range(B):
        tb = np.sort(rng.uniform(0.0, spans[b], ns[b])) + 50000.0
        t[offs[b]:offs[b + 1]] = tb
        x[offs[b]:offs[b + 1]] = np.sin(2 * np.pi * tb / rng.uniform(2, 40)) + rng.normal(size=ns[b])
    dev = torch.device("cuda", device)
    T, X = torch.as_tensor(t, device=dev), torch.as_tensor(x, device=dev)
    lags = torch.linspace(0.0, 10.0, K, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    res = {}
    for name, env in (("split", None), ("one_grid", "0")):
        old = os.environ.get("NCF_SPEC_BUCKETS")
        if env is None:
            os.environ.pop("NCF_SPEC_BUCKETS", None)
        else:
            os.environ["NCF_SPEC_BUCKETS"] = env
        try:
            ctx = api.Context(device)
            plan = api.Plan(offs, T, X, lags, kernel="gaussian", h=h, path="spectral", precision="fp32", ctx=ctx,
                            stream=stream)
            info = ctx.last_plan()
            out = None
            for _ in range(3):
                out = plan.execute(T, X, out=out, stream=stream)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(10):
                plan.execute(T, X, out=out, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            res[name] = {"ms": e0.elapsed_time(e1) / 10, "buckets": int(info["buckets"]),
                         "largest_grid": int(info["grid"]), "device_bytes": plan.device_bytes,
                         "c": out["c"].clone()}
            plan.close()
            ctx.close()
        finally:
            if old is None:
                os.environ.pop("NCF_SPEC_BUCKETS", None)
            else:
                os.environ["NCF_SPEC_BUCKETS"] = old
    diff = float((res["split"]["c"] - res["one_grid"]["c"]).abs().max().item())
    for r in res.values():
        r.pop("c")
    return {"workload": f"{B} series, spans log-uniform [20, 1460] d, n log-uniform [200, 2e4] "
                        f"({int(offs[-1])} points), {K} lags on [0, 10] d, Gaussian h = {h}, FP32 form",
            "split": res["split"], "one_grid": res["one_grid"],
            "speedup": res["one_grid"]["ms"] / res["split"]["ms"], "max_abs_diff_split_vs_one_grid": diff,
            "unit": "ms per plan execution (device-resident inputs)"}


def hanning_run(api, device, h=0.5):
    """Hanning kernel (FP64 windowed path) on the seasonal OU CCF at full size
    (1e5 x 8e4 points, 200 lags), beside the exact rectangle scan on the same data,
    and the spectral-sinc rectangle (FP64 spectral path, tol 1e-2) with its error
    against that exact scan."""
    import torch
    from paper_2609_03866_b300 import synth
    w = synth.ou_ccf()
    dev = torch.device("cuda", device)
    t, x, s, y, lags = (torch.from_numpy(a).to(dev) for a in (w.t, w.x, w.s, w.y, w.lags))
    ctx = api.Context(device)
    stream = torch.cuda.current_stream(dev)
    out = {}
    for kernel in ("hanning", "rectangle"):
        for _ in range(3):
            api.corr(t, x, lags, kernel=kernel, h=h, s=s, y=y, ctx=ctx, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(5):
            api.corr(t, x, lags, kernel=kernel, h=h, s=s, y=y, ctx=ctx, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        out[kernel + "_ms"] = e0.elapsed_time(e1) / 5
    # the spectral-sinc rectangle on the same data, against the exact scan's result
    exact = api.corr(t, x, lags, kernel="rectangle", h=h, s=s, y=y, ctx=ctx, stream=stream)["c"]
    sinc_tol = 1e-2
    sinc = lambda: api.corr(t, x, lags, kernel="rectangle", h=h, s=s, y=y, path="spectral", tol=sinc_tol,
                            ctx=ctx, stream=stream)
    approx = sinc()["c"]
    torch.cuda.synchronize()
    for _ in range(2):
        sinc()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(3):
        sinc()
    e1.record(stream)
    torch.cuda.synchronize()
    out["spectral_sinc"] = {"tol": sinc_tol, "ms": e0.elapsed_time(e1) / 3,
                            "max_abs_err_vs_exact_scan": float((approx - exact).abs().max())}
    ctx.close()
    out.update({"workload": "seasonal OU CCF, 1e5 x 8e4 points, 200 lags on [-100, 100] d, h = 0.5 d"})
    return out


def paper_run(api, device, h=0.5):
    """The paper's own NUFFT estimators (Algorithms 1-4 with the smoothing step, default N1)
    on the seasonal OU CCF at full size (1e5 x 8e4 points, 200 lags), both kernels, beside
    the b-hat spectral FP64 path on the same data.  Each call synchronises with the host
    (statistics, lags, pair counts), so the events around it measure the whole call.  The
    direct mode-sum kernel's time comes from the context's kernel profiler; its FP64 work
    is 6 operations per (mode, lag): a rotation (2 FMA + 2 MUL) and 2 FMA of accumulation.
    With 201 sorted lags the sorted array goes through the type-2 transform (one FFT)
    and the direct sum covers Algorithm 3's two symmetric arrays."""
    import math
    import torch
    from paper_2609_03866_b300 import synth
    w = synth.ou_ccf()
    dev = torch.device("cuda", device)
    t, x, s, y, lags = (torch.from_numpy(a).to(dev) for a in (w.t, w.x, w.s, w.y, w.lags))
    ctx = api.Context(device)
    stream = torch.cuda.current_stream(dev)
    span = max(w.t.max(), w.s.max()) - min(w.t.min(), w.s.min())
    L = span + 2.0 * np.abs(np.concatenate([[0.0], w.lags])).max()
    N1 = int(round(32.0 * max(w.t.size, w.s.size) * L / span))
    Mh = N1 // 2
    K1 = w.lags.size + 1
    out = {"workload": "seasonal OU CCF, 1e5 x 8e4 points, 200 lags on [-100, 100] d", "N1": N1,
           "unit": "ms per CCF (one call)"}

    def timed(fn, reps=3):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    for kernel, hh in (("gaussian", h), ("rectangle", 1.0)):
        call = lambda: api.corr_paper(t, x, lags, kernel=kernel, h=hh, s=s, y=y, ctx=ctx, stream=stream)
        ms = timed(call)
        ctx.profile_reset()
        ctx.profile(True)
        call()
        rep = ctx.profile_report()
        ctx.profile(False)
        ctx.profile_reset()
        n_h = max(math.ceil(4 * hh) + 2, 5)
        # the direct mode sum evaluates the symmetric arrays of Algorithm 3, and the
        # sorted lags only below 48 of them (above, a type-2 transform does)
        flops = 6.0 * (Mh + 1) * ((K1 if K1 < 48 else 0) + 2 * (2 * n_h + 1))
        ev_ms = rep.get("paper_eval_kernel", (0, float("nan")))[1]
        out[kernel] = {"h": hh, "ms": ms, "eval_kernel_ms": ev_ms,
                       "eval_fp64_tflops": flops / (ev_ms * 1e-3) / 1e12,
                       "kernels_ms": {k: round(v[1], 3) for k, v in rep.items()}}
    out["bhat_spectral_fp64_gaussian_ms"] = timed(lambda: api.corr(t, x, lags, kernel="gaussian", h=h, s=s, y=y,
                                                                  path="spectral", precision="fp64",
                                                                  norm="lag0", ctx=ctx, stream=stream))
    ctx.close()
    return out


def fp64_plain_run(api, ctx, stream, w, offs, t, x, lags, out_g, c32, g_ms, world):
    """The spec comparison on the Gaussian: the FP32 form against the plain
    FP64 GPU path, the faster of (i) the FP64 spectral path on the whole batch and
    (ii) the FP64 windowed path (8h window), timed on 16 series at evenly spaced
    size ranks and extrapolated to the batch by its work (points x lags x points
    in the window, the cost model of the windowed scan).  The FP32 form's error is
    taken against the FP64 spectral result on every value of the batch."""
    import torch
    B, K = w.B, lags.numel()

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    spec_ms = timed(lambda: api.corr_batch(offs, t, x, lags, kernel="gaussian", h=H, path="spectral",
                                           precision="fp64", ctx=ctx, stream=stream, out=out_g))
    c64 = out_g["c"].clone()
    diff = (c32 - c64).abs()
    # windowed: a sample of series at evenly spaced size ranks
    n = np.diff(offs)
    span = np.array([w.t[offs[b + 1] - 1] - w.t[offs[b]] for b in range(B)])
    R = 8.0
    work = n.astype(np.float64) * K * np.minimum(n, n / np.maximum(span, 1e-300) * 2 * R * H + 1)
    rank = np.argsort(n)
    sample = rank[np.linspace(0, B - 1, 16).astype(int)]
    so = np.concatenate([[0], np.cumsum(n[sample])]).astype(np.int64)
    ts = np.concatenate([w.t[offs[b]:offs[b + 1]] for b in sample])
    xs = np.concatenate([w.x[offs[b]:offs[b + 1]] for b in sample])
    dev = t.device
    tsd, xsd = torch.from_numpy(ts).to(dev), torch.from_numpy(xs).to(dev)
    win_sample_ms = timed(lambda: api.corr_batch(so, tsd, xsd, lags, kernel="gaussian", h=H, path="windowed",
                                                 precision="fp64", trunc_R=R, ctx=ctx, stream=stream), reps=1)
    win_ms = win_sample_ms * work.sum() / work[sample].sum()
    plain_ms = min(spec_ms, win_ms)
    return {
        "gaussian_fp32_form": {"ms": g_ms, "value": B * K * world / (g_ms / 1e3), "unit": "series*lags/s",
                               "max_abs_err_vs_fp64_every_value": float(diff.max().item()),
                               "rms_err_vs_fp64": float(diff.pow(2).mean().sqrt().item()),
                               "values_compared": int(diff.numel())},
        "plain_fp64_gpu_path": {"ms": plain_ms, "value": B * K * world / (plain_ms / 1e3),
                                "unit": "series*lags/s",
                                "path": "FP64 spectral" if spec_ms <= win_ms else "FP64 windowed (extrapolated)"},
        "fp64_spectral_ms": spec_ms,
        "fp64_windowed_ms_extrapolated": win_ms,
        "fp64_windowed_sample": {"series": int(len(sample)), "points": int(n[sample].sum()), "ms": win_sample_ms,
                                 "share_of_batch_work": float(work[sample].sum() / work.sum())},
        "speedup_fp32_form": plain_ms / g_ms,
        "target": "FP32 form within 1e-5 of FP64 on every value and faster than the plain FP64 GPU path",
        "met": bool(diff.max().item() <= 1e-5 and g_ms < plain_ms),
    }


def single_acf_run(api, device):
    """A single ACF in FP64: AR(1) (phi = 0.9) at 2000 uniform times on [0, 1000] d,
    50 lags on [0, 100] d; Gaussian h = 1 (path chosen by the cost model) and
    rectangle half-width 1; every value against the oracle's direct double sum,
    counts exactly."""
    import torch
    import oracle
    from paper_2609_03866_b300 import synth
    w = synth.ar1_acf(n=2000, K=50)
    dev = torch.device("cuda", device)
    t, x, lags = (torch.from_numpy(a).to(dev) for a in (w.t, w.x, w.lags))
    ctx = api.Context(device)
    stream = torch.cuda.current_stream(dev)
    out = {}
    for kernel in ("gaussian", "rectangle"):
        call = lambda: api.corr(t, x, lags, kernel=kernel, h=1.0, ctx=ctx, stream=stream)
        for _ in range(3):
            call()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(20):
            r = call()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 20
        ref = oracle.corr(w.t, w.x, w.lags, kernel, 1.0)
        got = {k: v.cpu().numpy() for k, v in r.items()}
        d = {"ms": ms, "value": w.lags.size / (ms / 1e3), "unit": "series*lags/s",
             "max_abs_err_vs_oracle": float(np.max(np.abs(got["c"] - ref["c"]))), "tolerance": 1e-10}
        if kernel == "rectangle":
            d["counts_bit_exact"] = bool(np.array_equal(got["count"], ref["count"]))
        out[kernel] = d
    ctx.close()
    out["workload"] = "AR(1) phi = 0.9, n = 2000 on [0, 1000] d, 50 lags on [0, 100] d, h = 1 (one call, FP64)"
    return out


def precision_run(api, device, h=0.1):
    """The precision workload: one ACF of 10^7 points at times 60000 + U[0, 20000] d
    (MJD scale), an OU-modulated 27-d sinusoid plus flicker noise, 1000 lags on
    [0, 200] d, Gaussian h = 0.1 d: the FP32 form (FP32 spreading and FFT, tensor-
    core lag evaluation) against the FP64 spectral path on every lag."""
    import torch
    from paper_2609_03866_b300 import synth
    w = synth.quasi_periodic(n=10_000_000, K=1000)
    dev = torch.device("cuda", device)
    t, x, lags = (torch.from_numpy(a).to(dev) for a in (w.t, w.x, w.lags))
    ctx = api.Context(device)
    stream = torch.cuda.current_stream(dev)
    res, ms = {}, {}
    for prec in ("fp32", "fp64"):
        call = lambda: api.corr(t, x, lags, kernel="gaussian", h=h, path="spectral", precision=prec, ctx=ctx,
                                stream=stream)
        call()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res[prec] = call()["c"]
        e1.record(stream)
        torch.cuda.synchronize()
        ms[prec] = e0.elapsed_time(e1)
    d = (res["fp32"] - res["fp64"]).abs()
    plan = ctx.last_plan()
    ctx.close()
    return {"workload": "10^7 points at 60000 + U[0, 20000] d, 1000 lags on [0, 200] d, Gaussian h = 0.1 d",
            "fp32_form_ms": ms["fp32"], "fp64_ms": ms["fp64"],
            "fp32_form_value": 1000 / (ms["fp32"] / 1e3), "fp64_value": 1000 / (ms["fp64"] / 1e3),
            "unit": "series*lags/s", "max_abs_diff_fp32_vs_fp64": float(d.max().item()),
            "rms_abs_diff_fp32_vs_fp64": float(d.pow(2).mean().sqrt().item()), "lags_compared": int(d.numel()),
            "grid": plan["grid"], "modes": plan["modes"]}


def serve_pool(n_pool=32, n_lo=1_000, n_hi=5_000_000, seed=11):
    """Request templates of the serving mix: half ACF light curves, half seasonal OU
    CCFs (n_B = 0.8 n_A); n log-uniform in [n_lo, n_hi]; K in {64, 256, 1024};
    Gaussian (FP32 form) or rectangle (exact scan), h = 0.5."""
    from paper_2609_03866_b300 import synth
    rng = np.random.default_rng(seed)
    pool = []
    for i in range(n_pool):
        n = int(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        K = int(rng.choice([64, 256, 1024]))
        kernel = "gaussian" if rng.random() < 0.5 else "rectangle"
        if i % 2 == 0:
            w = synth.light_curves(B=1, K=K, sizes=[n], seed=synth.BASE_SEED + 1000 + i)
            r = dict(t=w.t, x=w.x, lags=w.lags)
        else:
            w = synth.ou_ccf(nA=n, nB=max(2, int(0.8 * n)), K=K, series=1000 + i)
            r = dict(t=w.t, x=w.x, s=w.s, y=w.y, lags=w.lags)
        r.update(kernel=kernel, h=H)
        if kernel == "gaussian":
            r.update(path="spectral", precision="fp32")
        pool.append(r)
    return pool


def serve_run(api, device, n_req=5000, slots=4, seed=11):
    """Request stream through the serving loop.  A closed loop (slots requests
    kept in flight) gives the saturation throughput; open Poisson streams at 0.5,
    0.8 and 1.0 of it give the latency a client sees (queueing on the client
    while no slot is free + the server's submit-to-done time).  Every template's
    series are also resident on the device; half the requests name them by
    handle, the other half send their host arrays and pay their own upload."""
    rng = np.random.default_rng(seed)
    pool = serve_pool(seed=seed)
    order = rng.integers(0, len(pool), size=n_req)
    host = rng.random(n_req) < 0.5
    srv = api.Server(device=device, slots=slots, mem_budget_bytes=48 << 30)
    reqs, hreqs = [], []
    for r in pool:
        q = {k: v for k, v in r.items() if k not in ("t", "x", "s", "y")}
        q["x_series"] = srv.put(r["t"], r["x"])
        if "s" in r:
            q["y_series"] = srv.put(r["s"], r["y"])
        reqs.append(q)
        hreqs.append(dict(r))

    def submit(i, block=False):
        while True:
            if i >= 0:
                j = int(order[i % n_req])
                r = dict(hreqs[j] if host[i % n_req] else reqs[j])
            else:
                r = dict(reqs[-1 - i])
            if "x_series" not in r:
                t_, x_ = r.pop("t"), r.pop("x")
                try:
                    return srv.submit(t_, x_, r.pop("lags"), **r)
                except api.NcfError as e:
                    if e.status != api.Server.EBUSY:
                        raise
                    if not block:
                        return None
                    time.sleep(1e-3)
                    continue
            try:
                return srv.submit(None, None, r.pop("lags"), **r)
            except api.NcfError as e:
                if e.status != api.Server.EBUSY:
                    raise
                if not block:
                    return None
                time.sleep(1e-3)

    for i in range(len(pool)):              # every template once: warm workspaces and tuners
        srv.wait(submit(-1 - i, block=True))
    lags_of = lambda i: pool[int(order[i % n_req])]["lags"].size
    # closed loop
    t0 = time.perf_counter()
    inflight, nxt, done_k = [], 0, 0
    while nxt < n_req or inflight:
        while nxt < n_req and len(inflight) < slots:
            tk = submit(nxt)
            if tk is None:
                break
            inflight.append((tk, nxt))
            nxt += 1
        done = [(tk, i) for tk, i in inflight if srv.done(tk)]
        for tk, i in done:
            srv.wait(tk)
            inflight.remove((tk, i))
            done_k += lags_of(i)
        if not done:
            time.sleep(50e-6)
    dt_closed = time.perf_counter() - t0
    rate = n_req / dt_closed
    loads = []
    for load in (0.5, 0.8, 1.0):
        arr = np.cumsum(rng.exponential(1.0 / (load * rate), size=n_req))
        lat, inflight, nxt = [], {}, 0
        t0 = time.perf_counter()
        while nxt < n_req or inflight:
            now = time.perf_counter() - t0
            while nxt < n_req and arr[nxt] <= now:
                tk = submit(nxt)
                if tk is None:
                    break
                inflight[tk] = (time.perf_counter() - t0) - arr[nxt]
                nxt += 1
            done = [tk for tk in inflight if srv.done(tk)]
            for tk in done:
                lat.append(inflight.pop(tk) * 1e3 + srv.wait(tk)["latency_ms"])
            if not done:
                time.sleep(50e-6)
        span = time.perf_counter() - t0
        loads.append({"offered": load, "offered_per_s": load * rate, "achieved_per_s": n_req / span,
                      "samples": len(lat), "p50_ms": float(np.percentile(lat, 50)),
                      "p99_ms": float(np.percentile(lat, 99))})
    srv.close()
    return {"requests_per_level": n_req, "slots": slots, "saturation_requests_per_s": rate,
            "value": done_k / dt_closed, "unit": "series*lags/s", "loads": loads,
            "p50_ms": loads[1]["p50_ms"], "p99_ms": loads[1]["p99_ms"], "latency_samples": loads[1]["samples"],
            "mix": "50% ACF light curves / 50% OU CCF (n_B = 0.8 n_A), n log-uniform [1e3, 5e6], "
                   "K in {64, 256, 1024}, Gaussian FP32 form or rectangle exact scan, h = 0.5; "
                   "requests drawn from 32 seeded templates; half name device-resident series, "
                   f"half send host arrays and pay their upload ({int(host.sum())} of {n_req})"}

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ncf", choices=["ncf", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-serve", action="store_true",
                    help="skip the serving, bootstrap, regular-grid, Hanning and paper-NUFFT legs")
    ap.add_argument("--batch", type=int, default=B_SERIES, help="series per rank (profiling runs)")
    ap.add_argument("--only", choices=["paper", "hanning", "spectral-k1024", "mixed-spans"], default=None,
                    help="run one side leg alone and print its JSON (profiling runs)")
    args = ap.parse_args()

    from paper_2609_03866_b300 import shard
    rank, world, local = shard.dist_env()
    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import torch
    import torch.distributed as dist
    from paper_2609_03866_b300 import api, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.only == "paper":
        print(json.dumps({"paper_nufft": paper_run(api, local)}))
        return
    if args.only == "hanning":
        print(json.dumps({"hanning": hanning_run(api, local)}))
        return
    if args.only == "spectral-k1024":
        print(json.dumps({"spectral_k1024": spectral_k1024_run(api, local)}))
        return
    if args.only == "mixed-spans":
        print(json.dumps({"per_series_grids": mixed_spans_run(api, local)}))
        return
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    # ---- workload (each rank its own batch: weak scaling) ----
    w = synth.light_curves(B=args.batch, K=K_LAGS, seed=shard.rank_seed(synth.BASE_SEED, rank))
    offs = w.offs
    t = torch.from_numpy(w.t).to(dev)
    x = torch.from_numpy(w.x).to(dev)
    lags = torch.from_numpy(w.lags).to(dev)
    B, K = w.B, K_LAGS
    ctx = api.Context(local)
    stream = torch.cuda.current_stream(dev)
    out_g = {"c": torch.empty(B, K, dtype=torch.float64, device=dev),
             "b": torch.empty(B, K, dtype=torch.float64, device=dev)}
    out_r = {"c": torch.empty(B, K, dtype=torch.float64, device=dev),
             "b": torch.empty(B, K, dtype=torch.float64, device=dev),
             "count": torch.empty(B, K, dtype=torch.int64, device=dev)}
    G_OPT = dict(kernel="gaussian", h=H, path="spectral", precision="fp32")
    R_OPT = dict(kernel="rectangle", h=H)

    # ---- the step: one plan of both estimators (one statistics pass), its launches
    # captured in a CUDA graph; each estimator also as a plan of its own ----
    def capture(fn):
        g = torch.cuda.CUDAGraph()
        cs = torch.cuda.Stream(dev)
        cs.wait_stream(stream)
        l0 = ctx.launches
        with torch.cuda.stream(cs):
            with torch.cuda.graph(g, stream=cs):
                fn(cs)
        torch.cuda.synchronize()
        return g, ctx.launches - l0

    plan_m = api.MultiPlan(offs, t, x, lags, [G_OPT, R_OPT], ctx=ctx, stream=stream)
    plan_g = api.Plan(offs, t, x, lags, **G_OPT, ctx=ctx, stream=stream)
    plan_r = api.Plan(offs, t, x, lags, **R_OPT, ctx=ctx, stream=stream)
    for _ in range(max(args.warmup, 3)):
        plan_m.execute(t, x, outs=[out_g, out_r], stream=stream)
    plan_g.execute(t, x, out=out_g, stream=stream)
    plan_r.execute(t, x, out=out_r, stream=stream)
    torch.cuda.synchronize()
    g_step, graph_launches = capture(lambda cs: plan_m.execute(t, x, outs=[out_g, out_r], stream=cs))
    g_gauss, _ = capture(lambda cs: plan_g.execute(t, x, out=out_g, stream=cs))
    g_rect, _ = capture(lambda cs: plan_r.execute(t, x, out=out_r, stream=cs))
    for _ in range(max(args.warmup, 3)):
        g_step.replay()
    torch.cuda.synchronize()
    plan = ctx.last_plan()
    tuned = ctx.last_tuning()

    # ---- timed region: graph replays of the step ----
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        ev[0].record(stream)
        for s_ in range(args.steps):
            g_step.replay()
            ev[s_ + 1].record(stream)
        torch.cuda.synchronize()
        barrier()
    launches = graph_launches * args.steps
    step_ms = [ev[s_].elapsed_time(ev[s_ + 1]) for s_ in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    total_ms = shard.max_over_ranks(total_ms, device=dev)
    units = 2.0 * B * K * args.steps * world
    value = units / (total_ms / 1e3)
    c32 = out_g["c"].clone()
    counts = out_r["count"].clone()
    rect_c = out_r["c"].clone()
    if plan_m.status() != 0:
        raise RuntimeError("a plan's device guard flagged the benchmark data")

    # ---- each estimator alone (its own plan and graph, its own statistics pass) ----
    def graph_ms(g, reps=3):
        g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            g.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    g_ms, r_ms = graph_ms(g_gauss), graph_ms(g_rect)
    if plan_g.status() != 0 or plan_r.status() != 0:
        raise RuntimeError("a plan's device guard flagged the benchmark data")

    # ---- the same step through one call for both estimators (one statistics pass),
    # with the kernel profiler (shares, roofline) ----
    def step():
        api.corr_batch_multi(offs, t, x, lags, [G_OPT, R_OPT], ctx=ctx, stream=stream, outs=[out_g, out_r])

    step()
    torch.cuda.synchronize()
    ctx.profile(True)
    ctx.profile_reset()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(args.steps):
        step()
    p1.record(stream)
    torch.cuda.synchronize()
    prof = ctx.profile_report()
    ctx.profile(False)
    one_shot_ms = p0.elapsed_time(p1) / args.steps

    # ---- spec comparison: FP32 form vs the plain FP64 GPU path, Gaussian ----
    fp64 = None
    if not args.no_fp64:
        fp64 = fp64_plain_run(api, ctx, stream, w, offs, t, x, lags, out_g, c32, g_ms, world)

    # ---- end to end through the host-buffer C call ----
    e2e = None
    if not args.no_e2e:
        th = torch.from_numpy(w.t).pin_memory()
        xh = torch.from_numpy(w.x).pin_memory()
        lh = torch.from_numpy(w.lags).pin_memory()
        og = {"c": torch.empty(B, K, dtype=torch.float64).pin_memory()}
        orr = {"c": torch.empty(B, K, dtype=torch.float64).pin_memory(),
               "count": torch.empty(B, K, dtype=torch.int64).pin_memory()}

        # both estimators of the step from one upload of the batch (ncf_corr_batch_host_multi)
        hopts = [dict(G_OPT), dict(R_OPT)]

        def hstep():
            api.corr_batch_host_multi(offs, th, xh, lh, hopts, ctx=ctx, stream=stream, outs=[og, orr])

        hstep()
        n_e2e = max(2, min(args.steps, 3))
        barrier()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            hstep()
        torch.cuda.synchronize()
        barrier()
        dt = time.perf_counter() - t0
        h2d = w.t.nbytes + w.x.nbytes + w.lags.nbytes
        d2h = 8 * B * K + 16 * B * K
        e2e = {"value": 2.0 * B * K * n_e2e * world / dt, "unit": "series*lags/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "steps": n_e2e}

    mem = {"context_workspace_high_water_bytes": ctx.device_bytes,
           "plan_bytes": {"both_estimators": plan_m.device_bytes, "gaussian_fp32_form": plan_g.device_bytes,
                          "rectangle_exact_scan": plan_r.device_bytes},
           "workspace_bound_bytes": {
               "gaussian_fp32_form": api.workspace_bytes(int(offs[-1]), B, K, float(max(
                   w.t[offs[b + 1] - 1] - w.t[offs[b]] for b in range(B))), float(np.max(np.abs(w.lags))), **G_OPT)[0],
               "rectangle_exact_scan": api.workspace_bytes(int(offs[-1]), B, K, 0.0, float(np.max(np.abs(w.lags))),
                                                           **R_OPT)[0]},
           "inputs_bytes": int(w.t.nbytes + w.x.nbytes + w.lags.nbytes)}
    plan_m.close()
    plan_g.close()
    plan_r.close()

    serve = None
    if not args.no_serve:
        serve = serve_run(api, local)
    boot = None if args.no_serve else bootstrap_run(api, local)
    regular = None if args.no_serve else regular_run(api, local)
    hanning = None if args.no_serve else hanning_run(api, local)
    paper = None if args.no_serve else paper_run(api, local)
    single = None if args.no_serve else single_acf_run(api, local)
    precision = None if args.no_serve else precision_run(api, local)
    mixed = None if args.no_serve else mixed_spans_run(api, local)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- accuracy on a sample against the FP64 oracle; CPU baseline ----
    series, lag_idx = cpu_sample(w)
    acc = {}
    cpu = None
    if not args.no_cpu:
        rate, secs, res = time_oracle(w, series, lag_idx)
        g_err = max(float(np.max(np.abs(c32[b, lag_idx].cpu().numpy() - res[("gaussian", int(b))]["c"])))
                    for b in series)
        r_err = max(float(np.max(np.abs(rect_c[b, lag_idx].cpu().numpy() - res[("rectangle", int(b))]["c"])))
                    for b in series)
        cnt_ok = all(np.array_equal(counts[b, lag_idx].cpu().numpy(), res[("rectangle", int(b))]["count"])
                     for b in series)
        acc = {"gaussian_fp32_max_abs_err": g_err, "rectangle_max_abs_err": r_err,
               "rectangle_counts_bit_exact": bool(cnt_ok),
               "sample": f"{len(series)} series x {len(lag_idx)} lags vs FP64 oracle (Gaussian window 8h)"}
        cpu = {"value": rate, "unit": "series*lags/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{len(series)} random series x {len(lag_idx)} of 256 lags, both kernels, "
                         f"FP64 windowed scan; {secs:.1f} s"}

    # ---- roofline of the dominant kernel (profiled one-shot steps) ----
    hbm, tc_peak, src = peaks()
    n_pts = int(offs[-1])
    items = n_pts * K  # outer points x lags of the rectangle scan
    dom = max(prof.items(), key=lambda kv: kv[1][1]) if prof else ("none", (1, 1.0))
    name, (nl, ms) = dom
    per_launch_s = ms / nl / 1e3
    share = {k: round(v[1] / sum(u[1] for u in prof.values()), 4) for k, v in prof.items()}
    nf, M = plan["grid"], plan["modes"]
    if name.startswith("rect_scan"):
        # integer ALU: 16 int32 operations per (outer point, lag) item (two
        # 64-bit bound adds, two 64-bit window compares, one 64-bit window
        # difference, one 64x64->128-bit multiply-accumulate), against the
        # measured integer rates for that mix (INT_OPS_PER_CLK_SM)
        ops = 16.0 * items / (nl / args.steps)
        peak_ops = 148 * INT_OPS_PER_CLK_SM * 2032e6
        roof = {"bound": "alu", "achieved": ops / per_launch_s / 1e12, "peak": peak_ops / 1e12,
                "unit": "Tint32op/s", "frac": ops / per_launch_s / peak_ops, "traffic": None,
                "kernel": name, "peak_source": "measured integer rates: IADD3 120, LOP3/SHF/IMAD 60 ops per clock "
                                               "per SM; the item's 8 + 8 ops at 80 per clock, 148 SM x 2.032 GHz"}
    elif name == "spread_kernel":
        byts = (16.0 * n_pts + 8.0 * B * nf) / (nl / args.steps)
        roof = {"bound": "hbm", "achieved": byts / per_launch_s / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": byts / per_launch_s / 1e9 / hbm, "traffic": None, "kernel": name,
                "peak_source": src}
    elif name == "fft_pass_kernel":
        byts = 16.0 * B * nf
        roof = {"bound": "hbm", "achieved": byts / per_launch_s / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": byts / per_launch_s / 1e9 / hbm, "traffic": None, "kernel": name,
                "peak_source": src}
    else:
        byts = 16.0 * n_pts / max(1, nl / args.steps)
        roof = {"bound": "hbm", "achieved": byts / per_launch_s / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": byts / per_launch_s / 1e9 / hbm, "traffic": None, "kernel": name,
                "peak_source": src}
    roof["traffic"] = MEASURED_TRAFFIC.get((name, B))
    roof["share"] = share

    # the memory-side kernels of the FP32 form and the statistics pass against the HBM
    # roofline: algorithmic bytes per step (spreading: t and x in, one complex FP32 cell
    # out per grid cell; shared-memory FFT: the grid in, M complex FP32 spectrum values
    # out per series; global-pass FFT: the grid in and out once per radix-8/4/2 pass;
    # statistics: t and x in) over the kernel's time per step
    def hbm_frac(kname, byts):
        if kname not in prof:
            return None
        per_step_s = prof[kname][1] / 1e3 / args.steps
        gbs = byts / per_step_s / 1e9
        return {"ms_per_step": per_step_s * 1e3, "bytes_per_step": byts, "achieved": gbs, "unit": "GB/s",
                "peak": hbm, "frac": gbs / hbm}

    hbm_kernels = {k: v for k, v in (
        ("spread_kernel", hbm_frac("spread_kernel", 16.0 * n_pts + 8.0 * B * nf)),
        ("fft_spectrum_smem_kernel", hbm_frac("fft_spectrum_smem_kernel", 8.0 * B * nf + 8.0 * B * M)),
        ("fft_pass_kernel", hbm_frac("fft_pass_kernel", 16.0 * B * nf * int(np.ceil(np.log2(nf) / 3)))),
        ("stats_chunks_kernel", hbm_frac("stats_chunks_kernel", 16.0 * n_pts))) if v is not None}

    line = {
        "metric": METRIC, "value": value, "unit": "series*lags/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": total_ms / args.steps,
        "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "B": B, "K": K, "points": n_pts, "h": H,
                   "grid": nf, "modes": M, "period_d": plan["period"], "graph": True,
                   "tuned": {"rect_scan": ["lags on lanes, runs of 16", "lags on lanes, runs of 32",
                                           "lags on lanes, runs of 64",
                                           "outer points on lanes"][tuned["rect_variant"]]
                             if tuned["rect_variant"] >= 0 else None,
                             "fft": {0: "shared-memory FFT fused with the spectrum", 1: "global Stockham passes"}
                             .get(tuned["fft_variant"]),
                             "contraction": {0: "tensor cores (tcgen05, split TF32)", 1: "FP32 pipe"}
                             .get(tuned["contract_variant"]),
                             "spreading": {0: "CTAs of 4096 points, FP32 tile sums",
                                           1: "CTAs of 2048 points, FP32 tile sums",
                                           2: "CTAs of 4096 points, fixed-point tile sums",
                                           3: "CTAs of 2048 points, fixed-point tile sums"}
                             .get(tuned["spread_variant"])},
                   "l2": f"inputs larger than L2 ({(w.t.nbytes + w.x.nbytes) / 1e9:.2f} GB per step)"},
        "per_estimator": {
            "note": "each estimator alone: its own plan and graph, statistics pass included",
            "gaussian_fp32_form": {"ms": g_ms, "value": B * K * world / (g_ms / 1e3), "unit": "series*lags/s"},
            "rectangle_exact_scan": {"ms": r_ms, "value": B * K * world / (r_ms / 1e3), "unit": "series*lags/s"},
            "one_call_ms_per_step": one_shot_ms,
            "one_call": "ncf_corr_batch_multi: both estimators on one statistics pass, host analysis per call"},
        "gpu_launches": int(launches),
        "device_memory": mem,
        "clocks": clk.summary(),
        "roofline": roof,
        "hbm_kernels": hbm_kernels,
        "e2e": e2e,
        "north_star": fp64,
        "paper_timings": {
            "hardware": "MacBook Pro 2020, 2 GHz quad-core Intel Core i5, 16 GB LPDDR4X (the paper's benchmark machine)",
            "note": "context only: other hardware, single series, K = 366; not the target",
            "nufft_gaussian_s_per_point_per_lag": 1.13e-5 / 366, "nufft_rectangle_s_per_point_per_lag": 3.77e-6 / 366,
            "realspace_gaussian_s_per_point_per_lag": 1.80e-5 / 366,
            "realspace_rectangle_s_per_point_per_lag": 1.34e-6 / 366,
            "regular_fft_n256000": {"gaussian_s": 0.07, "rectangle_s": 0.04},
            "this_run_s_per_point_per_lag": {
                "gaussian_fp32_form": g_ms / 1e3 / (n_pts * K),
                "rectangle_exact_scan": share.get("rect_scan_pt_kernel", share.get("rect_scan_kernel", 0.0))
                * (total_ms / args.steps) / 1e3 / (n_pts * K)}},
        "serving": serve,
        "bootstrap": boot,
        "regular_fft": regular,
        "hanning": hanning,
        "paper_nufft": paper,
        "single_acf_fp64": single,
        "precision_mjd_1e7": precision,
        "per_series_grids": mixed,
        "accuracy": acc,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
