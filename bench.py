"""Benchmark of the wave propagators on one GB300.

Workload (default): the 3D isotropic elastic velocity-stress system, 256^3
physical grid at 10 m + 20-cell absorbing layer (296^3 computational
points), space order 8, 1000 time steps, smooth random model (vp 1.5-4.5
km/s, vs = vp/1.73, rho 1.0-2.5 g/cc, 200 m correlation length), explosive
10 Hz Ricker source at the centre, 64 x 64 receivers at the surface.
One benchmark step = one forward modelling + one adjoint modelling of that
shot (2 x 1000 propagator time steps).  Metric: grid-point updates per
second (Gpts/s, computational grid).

Reported beside it: the roofline of the dominant kernel (algorithmic bytes
per launch / CUDA-event launch time vs the measured HBM copy bandwidth),
the FP64 CPU oracle on a bounded sample of the same workload, the same
metric end to end through the C ABI with host buffers, and SM clocks sampled
during the timed region.

--impl reference times the FP64 CPU oracle instead (bounded sample per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

HBM_FALLBACK_GBS = 6800.0
# algorithmic bytes per point update of one fused time step (each state
# array read and written once, each parameter array read once):
#   elastic: 9 state reads + 9 writes + 3 parameters (b, lambda, mu) = 84 B
#   TTI:     4 state reads + 2 writes + 5 parameters                  = 44 B
#   acoustic: 2 state reads + 1 write + m                             = 16 B
ALG_BYTES = {"elastic": 84.0, "tti": 44.0, "acoustic": 16.0}
# DRAM bytes per point of one elastic step (velocity + stress pass) measured
# by ncu (dram__bytes_read.sum + dram__bytes_write.sum) on the benchmark's own
# 296^3 grid at the autotuned 8-row tile (118.1 at 16 rows;
# profiles/elastic_bench_launch_list_296cube_so8.md)
TRAFFIC_B_PER_PT = {"elastic": 118.7}
# algorithmic FP32 operations per point update, counted from the kernels'
# arithmetic (FMA = 2): elastic so 8 (velocity + stress pass), TTI so 12
# (rotation + update pass), acoustic so 12 (7 per stencil radius + 15)
FLOP_PER_PT = {"elastic": 263.0, "tti": 250.0, "tti_sp": 510.0, "acoustic": 57.0}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


class Clocks:
    """nvidia-smi sampling (every 200 ms) while the context is open.  Samples
    are stamped on arrival; ``region()`` brackets a timed region, and the
    summary covers only the samples inside the regions (all samples if none
    was marked)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu=0):
        self.gpu = gpu
        self.proc = None
        self.lines = []
        self.regions = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    class _Region:
        def __init__(self, clk):
            self.clk = clk

        def __enter__(self):
            self.t0 = time.perf_counter()
            return self

        def __exit__(self, *a):
            # the sample describing the last 200 ms arrives up to ~0.3 s later
            self.clk.regions.append((self.t0, time.perf_counter() + 0.3))

    def region(self):
        return Clocks._Region(self)

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for t, ln in self.lines:
            if self.regions and not any(a <= t <= b for a, b in self.regions):
                continue
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


_CLK = None


def timed_region():
    """Bracket a timed region of a secondary measurement for the clock record
    (a no-op context when no sampler runs)."""
    if _CLK is None:
        import contextlib
        return contextlib.nullcontext()
    return _CLK.region()


def elastic_workload(small=False):
    if small:
        # profiling case: 160^3 + 20-cell layer = 200^3 points, 32 MB per field
        # (working set ~0.7 GB > L2), 100 steps
        return synth.elastic_random(n=160, nbl=20, so=8, nt=100)
    return synth.elastic_random()      # 256^3 @ 10 m + 20, so 8, 1000 steps


def cpu_baseline(prob, budget_s=20.0):
    """FP64 oracle on the host cores: forward + adjoint time steps on the full
    computational grid of the workload from a seeded state, as many steps as
    fit the budget (at least one of each)."""
    import oracle
    o = oracle.Problem(prob)
    N = o.N
    st = np.random.default_rng(3).standard_normal((9,) + o.shape, dtype=np.float32)
    steps = 0
    t0 = time.perf_counter()
    while True:
        o.el_step(st, adjoint=(steps % 2 == 1), nsteps=1)
        steps += 1
        if time.perf_counter() - t0 > budget_s or steps >= 64:
            break
    dt = time.perf_counter() - t0
    return {"value": N * steps / dt / 1e9, "unit": "Gpts/s", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"{steps} elastic time steps (alternating forward/adjoint) of the "
                      f"{o.shape[0]}x{o.shape[1]}x{o.shape[2]} grid, FP64, OpenMP"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    prob = elastic_workload(args.small)
    import oracle
    o = oracle.Problem(prob)
    st = np.random.default_rng(3).standard_normal((9,) + o.shape, dtype=np.float32)
    per_step = 2   # bounded sample: one forward + one adjoint time step per bench step
    for _ in range(args.warmup):
        o.el_step(st, nsteps=1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.el_step(st, nsteps=1)
        o.el_step(st, adjoint=True, nsteps=1)
    dt = time.perf_counter() - t0
    v = o.N * per_step * args.steps / dt / 1e9
    line = {"impl": "reference", "metric": "elastic propagator grid-point updates per second",
            "value": v, "unit": "Gpts/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": prob.name, "grid": list(o.shape), "space_order": prob.so},
            "cpu_baseline": {"value": v, "unit": "Gpts/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{per_step} time steps per bench step (1 forward + 1 adjoint) "
                                       "of the full grid, FP64"},
            "e2e": {"value": v, "unit": "Gpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def aggregate(ms, units_per_rank, dist=None, device=None):
    """Whole-job throughput of independent replicas: every rank processes
    its own units (shots); time = max over ranks; value = all units / time.
    Returns (max_ms, units_per_second)."""
    world = 1
    if dist is not None and dist.is_initialized():
        import torch
        world = dist.get_world_size()
        t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, units_per_rank * world / (ms / 1e3)


def tti_throughput(wp, torch, dev, steps=40, nx=800, ny=800, nz=400, nbl=40, h=12.5, so=12, tti_operator=0):
    """TTI so-12 forward and adjoint step rates on the industry-scale grid
    (880 x 880 x 480 computational points) from a seeded random state; the
    model is uniform random within the workload's ranges (content does not
    change the work)."""
    rng = np.random.default_rng(7)
    f = lambda lo, hi: rng.uniform(lo, hi, (nx, ny, nz)).astype(np.float32)
    eps = f(0.0, 0.3)
    model = [f(1.5, 4.5), eps, (eps * f(0.0, 0.5)).astype(np.float32), f(0.0, 0.7), f(0.0, 1.57)]
    vmax = 4.5 * np.sqrt(1.6)
    dt = synth.cfl_dt(h, vmax)
    prop = wp.Propagator(wp.PROP_TTI, (nx, ny, nz), nbl, h, so, 10, model, dt=dt,
                         stream=torch.cuda.current_stream(dev).cuda_stream, tti_operator=tti_operator)
    del model
    N = int(np.prod(prop.grid))
    tile = {"z": 32, "y": prop.tile_rows, "x": prop.tile_planes}
    st = [torch.randn(prop.grid, device=dev) for _ in range(4)]
    prop.set_state(st)
    del st
    out = {}
    for adj, key, kid in ((False, "tti_forward", wp.K_TTI_FWD), (True, "tti_adjoint", wp.K_TTI_ADJ)):
        prop.step(5, adjoint=adj)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with timed_region():
            e0.record()
            prop.step(steps, adjoint=adj)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            prop.profile(True)
            prop.step(10, adjoint=adj)
            kms, kn = prop.kernel_stats(kid)
            prop.profile(False)
        t = kms / max(kn, 1) / 1e3
        hbm, src_peak = peaks()
        ach = ALG_BYTES["tti"] * N / t / 1e9
        out[key] = {"gpts_per_s": N / (ms / 1e3) / 1e9, "ms_per_step": ms,
                    "kernel_ms_per_step": t * 1e3,
                    "alg_gbs": ach,
                    "alg_tflops": FLOP_PER_PT["tti_sp" if tti_operator else "tti"] * N / t / 1e12,
                    "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                                 "frac": ach / hbm, "peak_source": src_peak,
                                 "alg_bytes_per_pt": ALG_BYTES["tti"], "launch_ms": t * 1e3}}
    prop.close()
    out["grid"] = list(prop.grid)
    out["tile"] = tile
    out["space_order"] = so
    out["hbm_peak_gbs"] = peaks()[0]
    out["fp32_peak_tflops"] = wp.fp32_peak()
    return out


def acoustic_throughput(wp, torch, dev, steps=40, nx=800, ny=800, nz=400, nbl=40, h=12.5, so=12):
    """Isotropic acoustic so-12 step rate on the industry-scale grid
    (880 x 880 x 480 computational points) from a seeded random state, and
    the transposed step with imaging (the gradient's inner step); the model
    is uniform random in [1.5, 4.5] km/s (content does not change the work)."""
    rng = np.random.default_rng(8)
    vp = rng.uniform(1.5, 4.5, (nx, ny, nz)).astype(np.float32)
    dt = synth.cfl_dt(h, 4.5)
    stream = torch.cuda.current_stream(dev).cuda_stream
    prop = wp.Propagator(wp.PROP_ACOUSTIC, (nx, ny, nz), nbl, h, so, 10, [vp], dt=dt, stream=stream)
    del vp
    N = int(np.prod(prop.grid))
    prop.set_state([torch.randn(prop.grid, device=dev) for _ in range(2)])
    out = {}
    prop.step(5)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with timed_region():
        e0.record()
        prop.step(steps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        prop.profile(True)
        prop.step(10)
        kms, kn = prop.kernel_stats(wp.K_AC_STEP)
        prop.profile(False)
    t = kms / max(kn, 1) / 1e3
    out["acoustic_forward"] = {"gpts_per_s": N / (ms / 1e3) / 1e9, "ms_per_step": ms,
                               "kernel_ms_per_step": t * 1e3,
                               "alg_gbs": ALG_BYTES["acoustic"] * N / t / 1e9,
                               "alg_tflops": FLOP_PER_PT["acoustic"] * N / t / 1e12}
    prop.close()
    out["grid"] = list(prop.grid)
    out["space_order"] = so
    out["hbm_peak_gbs"] = peaks()[0]
    return out


def elastic2d_throughput(wp, torch, dev, small=False):
    """2D elastic forward modelling (so 8) on the marine model standing in for
    the elastic Marmousi-II of the 2D example: 1701 x 701 cells at 5 m +
    40-cell layer (x, z), water 450 m deep, 15 Hz explosive source 10 m
    deep, pressure receivers every 10 m at 5 m depth.  Whole-run time and
    the step kernels' time (velocity + stress pass)."""
    kw = dict(nx=401, nz=201, nt=400) if small else dict(nt=2000)
    p = synth.marine_elastic_2d(**kw)
    stream = torch.cuda.current_stream(dev).cuda_stream
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    prop = wp.Propagator.from_problem(p, stream=stream)
    w, s_, r = to(p.wavelet), to(p.src), to(p.rec)
    prop.forward(w, s_, r)                                  # warm-up
    torch.cuda.synchronize()
    with timed_region():
        t0 = time.perf_counter()
        prop.forward(w, s_, r)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        prop.profile(True)
        prop.forward(w, s_, r)
        kms, kn = prop.kernel_stats(wp.K_EL_FWD)
        prop.profile(False)
    N = int(np.prod(prop.grid))
    prop.close()
    t_step = kms / max(kn, 1) / 1e3
    # algorithmic bytes: 5 state reads + 5 writes + b, lambda, mu = 52 B/pt
    return {"grid": list(prop.grid), "nt": p.nt, "seconds": sec,
            "gpts_per_s": N * p.nt / sec / 1e9, "kernel_ms_per_step": t_step * 1e3,
            "kernel_gpts_per_s": N / t_step / 1e9, "alg_gbs": 52.0 * N / t_step / 1e9}


def rtm_shots_per_hour(wp, torch, dev, nshots, nt, small=False):
    """Reverse-time migration over many shots (acoustic so 12, FP32
    checkpoints): per-shot images (dJ/dm against the true model's data, in
    the migration velocity) from one prop_gradient_batch call, stacked on the
    device into the global image at each window's offset."""
    kw = dict(size_range=(60, 120), nz=80, global_cells=(300, 300, 100)) if small else {}
    shots = synth.acoustic_rtm_shots(nshots, nt, **kw)
    stream = torch.cuda.current_stream(dev).cuda_stream
    to = lambda a: torch.from_numpy(a).to(dev)
    props, wav, src, rec, obs = [], [], [], [], []
    gx, gy, _ = kw.get("global_cells", (1000, 1000, 500))
    nz = shots[0][1].nz
    for true, p0, _ in shots:
        pt = wp.Propagator.from_problem(true, stream=stream)
        w, s_, r = to(true.wavelet), to(true.src), to(true.rec)
        obs.append(pt.forward(w, s_, r))
        pt.close()
        props.append(wp.Propagator.from_problem(p0, snap_mode=wp.SNAP_CKPT_FP32, stream=stream))
        wav.append(w); src.append(s_); rec.append(r)
    stack = torch.zeros((gx, gy, nz), dtype=torch.float32, device=dev)
    props[0].gradient(wav[0], src[0], rec[0], obs[0])        # warm-up
    torch.cuda.synchronize()
    with timed_region():
        t0 = time.perf_counter()
        grads, _ = wp.gradient_batch(props, wav, src, rec, obs)
        for p, g, (_, _, off) in zip(props, grads, shots):
            p.stack_image(g, stack, off)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
    npts = sum(int(np.prod(p.grid)) for p in props)
    for p in props:
        p.close()
    return {"shots": nshots, "nt": nt, "storage": "fp32 checkpoints", "points_total": npts,
            "seconds": sec, "shots_per_hour": 3600.0 * nshots / sec,
            "stack_dims": list(stack.shape), "stack_l2": float(torch.linalg.norm(stack))}


def gradient_shots_per_hour(wp, torch, dev, nt, modes, small=False):
    """TTI FWI gradient (so 12) shots/hour on the 400x400x300 + 40 workload
    for several wavefield-storage modes at equal nt."""
    if small:
        true, p0 = synth.tti_gradient_problem(nx=120, ny=120, nz=100, nt=nt)
    else:
        true, p0 = synth.tti_gradient_problem(nt=nt)
    stream = torch.cuda.current_stream(dev).cuda_stream
    ptrue = wp.Propagator.from_problem(true, stream=stream)
    d_obs = ptrue.forward(torch.from_numpy(true.wavelet).to(dev), torch.from_numpy(true.src).to(dev),
                          torch.from_numpy(true.rec).to(dev))
    ptrue.close()
    wav = torch.from_numpy(p0.wavelet).to(dev)
    src = torch.from_numpy(p0.src).to(dev)
    rec = torch.from_numpy(p0.rec).to(dev)
    res = {}
    ref = None
    runs = [(str(m), m, None) for m in modes]
    if 1 in modes:      # FP32 checkpoints without the full-storage tail
        runs.append(("1_no_tail", 1, "0"))
    for key, mode, tail in runs:
        if tail is not None:
            os.environ["WAVEPROP_CKPT_TAIL"] = tail
        prop = wp.Propagator.from_problem(p0, snap_mode=mode, stream=stream)
        try:
            g, J = prop.gradient(wav, src, rec, d_obs)          # warm-up + result
            torch.cuda.synchronize()
            with timed_region():
                t0 = time.perf_counter()
                g, J = prop.gradient(wav, src, rec, d_obs)
                torch.cuda.synchronize()
                s = time.perf_counter() - t0
            gd = g.double()
            if ref is None:
                ref = gd
            err = float(torch.linalg.norm(gd - ref) / torch.linalg.norm(ref))
            res[key] = {"seconds": s, "shots_per_hour": 3600.0 / s, "misfit": J,
                        "rel_l2_vs_first_mode": err}
        except wp.PropError as e:
            res[key] = {"error": str(e)}
        prop.close()
        if tail is not None:
            del os.environ["WAVEPROP_CKPT_TAIL"]
    # gradient w.r.t. (m, eps, delta, theta, phi), full FP32 storage
    prop = wp.Propagator.from_problem(p0, snap_mode=modes[0], stream=stream)
    try:
        prop.gradient_aniso(wav, src, rec, d_obs)
        torch.cuda.synchronize()
        with timed_region():
            t0 = time.perf_counter()
            _, J = prop.gradient_aniso(wav, src, rec, d_obs)
            torch.cuda.synchronize()
            s = time.perf_counter() - t0
        aniso = {"mode": str(modes[0]), "seconds": s, "shots_per_hour": 3600.0 / s, "misfit": J}
    except wp.PropError as e:
        aniso = {"error": str(e)}
    prop.close()
    return {"nt": nt, "grid": [p0.nx + 2 * p0.nbl, p0.ny + 2 * p0.nbl, p0.nz + 2 * p0.nbl],
            "modes": res, "aniso_m_eps_delta_theta_phi": aniso}


def elastic_gradient_shots_per_hour(wp, torch, dev, nt, modes, small=False):
    """Elastic FWI gradient (so 8, dJ/d(lambda, mu, b)) shots/hour on the
    benchmark grid (256^3 + 20-cell layer) for several storage modes at equal
    nt; starting model: true model with a smoothed vp (vs = vp/1.73 kept)."""
    n = 96 if small else 256
    true = synth.elastic_random(n=n, nt=nt)
    true.src[:, 2] = 5 * true.h        # shallow source: signal at the receivers within nt
    start = synth.smooth_model(true.model, 100.0 / true.h, keys=("vp", "vs"))
    p0 = synth.Problem(**{**true.__dict__, "model": start})
    stream = torch.cuda.current_stream(dev).cuda_stream
    to = lambda a: torch.from_numpy(a).to(dev)
    ptrue = wp.Propagator.from_problem(true, stream=stream)
    d_obs = ptrue.forward(to(true.wavelet), to(true.src), to(true.rec))
    ptrue.close()
    wav, src, rec = to(p0.wavelet), to(p0.src), to(p0.rec)
    res, ref = {}, None
    for mode in modes:
        prop = wp.Propagator.from_problem(p0, snap_mode=mode, stream=stream)
        try:
            g, J = prop.gradient(wav, src, rec, d_obs)          # warm-up + result
            torch.cuda.synchronize()
            with timed_region():
                t0 = time.perf_counter()
                g, J = prop.gradient(wav, src, rec, d_obs)
                torch.cuda.synchronize()
                sec = time.perf_counter() - t0
            gd = g.double()
            if ref is None:
                ref = gd
            err = [float(torch.linalg.norm(gd[c] - ref[c]) / torch.linalg.norm(ref[c])) for c in range(3)]
            res[str(mode)] = {"seconds": sec, "shots_per_hour": 3600.0 / sec, "misfit": J,
                              "rel_l2_vs_first_mode": err}
        except wp.PropError as e:
            res[str(mode)] = {"error": str(e)}
        prop.close()
    return {"nt": nt, "grid": [n + 2 * p0.nbl] * 3, "modes": res}


def gradient_small(wp, torch, dev):
    """Profiling case of the gradient paths: one elastic gradient (so 8,
    160^3 + 20-cell layer = 200^3, 60 steps, full storage, shallow source)
    and one TTI gradient (so 12, 240x240x200 + 40-cell layer = 320x320x280,
    40 steps, full storage), observed data 1.1 x the predicted traces."""
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    out = {}
    for key, p in (("elastic", synth.elastic_random(n=160, nt=60)),
                   ("tti", synth.tti_layered(nx=240, ny=240, nz=200, nt=40))):
        if key == "elastic":
            p.src[:, 2] = 5 * p.h
        prop = wp.Propagator.from_problem(p, stream=stream)
        w, s_, r = to(p.wavelet), to(p.src), to(p.rec)
        d = prop.forward(w, s_, r) * 1.1
        torch.cuda.synchronize()
        with timed_region():
            t0 = time.perf_counter()
            _, J = prop.gradient(w, s_, r, d)
            torch.cuda.synchronize()
        out[key] = {"grid": list(prop.grid), "nt": p.nt, "seconds": time.perf_counter() - t0, "misfit": J}
        prop.close()
    return out


def tile_heights(wp, torch, dev, small=False):
    """Step time of the TMA-fed passes at each tile height (8, 16, 32 rows of
    y; the x-extent tuned for each) and the autotuner's own choice, on the
    benchmark grids and on a small window: elastic so 8 at 296^3 and
    100^3, TTI so 12 at 880x880x480 and 100^3 (computational points),
    random models and states (content does not change the work)."""
    rng = np.random.default_rng(11)
    cases = [("elastic", 256, 256, 256, 20, 8, 10.0), ("elastic", 60, 60, 60, 20, 8, 10.0),
             ("tti", 800, 800, 400, 40, 12, 12.5), ("tti", 60, 60, 60, 20, 12, 12.5)]
    if small:
        cases = [c[:1] + (60, 60, 60) + c[4:] for c in cases]
    stream = torch.cuda.current_stream(dev).cuda_stream
    out = []
    for kind, nx, ny, nz, nbl, so, h in cases:
        f = lambda lo, hi: rng.uniform(lo, hi, (nx, ny, nz)).astype(np.float32)
        if kind == "elastic":
            vp = f(1.5, 4.5)
            model, K, vmax = [vp, (vp / 1.73).astype(np.float32), f(1.0, 2.5)], wp.PROP_ELASTIC, 4.5
        else:
            eps = f(0.0, 0.3)
            model = [f(1.5, 4.5), eps, (eps * f(0.0, 0.5)).astype(np.float32), f(0.0, 0.7), f(0.0, 1.57)]
            K, vmax = wp.PROP_TTI, 4.5 * np.sqrt(1.6)
        dt = synth.cfl_dt(h, vmax)
        row = {"kind": kind, "so": so}
        for ty in ("8", "16", "32", "auto"):
            if ty == "auto":
                os.environ.pop("WAVEPROP_TILE_Y", None)
            else:
                os.environ["WAVEPROP_TILE_Y"] = ty
            prop = wp.Propagator(K, (nx, ny, nz), nbl, h, so, 10, model, dt=dt, stream=stream)
            row["grid"] = list(prop.grid)
            nf = 9 if kind == "elastic" else 4
            prop.set_state([torch.randn(prop.grid, device=dev) for _ in range(nf)])
            steps = 10 if nx > 100 else 200
            prop.step(3)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with timed_region():
                e0.record()
                prop.step(steps)
                e1.record()
                torch.cuda.synchronize()
            row[ty] = {"rows": prop.tile_rows, "planes": prop.tile_planes,
                       "ms_per_step": e0.elapsed_time(e1) / steps}
            prop.close()
        os.environ.pop("WAVEPROP_TILE_Y", None)
        del model
        out.append(row)
    return out


def gradient_aniso_cost(wp, torch, dev, small=False):
    """Cost of the TTI gradient w.r.t. (m, eps, delta, theta, phi) against
    the m-only gradient, for the centred (0) and the staggered-pair (1)
    operators: so 12, 240x240x200 + 40-cell layer (320x320x280 points), 60
    steps, full FP32 storage (small: 80x80x60 + 20, 30 steps)."""
    kw = dict(nx=80, ny=80, nz=60, nbl=20, nt=30) if small else dict(nx=240, ny=240, nz=200, nt=60)
    p = synth.tti_layered(**kw)
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    w, s_, r = to(p.wavelet), to(p.src), to(p.rec)
    out = {"grid": [p.nx + 2 * p.nbl, p.ny + 2 * p.nbl, p.nz + 2 * p.nbl], "nt": p.nt}
    for op in (0, 1):
        prop = wp.Propagator.from_problem(p, stream=stream, tti_operator=op)
        d = prop.forward(w, s_, r) * 1.1
        prop.gradient(w, s_, r, d)                      # warm-up
        prop.gradient_aniso(w, s_, r, d)
        torch.cuda.synchronize()
        res = {}
        for key, fn in (("m", prop.gradient), ("m_eps_delta_theta_phi", prop.gradient_aniso)):
            with timed_region():
                t0 = time.perf_counter()
                fn(w, s_, r, d)
                torch.cuda.synchronize()
                res[key] = time.perf_counter() - t0
        res["ratio"] = res["m_eps_delta_theta_phi"] / res["m"]
        out[f"operator{op}"] = res
        prop.close()
    return out


def batch_shots_per_hour(wp, torch, dev, nshots, nt, small=False, kind="tti", windows=None):
    """Batched gradients (TTI so 12 or elastic so 8, BF16 checkpoints): shots
    on windows of one large model with nx, ny ~ U[200, 600], nz = 300 (+
    40-cell layer); shots/hour of one prop_gradient call after another
    against one prop_gradient_batch call over the same shots (results
    compared bitwise)."""
    kw = dict(size_range=(60, 120), nz=80) if small else {}
    if windows:
        kw.update(size_range=windows[:2], nz=windows[2])
    shots = (synth.tti_batch_shots if kind == "tti" else synth.elastic_batch_shots)(nshots, nt, **kw)
    stream = torch.cuda.current_stream(dev).cuda_stream
    to = lambda a: torch.from_numpy(a).to(dev)
    props, wav, src, rec, obs = [], [], [], [], []
    npts = 0
    for true, p0 in shots:
        pt = wp.Propagator.from_problem(true, stream=stream)
        w, s_, r = to(true.wavelet), to(true.src), to(true.rec)
        obs.append(pt.forward(w, s_, r))
        pt.close()
        props.append(wp.Propagator.from_problem(p0, snap_mode=wp.SNAP_CKPT_BF16, stream=stream))
        props[-1].trim()                 # idle handles hold only their model
        wav.append(w); src.append(s_); rec.append(r)
        npts += int(np.prod(props[-1].grid))
    torch.cuda.synchronize()
    # warm-up (tensor maps, autotuned tiles, allocator) on the first shot
    props[0].gradient(wav[0], src[0], rec[0], obs[0])
    torch.cuda.synchronize()
    props[0].trim()
    with timed_region():
        t0 = time.perf_counter()
        seq = []
        for i, p in enumerate(props):
            seq.append(p.gradient(wav[i], src[i], rec[i], obs[i]))
            p.trim()                         # as the batch does after each shot
        torch.cuda.synchronize()
        t_seq = time.perf_counter() - t0
    with timed_region():
        t0 = time.perf_counter()
        grads, J = wp.gradient_batch(props, wav, src, rec, obs)
        torch.cuda.synchronize()
        t_bat = time.perf_counter() - t0
    shared, alone = wp.batch_stats()
    # the same waves from one host thread per shot meeting at every step
    # (shared launches without the lockstep driver), then with every shot on
    # its own launches
    os.environ["WAVEPROP_LOCKSTEP"] = "0"
    with timed_region():
        t0 = time.perf_counter()
        grads3, _ = wp.gradient_batch(props, wav, src, rec, obs)
        torch.cuda.synchronize()
        t_rdv = time.perf_counter() - t0
    shared_rdv, alone_rdv = wp.batch_stats()
    del os.environ["WAVEPROP_LOCKSTEP"]
    os.environ["WAVEPROP_BATCH_LAUNCH"] = "0"
    with timed_region():
        t0 = time.perf_counter()
        grads2, _ = wp.gradient_batch(props, wav, src, rec, obs)
        torch.cuda.synchronize()
        t_own = time.perf_counter() - t0
    del os.environ["WAVEPROP_BATCH_LAUNCH"]
    same_own = all(bool(torch.equal(g, s_)) and bool(torch.equal(g, s3))
                   for g, s_, s3 in zip(grads, grads2, grads3))
    same = all(bool(torch.equal(g, s[0])) for g, s in zip(grads, seq))
    waves = wp.plan_waves([p.gradient_bytes(r.shape[0]) for p, r in zip(props, rec)],
                          int(torch.cuda.mem_get_info(dev)[0] * 0.9))[1]
    for p in props:
        p.close()
    return {"kind": kind, "shots": nshots, "nt": nt, "storage": "bf16 checkpoints",
            "windows": [s[1].name for s in shots], "points_total": npts,
            "sequential": {"seconds": t_seq, "shots_per_hour": 3600.0 * nshots / t_seq},
            "batched": {"seconds": t_bat, "shots_per_hour": 3600.0 * nshots / t_bat,
                        "waves": waves, "shared_launch_rounds": shared, "unshared_rounds": alone,
                        "driver": "lockstep with graph-replayed segments for qualifying waves of windows up to "
                                  "16 M points, else one host thread per shot meeting at every step"},
            "batched_rendezvous": {"seconds": t_rdv, "shots_per_hour": 3600.0 * nshots / t_rdv,
                                   "shared_launch_rounds": shared_rdv, "unshared_rounds": alone_rdv},
            "batched_own_launches": {"seconds": t_own, "shots_per_hour": 3600.0 * nshots / t_own},
            "bitwise_equal": same and same_own}


def oracle_tti_industry(steps=3, nx=800, ny=800, nz=400, nbl=40, h=12.5, so=12):
    """The FP64 oracle on the industry-scale TTI grid (880 x 880 x 480, so
    12): a few source-free steps from a seeded random state with a uniform
    random model (content does not change the work), timed and reported per
    step (the full 3000-step run is that time x 3000; the oracle holds about
    25 arrays of 371.7 M doubles, 74 GB of host memory)."""
    import oracle
    rng = np.random.default_rng(7)
    f = lambda lo, hi: rng.uniform(lo, hi, (nx, ny, nz)).astype(np.float32)
    eps = f(0.0, 0.3)
    model = {"vp": f(1.5, 4.5), "eps": eps, "delta": (eps * f(0.0, 0.5)).astype(np.float32),
             "theta": f(0.0, 0.7), "phi": f(0.0, 1.57)}
    dt = synth.cfl_dt(h, 4.5 * np.sqrt(1.6))
    z = np.zeros((1, 3), np.float32)
    p = synth.Problem(synth.TTI, nx, ny, nz, nbl, h, so, 10, dt, model, z, np.zeros((1, 10), np.float32), z)
    o = oracle.Problem(p)
    del model, eps
    st = [rng.standard_normal(o.shape, dtype=np.float32) for _ in range(4)]
    t0 = time.perf_counter()
    o.tti_run_d(*st, steps)
    sec = time.perf_counter() - t0
    N = o.N
    return {"grid": list(o.shape), "space_order": so, "steps_timed": steps, "seconds_per_step": sec / steps,
            "gpts_per_s": N * steps / sec / 1e9, "cores": os.cpu_count(),
            "full_run_estimate_hours": sec / steps * 3000 / 3600.0}


def forward_batch_shots_per_hour(wp, torch, dev, nshots, nt, windows=None, kind="tti"):
    """Forward modelling (TTI so 12 or elastic so 8) of many shots on
    windows of one large model: one prop_forward after another against one
    prop_forward_batch (lockstep, one launch per pass and step for every
    shot, two steps replayed from a CUDA graph); traces compared bitwise."""
    kw = {}
    if windows:
        kw.update(size_range=windows[:2], nz=windows[2])
    shots = (synth.tti_batch_shots if kind == "tti" else synth.elastic_batch_shots)(nshots, nt, **kw)
    stream = torch.cuda.current_stream(dev).cuda_stream
    to = lambda a: torch.from_numpy(a).to(dev)
    props, wav, src, rec = [], [], [], []
    npts = 0
    for true, _ in shots:
        props.append(wp.Propagator.from_problem(true, stream=stream))
        wav.append(to(true.wavelet)); src.append(to(true.src)); rec.append(to(true.rec))
        npts += int(np.prod(props[-1].grid))
    props[0].forward(wav[0], src[0], rec[0])                   # warm-up
    wp.forward_batch(props[:2], wav[:2], src[:2], rec[:2])
    torch.cuda.synchronize()
    with timed_region():
        t0 = time.perf_counter()
        seq = [p.forward(w, s_, r) for p, w, s_, r in zip(props, wav, src, rec)]
        torch.cuda.synchronize()
        t_seq = time.perf_counter() - t0
    with timed_region():
        t0 = time.perf_counter()
        bat = wp.forward_batch(props, wav, src, rec)
        torch.cuda.synchronize()
        t_bat = time.perf_counter() - t0
    # lockstep whatever the window size (the call above takes it only for
    # windows up to 16 M points)
    os.environ["WAVEPROP_LOCKSTEP"] = "1"
    with timed_region():
        t0 = time.perf_counter()
        bat2 = wp.forward_batch(props, wav, src, rec)
        torch.cuda.synchronize()
        t_lock = time.perf_counter() - t0
    del os.environ["WAVEPROP_LOCKSTEP"]
    same = all(bool(torch.equal(a, b)) and bool(torch.equal(a, c)) for a, b, c in zip(seq, bat, bat2))
    for p in props:
        p.close()
    return {"kind": kind, "shots": nshots, "nt": nt, "points_total": npts,
            "one_call_per_shot": {"seconds": t_seq, "shots_per_hour": 3600.0 * nshots / t_seq,
                                  "gpts_per_s": npts * nt / t_seq / 1e9},
            "forward_batch": {"seconds": t_bat, "shots_per_hour": 3600.0 * nshots / t_bat,
                              "gpts_per_s": npts * nt / t_bat / 1e9},
            "forward_batch_lockstep_forced": {"seconds": t_lock, "shots_per_hour": 3600.0 * nshots / t_lock,
                                              "gpts_per_s": npts * nt / t_lock / 1e9},
            "bitwise_equal": same}


def run_extras(wp, torch, dev, args, extras):
    """Secondary measurements (``--extra``); each timed region is marked for
    the clock record."""
    out = {}

    def _clocked(out, key, fn):
        if _CLK is not None:
            _CLK.regions = []
        out[key] = fn()
        if _CLK is not None and isinstance(out[key], dict):
            out[key]["clocks"] = _CLK.summary()
    if "tti" in extras:
        if args.small:      # profiling case: 240x240x200 + 40 (320x320x280 points)
            _clocked(out, "tti", lambda: tti_throughput(wp, torch, dev, steps=10, nx=240, ny=240, nz=200))
        else:
            _clocked(out, "tti", lambda: tti_throughput(wp, torch, dev))
    if "ttisp" in extras:              # staggered-pair operators
        if args.small:
            _clocked(out, "ttisp", lambda: tti_throughput(wp, torch, dev, steps=10, nx=240, ny=240, nz=200, tti_operator=1))
        else:
            _clocked(out, "ttisp", lambda: tti_throughput(wp, torch, dev, steps=20, tti_operator=1))
    if "acoustic" in extras:
        if args.small:
            _clocked(out, "acoustic", lambda: acoustic_throughput(wp, torch, dev, steps=10, nx=240, ny=240, nz=200))
        else:
            _clocked(out, "acoustic", lambda: acoustic_throughput(wp, torch, dev))
    if "el2d" in extras:
        _clocked(out, "el2d", lambda: elastic2d_throughput(wp, torch, dev, small=args.small))
    if "rtm" in extras:
        _clocked(out, "rtm", lambda: rtm_shots_per_hour(wp, torch, dev, args.batch_shots, args.batch_nt, small=args.small))
    if "grad" in extras:
        _clocked(out, "grad", lambda: gradient_shots_per_hour(
            wp, torch, dev, args.grad_nt, [int(v) for v in args.grad_modes.split(",")], small=args.small))
    if "elgrad" in extras:
        _clocked(out, "elgrad", lambda: elastic_gradient_shots_per_hour(
            wp, torch, dev, args.grad_nt, [int(v) for v in args.grad_modes.split(",")], small=args.small))
    if "tiles" in extras:
        _clocked(out, "tiles", lambda: tile_heights(wp, torch, dev, small=args.small))
    if "gradaniso" in extras:
        _clocked(out, "gradaniso", lambda: gradient_aniso_cost(wp, torch, dev, small=args.small))
    if "gradsmall" in extras:
        _clocked(out, "gradsmall", lambda: gradient_small(wp, torch, dev))
    if "oracle3" in extras:           # CPU only: no clock record needed, but harmless
        _clocked(out, "oracle3", lambda: oracle_tti_industry())
    if "fwdbatch" in extras:          # forward modelling, industry-size and small windows
        _clocked(out, "fwdbatch", lambda: forward_batch_shots_per_hour(wp, torch, dev, args.batch_shots,
                                                                       args.batch_nt, kind=args.batch_kind))
        _clocked(out, "fwdbatchsmall", lambda: forward_batch_shots_per_hour(wp, torch, dev, args.batch_shots,
                                                                            args.batch_nt, windows=(40, 80, 60),
                                                                            kind=args.batch_kind))
    if "batchsmall" in extras:       # many small windows: 40-80 x 40-80 x 60 cells
        _clocked(out, "batchsmall", lambda: batch_shots_per_hour(wp, torch, dev, args.batch_shots, args.batch_nt,
                                                                 kind=args.batch_kind, windows=(40, 80, 60)))
    if "batch" in extras:
        _clocked(out, "batch", lambda: batch_shots_per_hour(wp, torch, dev, args.batch_shots, args.batch_nt,
                                            small=args.small, kind=args.batch_kind))
    return out


def main():
    global _CLK
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--small", action="store_true", help="reduced grid (debug)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle baseline")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the TTI so-12 industry-scale step rates reported beside the headline")
    ap.add_argument("--extra", default="",
                    help="comma list: tti, ttisp, acoustic, el2d, grad, elgrad, gradsmall, gradaniso, tiles, batch, rtm "
                         "(secondary measurements)")
    ap.add_argument("--grad-nt", type=int, default=600)
    ap.add_argument("--grad-modes", default="0,1,2,3",
                    help="storage modes of the grad/elgrad extras (0 full FP32, 1 FP32, 2 BF16, 3 FP16 checkpoints)")
    ap.add_argument("--batch-kind", default="tti", choices=["tti", "elastic"])
    ap.add_argument("--batch-shots", type=int, default=8)
    ap.add_argument("--batch-nt", type=int, default=150)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2004_10519_gb300 as wp
    extras = [e for e in args.extra.split(",") if e]
    if extras:
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        with Clocks(0) as clk:
            _CLK = clk
            out = run_extras(wp, torch, dev, args, extras)
            _CLK = None
        out["clocks"] = clk.summary()
        print(json.dumps(out), flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))

    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    prob = elastic_workload(args.small)
    # replicas: every rank models its own shot (independent problems)
    prop = wp.Propagator.from_problem(prob, stream=torch.cuda.current_stream(dev).cuda_stream)
    N = int(np.prod(prop.grid))
    tile = {"z": 32, "y": prop.tile_rows, "x": prop.tile_planes}
    nt = prob.nt
    wav = torch.from_numpy(prob.wavelet).to(dev)
    src = torch.from_numpy(prob.src).to(dev)
    rec = torch.from_numpy(prob.rec).to(dev)
    nrec, nsrc = prob.rec.shape[0], prob.src.shape[0]
    traces = torch.empty((nrec, nt), dtype=torch.float32, device=dev)
    resid = torch.from_numpy(np.random.default_rng(1).standard_normal((nrec, nt)).astype(np.float32)).to(dev)
    qout = torch.empty((nsrc, nt), dtype=torch.float32, device=dev)

    def one_step():
        prop.forward(wav, src, rec, out=traces)
        n1 = prop.last_launches()
        prop.adjoint(resid, src, rec, out=qout)
        return n1 + prop.last_launches()

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e0.record(stream)
        for _ in range(args.steps):
            launches += one_step()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    upd = N * 2 * nt * args.steps * world
    ms, rate = aggregate(ms, N * 2 * nt * args.steps, dist, dev)
    value = rate / 1e9

    # roofline of the dominant kernel: per-launch CUDA events on the library's
    # stream, forward step (the adjoint step is reported beside it)
    prop.profile(True)
    prop.step(50)
    f_ms, f_n = prop.kernel_stats(wp.K_EL_FWD)
    prop.adjoint(resid, src, rec, out=qout)
    a_ms, a_n = prop.kernel_stats(wp.K_EL_ADJ_U)
    prop.profile(False)
    hbm, src_peak = peaks()
    t_launch = f_ms / max(f_n, 1) / 1e3
    ach = ALG_BYTES["elastic"] * N / t_launch / 1e9
    roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "traffic": TRAFFIC_B_PER_PT["elastic"] * N,
            "kernel": "elastic forward step (velocity + stress passes)",
            "peak_source": src_peak, "launch_ms": t_launch * 1e3,
            "alg_bytes_per_launch": ALG_BYTES["elastic"] * N,
            "adjoint_launch_ms": a_ms / max(a_n, 1),
            "fp32": {"alg_flop_per_pt": FLOP_PER_PT["elastic"],
                     "achieved_tflops": FLOP_PER_PT["elastic"] * N / t_launch / 1e12,
                     "peak_tflops": wp.fp32_peak(), "peak_source": "measured (FMA loop)"}}

    # end to end through the C ABI with pinned host buffers
    h_wav = torch.from_numpy(prob.wavelet).pin_memory()
    h_src = torch.from_numpy(prob.src).pin_memory()
    h_rec = torch.from_numpy(prob.rec).pin_memory()
    h_res = resid.cpu().pin_memory()
    h_tr = torch.empty((nrec, nt), dtype=torch.float32).pin_memory()
    h_q = torch.empty((nsrc, nt), dtype=torch.float32).pin_memory()
    prop.forward(h_wav, h_src, h_rec, out=h_tr)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        prop.forward(h_wav, h_src, h_rec, out=h_tr)
        prop.adjoint(h_res, h_src, h_rec, out=h_q)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    h2d = (h_wav.numel() + h_src.numel() + h_rec.numel() + h_res.numel() + h_src.numel() + h_rec.numel()) * 4
    d2h = (h_tr.numel() + h_q.numel()) * 4
    e2e = {"value": upd / e2e_s / 1e9, "unit": "Gpts/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h}

    prop.close()
    # secondary: TTI so 12 forward and adjoint steps at the industry-scale
    # grid (800x800x400 + 40-cell layer = 880x880x480), one GPU only
    secondary = None
    if world == 1 and not args.no_secondary:
        with Clocks(local) as clk2:
            _CLK = clk2
            if args.small:
                tti = tti_throughput(wp, torch, dev, steps=10, nx=240, ny=240, nz=200)
            else:
                tti = tti_throughput(wp, torch, dev)
            _CLK = None
        tti["clocks"] = clk2.summary()
        secondary = {"tti_so12_industry_grid": tti}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(prob)
    if rank == 0:
        line = {"metric": "elastic propagator grid-point updates per second",
                "value": value, "unit": "Gpts/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": prob.name, "grid": list(prop.grid), "space_order": prob.so,
                           "physical_grid": [prob.nx, prob.ny, prob.nz],
                           "physical_gpts_per_s": value * (prob.nx * prob.ny * prob.nz) / float(np.prod(prop.grid)),
                           "time_steps_per_bench_step": 2 * nt, "shots_per_gpu": 1,
                           "parallelism": f"replicas{world}", "tile": tile,
                           "l2": "working set 2.2 GB >> L2 (no flush needed)"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk.summary()}
        if secondary:
            line["secondary"] = secondary
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
