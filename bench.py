#!/usr/bin/env python3
"""Benchmark of the pseudospectral Navier-Stokes hot path on one GB300.

One "step" is one integrating-factor RK2 step (two nonlinear-term
evaluations: 6 inverse + 3 forward 3D transforms each, the cross product,
projection, dealiasing and update) plus the per-step FP64 energy/enstrophy
reduction, over the whole grid.

Default workload (the configuration the headline metric is quoted on, the
precision form): 512^3 forced turbulence (ABC forcing k = 3, F = 0.5,
nu = 2e-3, dt = 1e-3, seeded k^-2 start), in the plain FP64 form (the
paper's precision), timed over K RK2 steps; the fused FP32 form runs the same
workload beside it and its relative L2 distance to the FP64 state is
reported.  The plain form's transforms skip the lines the 2/3 rule zeroes
or discards; the same form with every line done runs too, and the line
reports its steps/s and whether its state equals the pruned one bit for bit.
The large form rides along in the same line: 1024^3 forced
turbulence in the fused FP32 form, and the plain FP64 form at 768^3 for
comparison.  The standalone 3-component FFT stage is timed at 512^3 and
1024^3, and the device's FP64 FMA rate is measured for the FP64 roofline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference      # the FP64 CPU oracle on the host cores

Under torchrun (N > 1) every rank advances its own replica (weak scaling,
no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RK2 steps/s and 3D-FFT HBM GB/s, FP32 fused vs FP64 plain at stated L2 error"

WORKLOADS = {
    "tg256": dict(desc="256^3 decaying Taylor-Green vortex, nu=1/1600, dt=2e-3, plain FP64 "
                       "(FP32 form alongside)", n=256, nu=1 / 1600, dt=2e-3, ic="tg",
                  prec="fp64", companion="fp32"),
    "forced512": dict(desc="512^3 forced turbulence, ABC forcing k=3 F=0.5, nu=2e-3, dt=1e-3, "
                           "seeded k^-2 start on 1<=|k|<=4 (seed 3), plain FP64 (fused FP32 "
                           "alongside)",
                      n=512, nu=2e-3, dt=1e-3, force_amp=0.5, force_k=3, ic=("turb", 3),
                      prec="fp64", companion="fp32", large=("forced1024", "plain768")),
    "forced1024": dict(desc="1024^3 forced turbulence, ABC forcing k=3 F=0.5, nu=5e-4, dt=5e-4, "
                            "seeded k^-2 start (seed 5), FP32", n=1024, nu=5e-4, dt=5e-4,
                       force_amp=0.5, force_k=3, ic=("turb", 5), prec="fp32", companion=None),
    "ensemble48": dict(desc="48 independent runs, 16 each at 64^3, 96^3 and 128^3, FP32, "
                            "nu_r = 5e-3 + 1.5e-2 U(4999, r), dt=1e-3, seeded k^-2 starts on "
                            "1<=|k|<=4 (seeds 4000+r); FP64 plain ensemble alongside",
                       n=128, ensemble=48, dt=1e-3, prec="fp32", companion="fp64"),
    "mhd256": dict(desc="256^3 forced MHD (Alfven units), nu=eta=2e-3, dt=1e-3, ABC forcing k=3 "
                        "F=0.5 on u, seeded k^-2 starts for u (seed 7) and b (seed 57), plain FP64 "
                        "(plain FP32 alongside)", n=256, nu=2e-3, eta=2e-3, dt=1e-3, force_amp=0.5,
                   force_k=3, ic=("mhd", 7), mhd=1, prec="fp64", companion="fp32"),
    "plain768": dict(desc="768^3 forced turbulence, ABC forcing k=3 F=0.5, nu=5e-4, dt=5e-4, "
                          "seeded k^-2 start (seed 5), plain FP64", n=768, nu=5e-4, dt=5e-4,
                     force_amp=0.5, force_k=3, ic=("turb", 5), prec="fp64", companion=None),
    "box512x512x256": dict(desc="512x512x256 grid on the box of sides (2pi, 2pi, pi) (aspect ratio "
                                "2, the spacing of 512^3), forced turbulence, ABC forcing k=2 F=0.5, "
                                "nu=2e-3, dt=1e-3, seeded k^-2 start on 1<=|k|<=4 (seed 3), plain "
                                "FP64 (plain FP32 alongside)", n=512, ny=512, nz=256, lz=0.5,
                           nu=2e-3, dt=1e-3, force_amp=0.5, force_k=2, ic=("grid", 3),
                           prec="fp64", companion="fp32"),
}


def dims_of(r):
    """Grid points (N_x, N_y, N_z) of a run (dict with n and optionally ny, nz)."""
    n = r["n"]
    return (n, r.get("ny", 0) or n, r.get("nz", 0) or n)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return dict(hbm_gbs=float(d["hbm_gbs"]), sm_max_mhz=float(d.get("sm_max_mhz", 2070.0)),
                    source="measured")
    return dict(hbm_gbs=6800.0, sm_max_mhz=2070.0, source="fallback")


# Kernel sources of each form, for telling whether a committed ncu capture
# still describes the kernels that run.
KERNEL_SOURCES = {
    "fp64": ("fft_core.cuh", "fft_passes.cu", "plain.cu", "plain.h", "grid.cuh", "reduce.cuh", "api.cu"),
    "fp32": ("fft_core.cuh", "fft_ct.cuh", "reduce.cuh", "fused.cu", "fused.h", "fused_access.cuh",
             "fused_s.cuh", "fused_k.cuh", "fused_kA.cu", "fused_kB.cu", "fused_kD.cu",
             "fused_kE.cu", "fused_keu.cu", "fused_update.cuh", "fused_sA.cu", "fused_sB.cu",
             "fused_sDE.cu", "fused_z.cu", "fused_zr.cuh", "fused_zr2.cu", "fused_zr3.cu",
             "fused_zr4.cu", "fused_zr5.cu", "fused_zm.cu"),
}


def source_hash(prec):
    import hashlib
    h = hashlib.sha256()
    for fn in KERNEL_SOURCES[prec]:
        with open(os.path.join(ROOT, "paper_1003_4322_gb300", "csrc", fn), "rb") as g:
            h.update(g.read())
    return h.hexdigest()


def captured_traffic(workload, prec, kernel):
    """DRAM bytes per launch of a kernel from the committed ncu summary of this
    workload, if that form's kernel sources are unchanged since the capture."""
    path = os.path.join(ROOT, "profiles", f"traffic_{workload}.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        t = json.load(f).get(prec, {})
    if t.get("source_sha256") != source_hash(prec):
        return None
    return t.get("kernels", {}).get(kernel)


# FP64 FMA pipes: GB300 lists 1.25 TFLOP/s FP64 at its 2070 MHz maximum SM
# clock over 152 SMs, i.e. 2 FP64 FMA (4 flop) per SM per clock.
FP64_FLOP_PER_SM_CLK = 4.0
N_SM = 152


def members(w):
    """(run parameters, initial states) of every run of the workload."""
    import numpy as np

    from paper_1003_4322_gb300 import inputs
    if w.get("ensemble"):
        runs, ics = [], []
        for r in range(w["ensemble"]):
            n = (64, 96, 128)[r * 3 // w["ensemble"]]
            runs.append(dict(n=n, nu=inputs.ensemble_nu(r), dt=w["dt"]))
            ics.append(inputs.turbulence_state(n, 4000 + r))
        return runs, ics
    run = dict(n=w["n"], nu=w["nu"], dt=w["dt"], force_amp=w.get("force_amp", 0.0),
               force_k=w.get("force_k", 0), dealias=w.get("dealias", 0))
    for k in ("ny", "nz", "lx", "ly", "lz"):
        if k in w:
            run[k] = w[k]
    if w["ic"] == "tg":
        return [run], [inputs.taylor_green_state(w["n"])]
    kind, seed = w["ic"]
    if kind == "mhd":   # state [u; b]
        run.update(eta=w["eta"], mhd=1)
        u = inputs.turbulence_state(w["n"], seed)
        b = inputs.random_solenoidal_state(w["n"], 1.0, 4.0, 0.7, seed=seed + 50)
        return [run], [np.concatenate([u, b])]
    if kind == "grid":
        box = tuple(run.get(k, 1.0) for k in ("lx", "ly", "lz"))
        return [run], [inputs.random_solenoidal_grid(dims_of(run), box, 1.0, 4.0, 1.0, seed)]
    return [run], [inputs.turbulence_state(w["n"], seed)]


def load_state(s, a0, run):
    """Velocity (and, for a six-component MHD state, the magnetic field)."""
    s.set_field(0, a0[:3], run=run)
    if a0.shape[0] == 6:
        s.set_field(1, a0[3:], run=run)


def read_state(s, runs, run):
    import numpy as np
    u = s.get_field(0, run=run)
    return np.concatenate([u, s.get_field(1, run=run)]) if runs[run].get("mhd") else u


# ---------------------------------------------------------------- kernel model

def plain_keep(dims, dealias=0):
    """Largest |m_i| per axis that the dealiasing rule keeps (3 |m| < N_i for
    the cubic and spherical 2/3 rules; 2 |m| < N_i and 9 m^2 < 2 N_i^2 for the
    phase-shift rule): the plain form's transforms skip the lines beyond it,
    unless NS_PLAIN_PRUNE=0 (then None)."""
    if os.environ.get("NS_PLAIN_PRUNE", "1").startswith("0"):
        return None
    def k(n):
        m = n // 2
        while m >= 0 and not ((2 * m < n and 9 * m * m < 2 * n * n) if dealias == 2 else 3 * m < n):
            m -= 1
        return m
    return tuple(k(d) for d in dims)


PLAIN_KERNELS = ("fft_x_inverse", "fft_x_forward", "fft_y_inverse", "fft_y_forward", "fft_z_c2r",
                 "fft_z_r2c")
PLAIN_POINTWISE = ("curl", "update", "update_b", "energy_partials")


def kernel_model(name, n, prec, keep=None):
    """Algorithmic (bytes, flops) of one launch of a kernel of the step (three
    vector components per launch) on the grid n (N of a cube, or (N_x, N_y,
    N_z) for the plain kernels).  FFT flops use 5 n log2 n per complex line
    of length n.  keep (plain form): the kept (K_x, K_y, K_z), whose lines
    alone the transforms do and whose rows alone they read (inverse) or
    write (forward); None: every line."""
    es = 8 if prec == "fp64" else 4
    nx, ny, nz = (n, n, n) if isinstance(n, int) else n
    n = nx
    nh = nz // 2 + 1
    M = nx * ny * nh        # half-layout modes per component
    V = nx * ny * nz
    f_zline = 5 * (nz // 2) * math.log2(nz // 2) + 10 * (nz // 2)
    kx, ky, kz = keep if keep else (nx, ny, nh - 1)
    rx, ry = (2 * kx + 1, 2 * ky + 1) if keep else (nx, ny)   # rows along x, y kept
    cx = (2 * ky + 1) * (kz + 1) if keep else ny * nh          # x lines per component
    cy = nx * (kz + 1) if keep else nx * nh                    # y lines per component
    zk = kz + 1 if keep else nh                                # kz entries per z line
    if name in ("fft_x_inverse", "fft_x_forward"):
        return 3 * cx * (rx + nx) * 2 * es, 3 * cx * 5 * nx * math.log2(nx)
    if name in ("fft_y_inverse", "fft_y_forward"):
        return 3 * cy * (ry + ny) * 2 * es, 3 * cy * 5 * ny * math.log2(ny)
    if name in ("fft_z_c2r", "fft_z_r2c"):
        return 3 * (nx * ny * zk * 2 * es + V * es), 3 * nx * ny * f_zline
    if name in ("fft_c2r_std", "fft_r2c_std"):   # all three passes of three components
        flops = 3 * (ny * nh * 5 * nx * math.log2(nx) + nx * nh * 5 * ny * math.log2(ny) + nx * ny * f_zline)
        return 3 * (M * 2 * es + V * es) + 2 * (2 * 3 * M * 2 * es), flops
    rect = (2 * kx + 1) * (2 * ky + 1) * (kz + 1) if keep else M   # modes the pruned FP64 form touches
    if name == "curl":
        return 2 * 3 * rect * 2 * es, 3 * rect * 6
    if name == "energy_partials":   # reads three components (of the rectangle, when pruned)
        return 3 * rect * 2 * es, 3 * rect * 4
    if name == "cross":
        return 9 * V * es, 9 * V
    if name == "cross_mhd":     # reads u, w, b, j; writes u x w + j x b and u x b
        return 18 * V * es, 30 * V
    if name in ("update", "update_b"):
        # writes three components of every mode (of the rectangle, when
        # pruned); reads the transformed product, the state (and the stage-1
        # state at stage 2: 7.5 components on average) of the kept modes only
        kept = (2 * ((nx - 1) // 3) + 1) * (2 * ((ny - 1) // 3) + 1) * ((nz - 1) // 3 + 1)
        return (3 * rect + 7.5 * kept) * 2 * es, 3 * kept * 20
    # fused form (FP32 complex = 8 bytes; only the kept modes move): compact
    # state [ikx][iky][kz], A / D fields [iky][x][kz], B / C fields [y][x][kz]
    f_line, f_yline = 5 * nx * math.log2(nx), 5 * ny * math.log2(ny)
    K, Ky, Kz = (nx - 1) // 3, (ny - 1) // 3, (nz - 1) // 3
    Mx, My, Mz = 2 * K + 1, 2 * Ky + 1, Kz + 1
    S = Mx * My * Mz            # compact modes per component
    Ax = My * nx * Mz           # pass A / D field size
    Bx = ny * nx * Mz           # pass B / C field size
    cb = 8
    if name == "fused_A_x_inverse_curl":
        return (3 * S + 6 * Ax) * cb, 6 * My * Mz * f_line
    if name == "fused_B_y_inverse":
        return (6 * Ax + 6 * Bx) * cb, 6 * nx * Mz * f_yline
    if name == "fused_C_z_nonlinear":
        return (6 * Bx + 3 * Bx) * cb, nx * ny * (9 * f_zline + 9 * nz)
    if name == "fused_D_y_forward":
        return (3 * Bx + 3 * Ax) * cb, 3 * nx * Mz * f_yline
    if name == "fused_E_x_forward":
        return (3 * Ax + 3 * S) * cb, 3 * My * Mz * f_line
    if name == "fused_update":
        return 10.5 * S * cb, 3 * S * 30   # reads N, a (and a1 at stage 2), writes 3
    if name == "fused_C_z_mhd":               # reads u, w, b, j; writes u x w + j x b, u x b
        return (12 * Bx + 6 * Bx) * cb, n * n * (18 * f_zline + 30 * n)
    if name == "fused_update_b":              # reads N_b, b (and b1 at stage 2), writes 3
        return 10.5 * S * cb, 3 * S * 25
    if name == "fused_E_x_forward_update":   # reads D, a (and a1 at stage 2), writes 3
        return (3 * Ax + 7.5 * S) * cb, 3 * Mx * Mz * f_line + 3 * S * 30
    return 0, 0


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.proc = None
        self.path = None
        self.gpu = gpu_index

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for i, nm in enumerate(names):
                if r[5 + i].lower().startswith("active"):
                    reasons.add(nm)
        load = [s for s, p in zip(sm, pw)] if sm else []
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(pw) if pw else None,
                "samples": len(rows), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- GPU arm

def time_form(w, prec, mem, steps, warmup, census_steps, dist, keep_states=True):
    """Advance one solver (all runs of the workload) through warm-up, K timed
    steps and a kernel census; returns timing, census, final states (host
    copies, unless keep_states is false) and the energy series of run 0."""
    import torch

    from paper_1003_4322_gb300 import _native as nat
    from paper_1003_4322_gb300.solver import Solver
    stream = torch.cuda.current_stream()
    runs, ics = mem
    s = Solver(runs, prec=prec, stream=stream)
    for i, a0 in enumerate(ics):
        load_state(s, a0, i)
    s.step(warmup)
    s.sync()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # one event between consecutive steps (graph launches) on the launching
    # stream: the total, and the median and best single step
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    evs[0].record(stream)
    for i in range(steps):
        s.step(1)
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = evs[0].elapsed_time(evs[-1])
    per = sorted(evs[i].elapsed_time(evs[i + 1]) for i in range(steps))
    clk = clocks.stop()
    E, O = s.series(count=steps)
    census = nat.ns_kernel_census(s.ctx, census_steps) if census_steps > 0 else []
    desc = nat.ns_describe_run(s.ctx, 0)
    states = [read_state(s, runs, i) for i in range(len(runs))] if keep_states else None
    return dict(solver=s, ms=ms, clocks=clk, census=census, states=states, E=E, O=O, desc=desc,
                step_ms_median=statistics.median(per), step_ms_min=per[0])


def roofline_of(census, w, prec, census_steps, peaks, sm_mhz, sizes=None):
    """Dominant kernel (largest share of device time in the census) against
    HBM or the FP64 ALU roof, whichever its algorithmic model says binds."""
    if not census:
        return None, None
    total = sum(t for _, _, t in census)
    name, launches, tms = max(census, key=lambda r: r[2])
    per_launch_ms = tms / launches
    # fused form: one launch covers every run of a group (runs of equal N);
    # plain form: one launch per run
    sizes = sizes or [dims_of(w)]
    # the plain transforms skip lines in both precisions; the pointwise
    # kernels keep to the rectangle in FP64 only
    plain = name in PLAIN_KERNELS or (prec == "fp64" and name in PLAIN_POINTWISE)
    per_size = [kernel_model(name, n, prec, plain_keep(n if not isinstance(n, int) else (n, n, n),
                                                       w.get("dealias", 0)) if plain else None)
                for n in sizes]
    launches_per_pass = len(sizes) if prec == "fp64" else len(set(sizes))
    bytes_ = sum(b for b, _ in per_size) / launches_per_pass
    flops = sum(f for _, f in per_size) / launches_per_pass
    gbs = bytes_ / (per_launch_ms * 1e-3) / 1e9
    hbm_frac = gbs / peaks["hbm_gbs"]
    roof = {"kernel": name, "launches_per_step": launches / census_steps,
            "share": tms / total, "avg_launch_ms": per_launch_ms,
            "traffic": captured_traffic(w.get("name", ""), prec, name), "algorithmic_bytes": bytes_}
    if prec == "fp64":
        if peaks.get("fp64_flops"):
            peak_flops = peaks["fp64_flops"]
            src = ("measured: ns_alu_peak, independent FP64 FMA chains on every SM, CUDA events, "
                   "in this run")
        else:
            peak_flops = N_SM * FP64_FLOP_PER_SM_CLK * peaks["sm_max_mhz"] * 1e6
            src = "FP64 FMA pipes x max SM clock (derived)"
        tflops = flops / (per_launch_ms * 1e-3) / 1e12
        alu_frac = tflops * 1e12 / peak_flops
        if alu_frac >= hbm_frac:
            roof.update(bound="alu", achieved=tflops, peak=peak_flops / 1e12, unit="TFLOP/s",
                        frac=alu_frac, peak_source=src, hbm_frac=hbm_frac)
            return roof, total
    roof.update(bound="hbm", achieved=gbs, peak=peaks["hbm_gbs"], unit="GB/s", frac=hbm_frac,
                peak_source=peaks["source"])
    return roof, total


def fft_stage(n, prec, reps=5, ncomp=3, window=False):
    """Standalone ns_fft_r2c + ns_fft_c2r of ncomp components (ns_fft_*_grid
    on a grid (N_x, N_y, N_z) that is not a cube): HBM GB/s by the
    algorithmic model (each of the 3 passes reads and writes the array).
    window: bracket one more r2c and c2r with cudaProfilerStart/Stop, for a
    profiler started with its capture off (ncu --profile-from-start off)."""
    import torch

    from paper_1003_4322_gb300 import _native as nat
    nx, ny, nz = (n, n, n) if isinstance(n, int) else n
    cube = nx == ny == nz
    rt = torch.float32 if prec == "fp32" else torch.float64
    ct = torch.complex64 if prec == "fp32" else torch.complex128
    g = torch.Generator(device="cuda").manual_seed(1)
    u = torch.randn((ncomp, nx, ny, nz), device="cuda", dtype=rt, generator=g)
    uh = torch.empty((ncomp, nx, ny, nz // 2 + 1), device="cuda", dtype=ct)
    back = torch.empty_like(u)
    stream = torch.cuda.current_stream()
    ctx = nat.ns_init([dict(n=8, dt=1e-3)], nat.NS_FP32 if prec == "fp32" else nat.NS_FP64,
                      stream)

    def fwd():
        if cube:
            nat.ns_fft_r2c(ctx, nx, ncomp, u, uh)
        else:
            nat.ns_fft_r2c_grid(ctx, nx, ny, nz, ncomp, u, uh)

    def inv():
        if cube:
            nat.ns_fft_c2r(ctx, nx, ncomp, uh, back)
        else:
            nat.ns_fft_c2r_grid(ctx, nx, ny, nz, ncomp, uh, back)
    try:
        for _ in range(2):
            fwd()
            inv()
        torch.cuda.synchronize()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        evs[0].record(stream)
        for _ in range(reps):
            fwd()
        evs[1].record(stream)
        for _ in range(reps):
            inv()
        evs[2].record(stream)
        torch.cuda.synchronize()
        r2c_ms = evs[0].elapsed_time(evs[1]) / reps
        c2r_ms = evs[1].elapsed_time(evs[2]) / reps
        if window:
            torch.cuda.profiler.start()
            fwd()
            inv()
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
    finally:
        nat.ns_destroy(ctx)
    es = 4 if prec == "fp32" else 8
    half = nx * ny * (nz // 2 + 1) * 2 * es
    real = nx * ny * nz * es
    model = ncomp * ((real + half) + 2 * half + 2 * half)   # z, y, x passes (read + write)
    out = {"n": nx if cube else [nx, ny, nz], "ncomp": ncomp, "prec": prec, "r2c_ms": r2c_ms,
           "c2r_ms": c2r_ms,
           "r2c_gbs": model / (r2c_ms * 1e-3) / 1e9, "c2r_gbs": model / (c2r_ms * 1e-3) / 1e9,
           "bytes_model": model}
    out["cufft_reference"] = cufft_reference(u, uh, back, reps, model)
    return out


def cufft_reference(u, uh, back, reps, model):
    """cuFFT (through torch.fft) on the same arrays, unnormalised both ways,
    timed the same way: a reference point only, never on the product path."""
    import torch
    shape = tuple(u.shape[-3:])
    dims = (-3, -2, -1)
    ours = uh.clone()
    ref_h = torch.empty_like(uh)
    ref_b = torch.empty_like(back)
    stream = torch.cuda.current_stream()
    for _ in range(2):
        torch.fft.rfftn(u, dim=dims, norm="backward", out=ref_h)
        torch.fft.irfftn(ref_h, s=shape, dim=dims, norm="forward", out=ref_b)
    torch.cuda.synchronize()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    evs[0].record(stream)
    for _ in range(reps):
        torch.fft.rfftn(u, dim=dims, norm="backward", out=ref_h)
    evs[1].record(stream)
    for _ in range(reps):
        torch.fft.irfftn(ref_h, s=shape, dim=dims, norm="forward", out=ref_b)
    evs[2].record(stream)
    torch.cuda.synchronize()
    r2c = evs[0].elapsed_time(evs[1]) / reps
    c2r = evs[1].elapsed_time(evs[2]) / reps
    diff = float(torch.linalg.vector_norm(ours - ref_h) / torch.linalg.vector_norm(ref_h))
    return {"library": "cuFFT via torch.fft.rfftn / irfftn", "r2c_ms": r2c, "c2r_ms": c2r,
            "r2c_gbs_by_same_model": model / (r2c * 1e-3) / 1e9,
            "c2r_gbs_by_same_model": model / (c2r * 1e-3) / 1e9,
            "rel_diff_r2c_vs_ours": diff}


def e2e(w, prec, mem, steps):
    """Through the public API with host buffers: every step uploads every
    run's input state from pinned host memory (ns_set_states; ns_set_field per
    run for MHD states), advances one RK2 step (ns_step), reads every run's
    energy, enstrophy and spectrum back (ns_energy_spectra) and reads every
    run's advanced state back into pinned host memory (ns_get_state, or
    ns_get_field per field for MHD states)."""
    import numpy as np
    import torch

    from paper_1003_4322_gb300.solver import Solver
    runs, ics = mem
    hosts, outs = [], []
    for a0 in ics:
        pinned = torch.empty(a0.shape, dtype=torch.complex128, pin_memory=True)
        pinned.numpy()[...] = a0
        hosts.append(pinned.numpy())
        outs.append(torch.empty(a0.shape, dtype=torch.complex128, pin_memory=True).numpy())
    s = Solver(runs, prec=prec, stream=torch.cuda.current_stream())
    nr = len(runs)

    mhd = any(r.get("mhd") for r in runs)

    def one_step():
        if mhd:   # velocity and magnetic field, run by run
            for i, h in enumerate(hosts):
                load_state(s, h, i)
        else:     # every run's state in one call, one synchronisation
            s.set_states(hosts)
        s.step(1)
        E, O, spec = s.energy_spectra()   # every run's diagnostics in one round trip
        for i, o in enumerate(outs):
            s.get_field(0, run=i, out=o[:3])
            if o.shape[0] == 6:
                s.get_field(1, run=i, out=o[3:])
        return [E, O, spec]
    try:
        for _ in range(2):
            one_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            specs = one_step()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    finally:
        s.close()
    if not all(np.isfinite(o).all() for o in outs[:1]):
        raise RuntimeError("e2e: the state read back is not finite")
    return {"value": nr * steps / dt, "unit": "run-steps/s" if nr > 1 else "steps/s",
            "h2d_bytes_per_step": int(sum(h.nbytes for h in hosts)),
            "d2h_bytes_per_step": int(sum(x.nbytes for x in specs) + sum(o.nbytes for o in outs)),
            "steps": steps}


def oracle_steps(mem, budget_s, max_steps, warmup=0, warm_budget_s=None):
    """Whole RK2 steps of the oracle (as it stands) over the workload's runs,
    cycling through the members: `warmup` untimed steps (fewer if they use
    warm_budget_s, by default budget_s), then timed steps until max_steps or
    the budget (at least one of each kind asked for).
    Returns (timed steps, their seconds, threads, warm-up steps done)."""
    import oracle
    cores = oracle.set_threads(os.cpu_count() or 1)
    runs, ics = mem
    states = list(ics)
    params = [oracle.Params(n=r["n"], nu=r["nu"], dt=r["dt"], force_amp=r.get("force_amp", 0.0),
                            force_k=r.get("force_k", 0), dealias=r.get("dealias", 0),
                            eta=r.get("eta", 0.0), mhd=r.get("mhd", 0), ny=r.get("ny", 0),
                            nz=r.get("nz", 0), lx=r.get("lx", 0.0), ly=r.get("ly", 0.0),
                            lz=r.get("lz", 0.0)) for r in runs]
    done = 0

    def one():
        nonlocal done
        i = done % len(runs)
        states[i] = oracle.step(states[i], params[i], 1)
        done += 1

    tw = time.perf_counter()
    warm = 0
    wb = budget_s if warm_budget_s is None else warm_budget_s
    while warm < warmup and time.perf_counter() - tw <= wb:
        one()
        warm += 1
    t0 = time.perf_counter()
    steps = 0
    while steps < max_steps:
        one()
        steps += 1
        if time.perf_counter() - t0 > budget_s:
            break
    return steps, time.perf_counter() - t0, cores, warm


def cpu_baseline(w, mem, budget_s=30.0):
    """The FP64 oracle (test infrastructure, as it stands) on the host cores:
    whole RK2 steps of the same workload until the time budget is used (at
    least one; after one untimed step when the grid is small enough that a
    step takes well under the budget)."""
    big = max(math.prod(dims_of(r)) for r in mem[0]) >= 256 ** 3
    steps, dt, cores, warm = oracle_steps(mem, budget_s, 1000, warmup=0 if big else 1)
    nr = len(mem[0])
    unit = "run-steps/s" if nr > 1 else "steps/s"
    return {"value": steps / dt, "unit": unit, "cores": cores, "kind": "oracle",
            "sample": f"{steps} whole RK2 step(s) of {'members of ' if nr > 1 else ''}the "
                      f"workload on {cores} host threads ({dt:.1f} s), after {warm} untimed"}


def max_over_ranks(ms, dist, device=None):
    """Largest elapsed time over all ranks (the job's time); a plain float
    when there is no process group."""
    if not dist:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, ms):
    """Whole-job throughput: the units all ranks processed over the job time."""
    return world * units_per_rank / (ms * 1e-3)


def config_of(args, w, world):
    """The workload block both arms print, identical for the same command."""
    return {"workload": args.workload, "description": w["desc"], "n": w["n"],
            "grid": list(dims_of(w)), "box_over_2pi": [w.get(k, 1.0) for k in ("lx", "ly", "lz")],
            "dealias": w.get("dealias", 0), "nu": w.get("nu"), "dt": w["dt"],
            "runs": w.get("ensemble", 1), "parallelism": f"replicas x{world}",
            "l2": "working set above 129 MB L2 (no flush needed)"}


def measure_alu_peaks(peaks):
    """FP64 (and FP32) FMA rate of this device, with the SM clock sampled
    while the FP64 probe runs; the FP64 rate becomes the plain form's roof."""
    import torch

    from paper_1003_4322_gb300 import _native as nat
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    fp64 = nat.ns_alu_peak(nat.NS_FP64, 400.0, torch.cuda.current_stream())
    clk = clocks.stop()
    fp32 = nat.ns_alu_peak(nat.NS_FP32, 200.0, torch.cuda.current_stream())
    peaks["fp64_flops"] = fp64
    sm = (clk or {}).get("sm_mhz")
    return {"fp64_tflops": fp64 / 1e12, "fp32_tflops": fp32 / 1e12,
            "fp64_fma_per_sm_per_clk": fp64 / 2 / (N_SM * sm * 1e6) if sm else None,
            "clocks": clk, "how": "ns_alu_peak: 8 independent FMA chains per thread, every SM "
                                  "filled to its occupancy limit, best of 3 launches (CUDA events)"}


def large_form(args, peaks, dist):
    """The large configuration beside the headline: 1024^3 forced turbulence
    in the fused FP32 form (steps/s, roofline, e2e, FFT stage at 1024^3) and
    the plain FP64 form at 768^3 for comparison."""
    out = {}
    w = dict(WORKLOADS["forced1024"], name="forced1024")
    mem = members(w)
    steps = min(args.steps, 20)
    t = time_form(w, "fp32", mem, steps, 3, 2, dist, keep_states=False)
    roof, _ = roofline_of(t["census"], w, "fp32", 2, peaks, None, [dims_of(w)])
    t["solver"].close()
    out["forced1024_fp32"] = {
        "description": w["desc"], "value": steps / (t["ms"] * 1e-3), "unit": "steps/s",
        "ms_per_step": t["ms"] / steps, "steps": steps, "warmup": 3, "roofline": roof,
        "execution": t["desc"], "clocks": t["clocks"],
        "kernels": [{"name": n, "launches": l, "ms": ms} for n, l, ms in t["census"]],
        "e2e": e2e(w, "fp32", mem, min(steps, 10))}
    if not args.no_fft:
        out["fft_1024"] = fft_stage(1024, "fp32")
    del mem
    w = dict(WORKLOADS["plain768"], name="plain768")
    mem = members(w)
    steps = min(args.steps, 5)
    t = time_form(w, "fp64", mem, steps, 3, 1, dist, keep_states=False)
    roof, _ = roofline_of(t["census"], w, "fp64", 1, peaks, None, [dims_of(w)])
    t["solver"].close()
    out["plain768_fp64"] = {"description": w["desc"], "value": steps / (t["ms"] * 1e-3),
                            "unit": "steps/s", "ms_per_step": t["ms"] / steps, "steps": steps,
                            "warmup": 3, "roofline": roof, "clocks": t["clocks"]}
    return out


def plain_unpruned(w, mem, steps, warmup, census_steps, main, dist):
    """The plain form with every line of its transforms done (NS_PLAIN_PRUNE=0):
    the same workload and step counts, its steps/s, and whether its states
    equal the pruned run's bit for bit (they must: the skipped lines are the
    ones the 2/3 rule zeroes or discards)."""
    import numpy as np
    old = os.environ.get("NS_PLAIN_PRUNE")
    os.environ["NS_PLAIN_PRUNE"] = "0"
    try:
        u = time_form(w, "fp64", mem, steps, warmup, census_steps, dist)
    finally:
        if old is None:
            del os.environ["NS_PLAIN_PRUNE"]
        else:
            os.environ["NS_PLAIN_PRUNE"] = old
    u["solver"].close()
    nr = len(mem[0])
    same = all(np.array_equal(a, b) for a, b in zip(u["states"], main["states"]))
    return {"value": nr * steps / (u["ms"] * 1e-3), "unit": "run-steps/s" if nr > 1 else "steps/s",
            "ms_per_step": u["ms"] / steps, "states_bitwise_equal_to_pruned": bool(same),
            "kernels": [{"name": n, "launches": l, "ms": t} for n, l, t in u["census"]]}


def ours(args, w):
    import numpy as np
    import torch

    from paper_1003_4322_gb300 import _native as nat
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as td
        td.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = td
    torch.cuda.set_device(local)
    nat.load()
    peaks = load_peaks()
    alu = measure_alu_peaks(peaks)
    mem = members(w)
    nr = len(mem[0])
    warmup = max(args.warmup, 3)
    census_steps = min(args.steps, 3)

    main = time_form(w, w["prec"], mem, args.steps, warmup, census_steps, dist)
    ms = max_over_ranks(main["ms"], dist, "cuda")
    value = job_rate(nr * args.steps, world, ms)
    points = sum(math.prod(dims_of(r)) for r in mem[0])
    clk = main["clocks"] or {}
    sizes = [dims_of(r) for r in mem[0]]
    roof, census_total = roofline_of(main["census"], w, w["prec"], census_steps, peaks,
                                     clk.get("sm_mhz"), sizes)
    launches_per_step = sum(l for _, l, _ in main["census"]) / census_steps if main["census"] else 0
    main["solver"].close()

    comp = None
    if w.get("companion") and not args.no_companion:
        c = time_form(w, w["companion"], mem, args.steps, warmup, census_steps, dist)
        croof, _ = roofline_of(c["census"], w, w["companion"], census_steps, peaks, None, sizes)
        from oracle import rel_l2
        fp32, fp64 = (c["states"], main["states"]) if w["companion"] == "fp32" else \
            (main["states"], c["states"])
        comp = {"form": w["companion"], "value": nr * args.steps / (c["ms"] * 1e-3),
                "unit": "run-steps/s" if nr > 1 else "steps/s", "ms_per_step": c["ms"] / args.steps,
                "rel_l2_fp32_vs_fp64": max(rel_l2(a, b) for a, b in zip(fp32, fp64)),
                "after_steps": warmup + args.steps + census_steps, "roofline": croof,
                "execution": c["desc"], "clocks": c["clocks"],
                "kernels": [{"name": n, "launches": l, "ms": t} for n, l, t in c["census"]]}
        c["solver"].close()
    unpruned = None
    if w["prec"] == "fp64" and not args.no_unpruned:
        unpruned = plain_unpruned(w, mem, args.steps, warmup, census_steps, main, dist)
    main["states"] = None

    fft = fft_stage(dims_of(w) if "ny" in w else w["n"], "fp32") if not args.no_fft else None
    ee = e2e(w, w["prec"], mem, min(args.steps, 20))
    large = large_form(args, peaks, dist) if w.get("large") and not args.no_large else None
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, mem, args.cpu_budget)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    step_idx = [i for i in (49, 99, 149, 199) if i < len(main["E"])]
    line = {
        "metric": METRIC, "value": value, "unit": "run-steps/s" if nr > 1 else "steps/s",
        "n_gpus": world, "runs": nr, "grid_point_steps_per_s": value * points / nr,
        "steps": args.steps, "warmup": warmup, "ms_per_step": ms / args.steps,
        "ms_per_step_median": main["step_ms_median"], "ms_per_step_min": main["step_ms_min"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if w["prec"] == "fp64" else "f32",
        "data": "synthetic (analytic / seeded initial condition, no dataset)",
        "config": config_of(args, w, world),
        "form": main["desc"]["form"], "execution": main["desc"],
        "roofline": roof, "gpu_launches": int(round(launches_per_step * args.steps)),
        "e2e": ee, "cpu_baseline": cpu, "clocks": clk or None, "alu_peaks": alu,
        "kernels": [{"name": n, "launches": l, "ms": t} for n, l, t in main["census"]],
        "series": {"at_step": [i + 1 + warmup for i in step_idx],
                   "energy": [float(main["E"][i]) for i in step_idx],
                   "enstrophy": [float(main["O"][i]) for i in step_idx]},
        "companion": comp, "plain_unpruned": unpruned, "fft": fft, "large": large,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------- reference arm

def reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    mem = members(w)
    steps, dt, cores, warm = oracle_steps(mem, args.cpu_budget * 4, args.steps, args.warmup,
                                          warm_budget_s=args.cpu_budget)
    v = steps / dt
    unit = "run-steps/s" if len(mem[0]) > 1 else "steps/s"
    what = (f"members of the {len(mem[0])}-run ensemble (in turn)" if len(mem[0]) > 1 else
            f"the {'x'.join(str(d) for d in dims_of(w))} workload")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": unit,
            "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": steps, "warmup": warm,
            "ms_per_step": 1e3 * dt / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(args, w, int(os.environ.get("WORLD_SIZE", "1"))),
            "cpu_baseline": {"value": v, "unit": unit, "cores": cores, "kind": "oracle",
                             "sample": f"{steps} of {args.steps} RK2 steps of {what} "
                                       f"after {warm} untimed (warm-up bounded to "
                                       f"{args.cpu_budget:.0f} s, timed steps to "
                                       f"{args.cpu_budget * 4:.0f} s; at least one of each)"},
            "e2e": {"value": v, "unit": unit, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="forced512", choices=sorted(WORKLOADS))
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 1024^3 / 768^3 forms that ride along with forced512")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-companion", action="store_true")
    ap.add_argument("--no-unpruned", action="store_true",
                    help="skip the plain FP64 form with every transform line done")
    ap.add_argument("--no-fft", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--mode", default="step", choices=["step", "fft"],
                    help="fft: only the standalone 3-component r2c/c2r stage")
    ap.add_argument("--fft-n", type=int, default=256)
    ap.add_argument("--fft-prec", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--fft-dims", default=None,
                    help="NX,NY,NZ: the stage on that grid instead of --fft-n cubed")
    ap.add_argument("--fft-ncomp", type=int, default=3)
    ap.add_argument("--fft-window", action="store_true",
                    help="bracket one more r2c + c2r with cudaProfilerStart/Stop")
    ap.add_argument("--prec", default=None, choices=["fp32", "fp64"],
                    help="override the workload's headline form")
    ap.add_argument("--dealias", type=int, default=None, choices=[0, 1, 2],
                    help="override the dealiasing rule (0 cubic 2/3, 1 spherical 2/3, "
                         "2 phase shift with the sphere 9|k|^2 < 2N^2; Navier-Stokes runs)")
    args = ap.parse_args()
    w = dict(WORKLOADS[args.workload])
    w["name"] = args.workload
    if args.prec and args.prec != w["prec"]:
        w["prec"] = args.prec
        w["companion"] = None
    if args.dealias is not None:
        w["dealias"] = args.dealias
        w["desc"] += f", dealias rule {args.dealias}"
    if args.mode == "fft":
        import torch

        from paper_1003_4322_gb300 import _native as nat
        nat.load()
        peaks = load_peaks()
        size = tuple(int(x) for x in args.fft_dims.split(",")) if args.fft_dims else args.fft_n
        r = fft_stage(size, args.fft_prec, ncomp=args.fft_ncomp, window=args.fft_window)
        r["r2c_frac"] = r["r2c_gbs"] / peaks["hbm_gbs"]
        r["c2r_frac"] = r["c2r_gbs"] / peaks["hbm_gbs"]
        print(json.dumps(r), flush=True)
        return
    if args.impl == "reference":
        reference(args, w)
    else:
        ours(args, w)


if __name__ == "__main__":
    main()
