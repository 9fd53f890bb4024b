#!/usr/bin/env python
"""Benchmark of the moving-mesh MUSCL-Hancock update on GB300.

Default workload (lognormal192): a 192^3 jittered lattice (+-0.2 spacing,
seed 3, 7,077,888 cells, ~55.5 M faces) in a periodic unit box, gamma =
5/3, log-normal density (sigma_lnrho = 1), P = rho^(5/3), a random-phase
Gaussian velocity field with P(k) ~ k^-4 on 2 <= k <= 8 at rms Mach 3, a
static (Eulerian) mesh; the Voronoi tessellation is built on the host
before timing.  One "step" is one pass of the whole hot path on the device:
gradients + limiter + Courant minimum, fluxes (exact Riemann), signed cell
update + primitives + conservation sums, replayed from a captured CUDA
graph, with the time step kept on the device.

Metric: face-flux updates per second = faces x steps / device time.  The
headline value is the FP32 form (FP32 bulk, exact fixed-point flux sums,
FP64 state and sums); the plain FP64 form and the FP32 form with the learned
Riemann-pressure proposal are measured on the same workload, each with its
error against the FP64 CPU oracle after one step, and 20 steps on the fixed
tessellation compare the FP32 and FP64 forms.  The input (state, faces,
cells) exceeds the L2 many times over; between timed steps the state is
also reset to the same input and the L2 flushed (256 MiB write).

Other workloads (--workload), each printed as one line of the same shape:
  turbulent64   64^3 jittered lattice, gamma 5/3, rho = P = 1, the Gaussian
                velocity field at rms Mach 2, Lagrangian mesh motion; FP32,
                FP64 and learned forms, proposal-training throughput
  learned192    the turbulent field at 192^3 (Lagrangian): FP32 learned
                proposal vs the standard starting value, Newton iterations
  moving64      the whole moving-mesh step at 64^3 (drift and a new Voronoi
                mesh every step): on the device vs host-driven
  sedov64       the point explosion at 64^3 to t = 0.06: global steps vs
                individual power-of-two time steps, FP32 and FP64 forms,
                times to solution and face-flux counts
  ensemble      64 independent periodic boxes of 16^3..96^3 cells (log-
                uniform), Mach 0.5..4, Eulerian, per-box Courant step, 50
                steps, one persistent launch per step inside a CUDA graph

`--impl reference` times the FP64 CPU oracle instead (all host cores) on a
sample of the same workload.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Voronoi face-flux updates/s on 1 GB300 (FP32/learned vs plain FP64, same error)"
UNIT = "face-flux updates/s"
CFL = 0.3
FIELD = "Gaussian velocity field P(k)~k^-4 (2<=k<=8)"
WORKLOADS = {
    "turbulent64": ("config-2 workload: 64^3 jittered lattice (+-0.2h, seed 2) in a periodic unit box, gamma=5/3, "
                    "rho=P=1, " + FIELD + " at rms Mach 2, Lagrangian mesh motion, one MUSCL-Hancock step on the "
                    "given tessellation"),
    "lognormal192": ("config-3 workload: 192^3 jittered lattice (+-0.2h, seed 3), log-normal density sigma_lnrho=1 "
                     "(same spectrum), P=rho^(5/3), " + FIELD + " at rms Mach 3, gamma=5/3, stationary mesh; one "
                     "step and 20 steps on the fixed tessellation; FP32 headline, plain FP64 and FP32 + learned "
                     "p* proposal forms"),
    "learned192": ("config-4 workload: the config-2 field at 192^3 (jittered lattice +-0.2h, seed 2, rms Mach 2, "
                   "Lagrangian); FP32 flux with the learned p* proposal vs the standard starting value, Newton to "
                   "1e-6 relative in both"),
    "training": ("proposal-network training step: 2^20 face states harvested from one step of the config-2 workload "
                 "(64^3), BF16 tcgen05 forward and backward of the 6-64-64-1 SiLU network, gradient reduction, Adam"),
    "ensemble": ("config-5 workload: 64 independent periodic unit boxes, n^3 cells with n=round(exp(U(ln16,ln96))) "
                 "(seed 5), each the config-2 field at rms Mach U[0.5,4], gamma=5/3, stationary mesh, per-box "
                 "Courant step, entropy switch of Sec. 3.5 (Mach 1.1, alpha_S 0.01), 50 steps, each step one "
                 "CUDA-graph replay of either one persistent cooperative launch or the kernel sequence, whichever "
                 "the autotuner measures faster (config.step_mode; both timed in step_modes)"),
    "moving64": ("the moving-mesh cycle of Sec. 3 (Courant step, drift, MUSCL-Hancock update, new Voronoi mesh of "
                 "the moved generators) on the config-2 workload: 64^3 jittered lattice (+-0.2h, seed 2), rms Mach 2, "
                 "Lagrangian; the mesh built on the GPU (amm_retessellate) against the host tessellator and a new "
                 "context every step"),
    "sedov64": ("point explosion of Sec. 8.4: 64^3 Cartesian lattice in a periodic unit box, rho=1, P=1e-4, E=1 in "
                "the cell nearest the centre, gamma=5/3, static mesh, to t=0.06; global Courant steps vs one cycle "
                "of individual power-of-two time steps (Sec. 7.2, signal-speed criterion) per 0.01"),
}


def parse():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default 2000; ensemble 50)")
    ap.add_argument("--warmup", type=int, default=None, help="untimed warm-up steps (default 20; ensemble 5)")
    ap.add_argument("--impl", default="amm", choices=["amm", "reference"])
    ap.add_argument("--workload", default="lognormal192", choices=sorted(WORKLOADS))
    ap.add_argument("--n", type=int, default=None, help="lattice size per dimension (single-box workloads)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle legs")
    ap.add_argument("--no-extras", action="store_true", help="headline form only (profiling runs)")
    ap.add_argument("--form", default=None, choices=["fp32", "fp64", "fp32_learned"],
                    help="single-box workloads: the form timed as the headline (default: the workload's own)")
    ap.add_argument("--proposal-epochs", type=int, default=4, help="training epochs of the learned p* proposal")
    ap.add_argument("--individual-host-loop", action="store_true",
                    help="sedov64: launch each tick of the individual time steps from the host (for profilers "
                         "that cannot look inside graphs with conditional nodes)")
    ap.add_argument("--tuning", default=None,
                    help="fixed launch shapes grad_lanes,update_lanes,flux_block,persistent instead of autotuning")
    a = ap.parse_args()
    ens = a.workload == "ensemble"
    if a.steps is None:
        a.steps = 50 if ens else 2000
    if a.warmup is None:
        a.warmup = 5 if ens else 20
    if a.n is None:
        a.n = {"turbulent64": 64, "lognormal192": 192, "learned192": 192}.get(a.workload, 0)
    return a


# ------------------------------------------------------------------ helpers
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# the sources each profiled kernel is compiled from (its DRAM traffic in
# profiles/ncu_traffic.json and its FLOP counts in profiles/ncu_alu.json hold
# only while these are unchanged)
_COMMON = ["amm_internal.cuh", "hydro.cuh", "riemann.cuh", "hydro_f32.cu", "../../include/amm.h"]
KERNEL_SOURCES = {
    "gradients": _COMMON, "update": _COMMON,
    "flux": _COMMON + ["flux_chunks.cu", "learned.cuh"],
    "flux_fp64": ["amm_internal.cuh", "hydro.cuh", "riemann.cuh", "hydro_f64.cu", "../../include/amm.h"],
    "learned_flux": _COMMON + ["flux_chunks.cu", "flux_learned.cu", "learned.cuh", "tc.cuh", "persistent.cuh"],
}


def _code_only(text):
    """C/C++ source without comments, trailing blanks and blank lines: a
    change to comments alone leaves the kernel, and so the hash, unchanged."""
    out, i, n = [], 0, len(text)
    while i < n:
        if text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        elif text[i] == '"':
            j = i + 1
            while j < n and text[j] != '"':
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        else:
            out.append(text[i])
            i += 1
    lines = (l.rstrip() for l in "".join(out).split("\n"))
    return "\n".join(l for l in lines if l)


def source_hash(kernel):
    """Hash of the code (comments excluded) of the sources a kernel is built
    from: the committed ncu counters count only while it matches."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_0901_4107_gb300", "csrc")
    for fn in KERNEL_SOURCES[kernel]:
        with open(os.path.join(d, fn), encoding="utf-8") as f:
            h.update(fn.encode() + _code_only(f.read()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, nf):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the kernel's current sources (else None), scaled to this launch's faces."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(p) as f:
            k = json.load(f)["kernels"][kernel]
    except Exception:
        return None
    if kernel not in KERNEL_SOURCES or k.get("source_hash") != source_hash(kernel):
        return None
    return k["dram_bytes"] * (nf / k["faces"])


def ncu_flops(kernel, nf):
    """FP32 and FP64 FLOPs per launch counted by ncu on the kernel's current
    sources (fadd + fmul + 2 ffma, and the FP64 equivalents), scaled to this
    launch's faces; None when the counts were taken on other sources."""
    p = os.path.join(ROOT, "profiles", "ncu_alu.json")
    try:
        with open(p) as f:
            k = json.load(f)["kernels"][kernel]
    except Exception:
        return None
    if kernel not in KERNEL_SOURCES or k.get("source_hash") != source_hash(kernel):
        return None
    return {"fp32": k["fp32_flop"] * nf / k["faces"], "fp64": k["fp64_flop"] * nf / k["faces"],
            "case": k.get("case")}


def alu_peaks(amm, stream):
    """FP32 and FP64 fused multiply-add throughput of this device in TFLOP/s
    (FMA-chain probe, best of 3 launches of ~30-40 ms)."""
    out = {}
    for name, fp64, iters in (("fp32", 0, 1000000), ("fp64", 1, 20000)):
        amm.amm_alu_peak(fp64, max(1, iters // 50), stream)
        best = 0.0
        for _ in range(3):
            flop, ms = amm.amm_alu_peak(fp64, iters, stream)
            best = max(best, flop / (ms * 1e-3) / 1e12)
        out[name] = best
    return out


def alu_roofline(kernel, ms, nf, apk, pipe):
    """The flux kernel against the FMA pipe it computes on: counted FLOPs per
    launch over its event time, against the probe's rate."""
    f = ncu_flops(kernel, nf)
    out = {"kernel": kernel, "bound": "alu", "unit": "TFLOP/s", "pipe": pipe,
           "peak": apk.get(pipe) if apk else None, "peak_source": "FMA-chain probe in this run (amm_alu_peak)"}
    if f is None or not apk or not ms:
        out.update({"achieved": None, "frac": None, "note": "no ncu FLOP count for the current sources"})
        return out
    achieved = f[pipe] / (ms * 1e-3) / 1e12
    out.update({"achieved": achieved, "frac": achieved / apk[pipe], "flop_per_launch": f[pipe],
                "flop_source": "ncu thread-instruction counts of this kernel's sources (%s), scaled by faces"
                               % f["case"]})
    return out


def algorithmic_bytes(kernel, n, nf, rb, static=False):
    """Bytes each kernel must move per launch (each array touched once; the
    gathered neighbour data counted once per cell).  rb = bytes of the bulk
    real type (4 FP32 form, 8 FP64 form); static: a static mesh, whose
    gradient stage also runs the Courant pass and writes the predicted
    records."""
    inc = 2 * nf                                  # cell->face incidences
    if kernel == "gradients":
        # per cell: W, P, 1/V and R read, CSR offset, the gradients written;
        # per incidence: its precomputed record streamed (A c / |d|, A / |d|,
        # the lever arm and the neighbour index: 8 reals); the gathered
        # neighbour W, P counted once per cell.  Static mesh: W, P and R read
        # again by the Courant pass before the gradients, and the predicted
        # record ({rho, v}, {P, s - r}) written
        b = n * (5 * rb + 4 * rb + rb + 4 + 16 * rb) + n * 5 * rb + inc * (8 * rb)
        return b + (n * (6 * rb + 8 * rb) if static else 0)
    if kernel == "flux":
        # left/right indices and face geometry read; 5-component flux written;
        # per cell: W, P, gradients, cell geometry read once
        return nf * (8 + 8 * rb + 5 * rb) + n * (5 * rb + 16 * rb + 4 * rb)
    if kernel == "update":
        # CSR + offsets, each face flux read once, Q read+written (FP64),
        # V read (FP64), new W, P written
        return inc * 8 + nf * 5 * rb + n * (4 + 80 + 8 + 5 * rb)
    if kernel == "finish":
        return 0
    if kernel == "step":
        return sum(algorithmic_bytes(k, n, nf, rb, static) for k in ("gradients", "flux", "update"))
    raise KeyError(kernel)


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed loop runs."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.05)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        load = [r for r in rows if (num(r[9]) or 0) > 0] or rows
        sm = [num(r[1]) for r in load if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "samples_under_load": len(load),
                "power_w_max": max((num(r[3]) or 0) for r in rows)}


def floors(Q0, W0, dim, gamma):
    """Per-component error floor: RMS |Q| for mass and energy, RMS(m c) for
    the momentum components."""
    import numpy as np
    fl = np.sqrt(np.mean(Q0 * Q0, axis=0))
    c = np.sqrt(gamma * W0[:, dim + 1] / W0[:, 0])
    fl[1:1 + dim] = np.sqrt(np.mean((Q0[:, 0] * c) ** 2))
    return fl


def parity_errors(out, ref, fl):
    import numpy as np
    e = np.abs(out - ref) / np.maximum(np.abs(ref), fl)
    return float(e.max()), float(np.quantile(e, 0.999))


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu part", "hardware"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


# ------------------------------------------------------------------ oracle arm
def host_threads():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_rate(P, motion, steps, budget_s=None, threads=1):
    """Times full oracle steps of problem P on `threads` host threads; returns
    (faces/s, steps run, seconds, (first-step output, its dt, geometry))."""
    from oracle import oracle as O
    O.set_threads(threads)
    M = O.Mesh(P.tess)
    geom = O.geometry(M)
    Q0 = P.conserved()
    t_all = 0.0
    first = None
    k = 0
    while k < steps:
        t0 = time.perf_counter()
        Qn, dt, cnt, rc = O.step(M, Q0, P.gamma, motion, cfl=CFL, geom=geom)
        t_all += time.perf_counter() - t0
        if first is None:
            first = (Qn, dt, geom)
        k += 1
        if budget_s is not None and t_all >= budget_s:
            break
    return P.n_faces * k / t_all, k, t_all, first


def run_reference(args):
    world, rank, local = dist_env()
    if rank != 0:
        return 0
    from harness import ics
    # the oracle on all host cores; size the sample so warmup + steps stay
    # within ~2 minutes
    cores = host_threads()
    calib = ics.turbulent_3d(24, seed=2)
    r_cal, _, _, _ = oracle_rate(calib, "lagrangian", 2, threads=cores)
    total = max(1, args.steps + args.warmup)
    faces_budget = 120.0 * r_cal / total
    n_max = args.n if args.n else 64
    n = int(max(8, min(n_max, round((faces_budget / 7.84) ** (1.0 / 3.0)))))
    if args.workload == "lognormal192":
        P, motion = ics.lognormal_3d(n, seed=3), "eulerian"
    elif args.workload == "ensemble":
        P, motion = ics.turbulent_3d(n, seed=5, mach=2.25), "eulerian"
    elif args.workload == "sedov64":
        P, motion = ics.sedov(3, n), "eulerian"
    else:
        P, motion = ics.turbulent_3d(n, seed=2), "lagrangian"
    if args.workload == "moving64":
        # the moving-mesh step on the host: oracle update and a new host
        # tessellation of the moved generators every step
        from harness import moving
        from oracle import oracle as O
        O.set_threads(cores)
        if args.warmup:
            moving.run(P, moving.OracleBackend(O, "lagrangian"), steps=args.warmup, nthreads=cores)
        t0 = time.perf_counter()
        k = max(1, args.steps)
        moving.run(P, moving.OracleBackend(O, "lagrangian"), steps=k, nthreads=cores)
        secs = time.perf_counter() - t0
        rate = P.n_faces * k / secs
        sample = "%d oracle moving-mesh steps (update and host re-tessellation) at %d^3 (%d faces), %d host threads"
    else:
        if args.warmup:
            oracle_rate(P, motion, args.warmup, threads=cores)
        rate, k, secs, _ = oracle_rate(P, motion, args.steps, threads=cores)
        sample = "%d full oracle steps of the same recipe at %d^3 (%d faces), %d host threads"
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus, "steps": k,
        "warmup": args.warmup, "ms_per_step": 1e3 * secs / k, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "sample_lattice": n, "cells": P.n_cells,
                   "faces": P.n_faces},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
                         "sample": sample % (k, n, P.n_faces, cores)},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
class Gpu:
    """Device, stream, L2-flush buffer and the library, shared by the forms."""

    def __init__(self, local, epochs=4):
        import torch
        self.epochs = epochs
        self.torch = torch
        torch.cuda.set_device(local)
        import __graft_entry__
        __graft_entry__.build()
        from paper_0901_4107_gb300 import amm
        self.amm = amm
        self.stream = torch.cuda.Stream()
        self.flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device="cuda")   # 256 MiB > L2
        self.net = None
        self.train_stats = None
        self._alu = None

    def alu(self):
        if self._alu is None:
            self._alu = alu_peaks(self.amm, self.stream.cuda_stream)
        return self._alu

    def proposal(self):
        if self.net is None:
            from harness import ics
            from paper_0901_4107_gb300 import learned
            t0 = time.perf_counter()
            self.net, self.train_stats = learned.train_proposal(ics, self.torch, small=False, epochs=self.epochs)
            self.train_stats["train_seconds"] = time.perf_counter() - t0
        return self.net

    def tune(self, ctx, fixed, reps):
        if fixed:
            g, u, fb, p = (int(x) for x in fixed.split(","))
            self.amm.amm_set_tuning(ctx, g, u, fb, p)
            return self.amm.amm_get_tuning(ctx)
        return self.amm.amm_autotune(ctx, CFL, reps=reps)


def timed_form(g, ctx, Q0d, steps, warmup, kernel_steps=200):
    """Event-timed steps of one context; state reset and L2 flushed between.
    The timed steps replay the plain step graph; the per-kernel times come
    from a second pass whose graph also records events between the kernels.
    Returns per-step ms, per-kernel median ms and wall seconds."""
    amm, torch, stream = g.amm, g.torch, g.stream

    def one(i, before=None, after=None):
        amm.amm_set_state_device(ctx, Q0d.data_ptr())
        with torch.cuda.stream(stream):
            g.flush.fill_(i)
            if before is not None:
                before.record(stream)
        amm.amm_advance(ctx, CFL, 1, True)
        if after is not None:
            with torch.cuda.stream(stream):
                after.record(stream)

    amm.amm_profile(ctx, False)
    for i in range(warmup):
        one(i)
    torch.cuda.synchronize()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    t0 = time.perf_counter()
    for i in range(steps):
        one(i, ev0[i], ev1[i])
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    amm.amm_profile(ctx, True)
    kt = []
    for i in range(min(steps, kernel_steps) + 2):
        one(i)
        if i >= 2:
            kt.append(amm.amm_get_kernel_times(ctx))
    amm.amm_profile(ctx, False)
    ker = {k: statistics.median([d[k] for d in kt]) for k in kt[0]}
    return ms, ker, wall


def kernel_split(g, ctx, Q0d, tuning, steps=50):
    """Per-kernel device times of the chosen shapes.  A persistent step is one
    launch, so its phases are timed from the kernel sequence of the same
    shapes (same per-item code)."""
    amm = g.amm
    if not tuning["persistent"]:
        return None
    amm.amm_set_tuning(ctx, tuning["grad_lanes"], tuning["update_lanes"], tuning["flux_block"], 0)
    _, ker, _ = timed_form(g, ctx, Q0d, steps, 3)
    amm.amm_set_tuning(ctx, tuning["grad_lanes"], tuning["update_lanes"], tuning["flux_block"], 1)
    return ker


def kernel_table(ker, n, nf, rb, static=False):
    tot = sum(ker.values())
    out = {}
    for k, t in ker.items():
        b = algorithmic_bytes(k, n, nf, rb, static)
        out[k] = {"ms": t, "share": t / tot if tot else None, "algorithmic_bytes": b,
                  "gbs": (b / (t * 1e-3) / 1e9) if t > 0 else None}
    return out


def roofline(kern, nf, kernel_name_prefix=""):
    hbm, src = peaks()
    dom = max((k for k in kern if k != "finish"), key=lambda k: kern[k]["ms"])
    achieved = kern[dom]["gbs"]
    return {"kernel": kernel_name_prefix + dom, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": ncu_traffic(kernel_name_prefix + dom, nf),
            "peak_source": src + " hbm_gbs (copy bandwidth)", "algorithmic_bytes": kern[dom]["algorithmic_bytes"]}


def newton_stats(amm, ctx, Q0, steps=1):
    amm.amm_set_state(ctx, Q0)
    amm.amm_reset_stats(ctx)
    amm.amm_advance(ctx, CFL, steps, False)
    s = amm.amm_get_stats(ctx)
    return {"newton_iters_per_face": s["newton_iters"] / max(1, s["faces"]), "newton_hist": s["newton_hist"][:8],
            "fallback_faces": s["fallback_faces"], "vacuum_faces": s["vacuum_faces"], "guard_faces": s["guard_faces"]}


def e2e_rate(g, ctx, Q0, steps):
    """Whole-step rate through the C ABI with pinned host buffers: host->device
    state copy, one step, device->host state copy, every step."""
    amm, torch = g.amm, g.torch
    Qh = torch.from_numpy(Q0.copy()).pin_memory()
    Qo = torch.empty_like(Qh).pin_memory()
    amm.amm_profile(ctx, False)
    for _ in range(3):
        amm.amm_set_state(ctx, Qh.numpy())
        amm.amm_advance(ctx, CFL, 1, True)
        amm.amm_get_state(ctx, Qo.numpy())
    t0 = time.perf_counter()
    for _ in range(steps):
        amm.amm_set_state(ctx, Qh.numpy())
        amm.amm_advance(ctx, CFL, 1, True)
        amm.amm_get_state(ctx, Qo.numpy())
    return (time.perf_counter() - t0) / steps, Q0.nbytes


# algorithmic FLOPs per sample of one training step of the 6-64-64-1
# proposal network: forward 2(6*64 + 64*64 + 64), backward the three
# transposed products (dH1, dW2, dW1) plus the output layer
MLP_FLOP_FWD = 2 * (6 * 64 + 64 * 64 + 64)
MLP_FLOP_STEP = MLP_FLOP_FWD + 2 * (64 * 64 + 64 * 64 + 6 * 64 + 64)


def bench_training(g, P, motion, samples=1 << 20, reps=20, warmup=3):
    """Device time of one training step (tcgen05 forward + backward over a
    batch, gradient reduction, Adam) on `samples` harvested face states."""
    from paper_0901_4107_gb300 import learned
    amm, torch = g.amm, g.torch
    st = learned.harvest(P.tess, P.conserved(), P.gamma, motion, 1, torch=torch)
    x, t = learned.dataset(st, P.gamma, torch, gate=-1.0)      # every face: throughput only
    n = min(samples, x.shape[0])
    idx = torch.arange(n, dtype=torch.int32, device="cuda")
    net = amm.amm_mlp_create(P.gamma, g.stream.cuda_stream)
    amm.amm_mlp_set_params(net, learned.init_params(7))
    for _ in range(warmup):
        amm.amm_mlp_train_step(net, x.data_ptr(), t.data_ptr(), idx.data_ptr(), n, 1e-4)
    amm.amm_mlp_sync(net)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(g.stream):
        e0.record(g.stream)
    for _ in range(reps):
        amm.amm_mlp_train_step(net, x.data_ptr(), t.data_ptr(), idx.data_ptr(), n, 1e-4)
    with torch.cuda.stream(g.stream):
        e1.record(g.stream)
    amm.amm_mlp_sync(net)
    ms = e0.elapsed_time(e1) / reps
    bf16 = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16 = float(json.load(f)["bf16_tflops"])
    except Exception:
        pass
    tflops = MLP_FLOP_STEP * n / (ms * 1e-3) / 1e12
    return {"samples": n, "ms_per_step": ms, "samples_per_s": n / (ms * 1e-3),
            "algorithmic_flop_per_sample": MLP_FLOP_STEP, "achieved_tflops": tflops,
            "peak_tflops": bf16, "frac": (tflops / bf16) if bf16 else None,
            "peak_source": "measured bf16_tflops (burst)"}


def bench_train_workload(args, g, world, rank, local):
    """The proposal network's training step as its own workload (the dense
    contraction of the learned form): samples per second and BF16 tensor
    throughput against the measured peak."""
    from harness import ics
    P = ics.turbulent_3d(64, seed=2 + rank)
    sampler = ClockSampler(local)
    sampler.start()
    r = bench_training(g, P, "lagrangian", reps=args.steps, warmup=args.warmup)
    clocks = sampler.stop()
    rate = r["samples_per_s"] * world
    return {
        "metric": "proposal-network training samples/s on 1 GB300 (BF16 tcgen05 forward + backward + Adam)",
        "value": rate, "unit": "samples/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16", "data": "synthetic",
        "config": {"workload": WORKLOADS["training"], "batch": r["samples"]},
        "roofline": {"kernel": "training step", "bound": "tensor", "achieved": r["achieved_tflops"],
                     "peak": r["peak_tflops"], "unit": "TFLOP/s", "frac": r["frac"], "traffic": None,
                     "peak_source": r["peak_source"], "algorithmic_flop_per_sample": r["algorithmic_flop_per_sample"]},
        "gpu_launches": 4 * args.steps, "clocks": clocks,
    }


def bench_gated(g, n=48, mach=4.0, seed=9, steps=50, warmup=5, oracle_check=True):
    """The learned proposal where its gate fires often: a held-out turbulent
    box (a seed the training never saw) at high Mach number and modest
    resolution, Lagrangian.  FP32 with and without the proposal: faces/s of
    whole steps (CUDA graph, state reset and L2 flushed between steps),
    Newton iterations per face, the share of faces past the gate, and each
    form's error against the oracle after one step."""
    import numpy as np
    from harness import ics
    from paper_0901_4107_gb300 import learned
    amm, torch = g.amm, g.torch
    P = ics.turbulent_3d(n, seed=seed, mach=mach)
    Q0 = P.conserved()
    Q0d = torch.from_numpy(Q0).to("cuda")
    st = learned.harvest(P.tess, Q0, P.gamma, "lagrangian", 1, torch=torch)
    ratio = torch.empty(st.shape[0], dtype=torch.float32, device="cuda")
    x = torch.empty((st.shape[0], 6), dtype=torch.float32, device="cuda")
    amm.amm_mlp_features(P.gamma, st.shape[0], st.data_ptr(), x.data_ptr(), 0, 0, ratio.data_ptr())
    torch.cuda.synchronize()
    out = {"workload": "held-out turbulent box: %d^3 jittered lattice, seed %d (not in training), rms Mach %.1f, "
                       "gamma 5/3, Lagrangian" % (n, seed, mach),
           "faces": P.n_faces, "faces_past_gate": float((ratio > 1.25).float().mean().item())}
    ref = dt = fl = None
    if oracle_check:
        from oracle import oracle as O
        M = O.Mesh(P.tess)
        geom = O.geometry(M)
        ref, dt, _, _ = O.step(M, Q0, P.gamma, "lagrangian", cfl=CFL, geom=geom)
        fl = floors(Q0, O.primitives(M, Q0, geom[0], P.gamma), 3, P.gamma)
    for prec in ("fp32", "fp32_learned"):
        ctx = amm.create_from_mesh(P.tess, Q0, P.gamma, precision=prec, mesh_motion="lagrangian",
                                   stream=g.stream.cuda_stream)
        if prec == "fp32_learned":
            amm.amm_mlp_attach(ctx, g.proposal())
        t = g.tune(ctx, None, 3)
        # the kernel sequence (the learned form's deferred proposal kernel),
        # not the one-launch step the autotuner may prefer for a small box
        amm.amm_set_tuning(ctx, t["grad_lanes"], t["update_lanes"], t["flux_block"], 0)
        ms, ker, _ = timed_form(g, ctx, Q0d, steps, warmup, kernel_steps=20)
        r = {"value": P.n_faces / (statistics.mean(ms) * 1e-3), "ms_per_step": statistics.mean(ms),
             "flux_ms": ker.get("flux")}
        r.update(newton_stats(amm, ctx, Q0))
        if ref is not None:
            amm.amm_set_state(ctx, Q0)
            amm.amm_step(ctx, dt)
            r["err_max"], r["err_p999"] = parity_errors(amm.amm_get_state(ctx), ref, fl)
        out[prec] = r
        amm.amm_destroy(ctx)
    out["learned_vs_fp32"] = out["fp32_learned"]["value"] / out["fp32"]["value"]
    out["newton_iterations_saved_per_face"] = (out["fp32"]["newton_iters_per_face"] -
                                                out["fp32_learned"]["newton_iters_per_face"])
    return out


def bench_box(args, g, world, rank, local):
    """Single-box workloads: turbulent64, lognormal192, learned192."""
    import numpy as np
    from harness import ics
    amm, torch = g.amm, g.torch
    wl = args.workload
    if wl == "lognormal192":
        P, motion, head = ics.lognormal_3d(args.n, seed=3 + rank), "eulerian", "fp32"
    elif wl == "learned192":
        P, motion, head = ics.turbulent_3d(args.n, seed=2 + rank), "lagrangian", "fp32_learned"
    else:
        P, motion, head = ics.turbulent_3d(args.n, seed=2 + rank), "lagrangian", "fp32"
    default_head = head
    if args.form:
        head = args.form
    n, nf = P.n_cells, P.n_faces
    Q0 = P.conserved()
    Q0d = torch.from_numpy(Q0).to("cuda")
    torch.cuda.synchronize()

    def make(prec):
        ctx = amm.create_from_mesh(P.tess, Q0, P.gamma, precision=prec, mesh_motion=motion,
                                   stream=g.stream.cuda_stream)
        if prec == "fp32_learned":
            amm.amm_mlp_attach(ctx, g.proposal())
        return ctx

    ctxs = {head: make(head)}
    tuning = g.tune(ctxs[head], args.tuning, 5)
    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        torch.distributed.barrier()
    ms, ker, wall = timed_form(g, ctxs[head], Q0d, args.steps, args.warmup)
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    step_ms, faces_all = reduce_replicas(torch, statistics.mean(ms), nf, world, "cuda")
    value = faces_all / (step_ms * 1e-3)
    split = kernel_split(g, ctxs[head], Q0d, tuning)
    rb = 8 if head == "fp64" else 4
    kern = kernel_table(split or ker, n, nf, rb, motion == "eulerian")
    prefix = "learned_" if head == "fp32_learned" else ""
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if head == "fp64" else "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS[wl], "cells": n, "faces": nf,
                   "form": head + (" (FP64 throughout)" if head == "fp64" else
                                   (" (learned p* proposal, " if head == "fp32_learned" else " (")
                                   + "FP32 bulk, exact fixed-point flux sums, FP64 state and sums)"),
                   "l2": "flushed between timed steps (256 MiB write); state reset to the same input",
                   "graph": "one captured CUDA graph per step", "parallelism": "replicas" if world > 1 else "1 GPU",
                   "tuning": tuning},
        "cells_per_s": n * (faces_all / nf) / (step_ms * 1e-3),
        "roofline": roofline(kern, nf, prefix),
        "alu_roofline": (alu_roofline("flux_fp64", kern["flux"]["ms"], nf, g.alu(), "fp64") if head == "fp64" else
                         alu_roofline(prefix + "flux", kern["flux"]["ms"], nf, g.alu(), "fp32")),
        "alu_peaks_tflops": g.alu(),
        "kernels": kern,
        "kernel_times_from": "per-phase launches of the same shapes" if split else "the timed steps",
        "gpu_launches": (1 if tuning["persistent"] else 4) * args.steps,
        "clocks": clocks,
    }
    if rank != 0 or args.no_extras:
        return line
    from oracle import oracle as O
    forms = {head: {"value": value, "ms_per_step": step_ms, "wall_s": wall}}
    others = {"turbulent64": ("fp64", "fp32_learned"), "lognormal192": ("fp64", "fp32_learned"),
              "learned192": ("fp32", "fp64")}[wl]
    others = tuple(f for f in (default_head,) + others if f != head)
    for prec in others:
        ctxs[prec] = make(prec)
        g.tune(ctxs[prec], args.tuning, 2)
        # at most a few seconds of device time per extra form
        k = max(3, min(args.steps, 200 if prec == "fp64" else 500, int((4e8 if prec == "fp64" else 2e9) / nf)))
        msf, kerf, _ = timed_form(g, ctxs[prec], Q0d, k, min(args.warmup, 5))
        forms[prec] = {"value": nf / (statistics.mean(msf) * 1e-3), "ms_per_step": statistics.mean(msf),
                       "steps": k, "kernels_ms": kerf}
        if prec == "fp64":
            forms[prec]["alu_roofline"] = alu_roofline("flux_fp64", kerf["flux"], nf, g.alu(), "fp64")
        elif prec == "fp32":
            forms[prec]["alu_roofline"] = alu_roofline("flux", kerf["flux"], nf, g.alu(), "fp32")
    if "fp32_learned" in ctxs:
        forms["fp32_learned"]["training"] = g.train_stats
    for prec, ctx in ctxs.items():
        forms[prec].update(newton_stats(amm, ctx, Q0))
    if not args.no_cpu:
        # error of each form against the oracle on one step (oracle dt); the
        # oracle's own rate on a bounded sample is the CPU baseline
        cores = host_threads()
        rate, kcpu, secs, first = oracle_rate(P, motion, 8, budget_s=12.0, threads=cores)
        if P.n_cells <= 300000:
            rate1, kcpu1, _, _ = oracle_rate(P, motion, 8, budget_s=12.0, threads=1)
            sample1 = "%d full oracle step(s) of the workload, 1 host thread" % kcpu1
        else:
            # one thread on the whole 192^3 box would take ~30 s per step: a
            # 64^3 box of the same recipe stands in
            Ps = ics.lognormal_3d(64, seed=3) if wl == "lognormal192" else ics.turbulent_3d(64, seed=2)
            rate1, kcpu1, _, _ = oracle_rate(Ps, motion, 8, budget_s=8.0, threads=1)
            sample1 = "%d full oracle step(s) of a 64^3 box of the same recipe (%d faces), 1 host thread" % (
                kcpu1, Ps.n_faces)
        ref, dt, geom = first
        W0 = O.primitives(O.Mesh(P.tess), Q0, geom[0], P.gamma)
        fl = floors(Q0, W0, 3, P.gamma)
        for prec, ctx in ctxs.items():
            amm.amm_set_state(ctx, Q0)
            amm.amm_step(ctx, dt)
            emax, e999 = parity_errors(amm.amm_get_state(ctx), ref, fl)
            forms[prec].update({"err_max": emax, "err_p999": e999})
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
                                "sample": "%d full oracle step(s) of the workload (%d faces each), %d host threads"
                                          % (kcpu, nf, cores),
                                "one_thread": {"value": rate1, "steps": kcpu1, "sample": sample1}}
    if wl == "lognormal192":
        # 20 steps on the fixed tessellation, FP32 vs FP64 GPU forms
        res = {}
        for prec in ("fp32", "fp64"):
            ctx = ctxs[prec]
            amm.amm_set_state(ctx, Q0)
            t0 = amm.amm_get_totals(ctx)
            amm.amm_advance(ctx, CFL, 20, True)
            res[prec] = (amm.amm_get_state(ctx), amm.amm_get_totals(ctx), t0, amm.amm_get_box_status(ctx))
        c2 = P.gamma * (P.gamma - 1) * (Q0[:, 4] / Q0[:, 0] - 0.5 * (Q0[:, 1:4] ** 2).sum(1) / Q0[:, 0] ** 2)
        fl = np.sqrt(np.mean(Q0 * Q0, axis=0))
        fl[1:4] = np.sqrt(np.mean(Q0[:, 0] ** 2 * c2))
        emax, e999 = parity_errors(res["fp32"][0], res["fp64"][0], fl)
        mag = np.abs(Q0).sum(0)
        line["twenty_steps"] = {
            "fp32_vs_fp64_err_max": emax, "fp32_vs_fp64_err_p999": e999,
            "conservation_drift": {p: (np.abs(np.asarray(r[1]).ravel() - np.asarray(r[2]).ravel()) / mag).tolist()
                                   for p, r in res.items()},
            "box_status": {p: int(np.asarray(r[3]).max()) for p, r in res.items()}}
    if "fp64" in forms:
        for prec in forms:
            forms[prec]["vs_fp64"] = forms[prec]["value"] / forms["fp64"]["value"]
    if wl == "turbulent64":
        line["proposal_training"] = bench_training(g, P, motion)
    if "fp32_learned" in forms:
        # the learned proposal where its gate fires often (a held-out field)
        line["proposal_where_gated"] = bench_gated(g, oracle_check=not args.no_cpu)
    ke = max(3, min(args.steps, 200))
    e2e_s, nbytes = e2e_rate(g, ctxs[head], Q0, ke)
    line["e2e"] = {"value": nf / e2e_s, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                   "ms_per_step": 1e3 * e2e_s, "steps": ke}
    line["forms"] = forms
    return line


def bench_moving(args, g, world, rank, local):
    """Whole moving-mesh steps: everything on the device (one context,
    amm_retessellate after each drift) against the host-driven cycle (host
    tessellator, a new context per step); value = face-flux updates per
    second of the device cycle, whole step included."""
    from harness import ics, moving
    amm, torch = g.amm, g.torch
    n = args.n or 64
    P = ics.turbulent_3d(n, seed=2 + rank)
    nf = P.n_faces
    steps = max(3, min(args.steps, 20))
    res = {}
    sampler = ClockSampler(local)
    sampler.start()
    for prec in ("fp32", "fp64"):
        # the device cycle: one context (created once), then per step the
        # Courant step, drift, update and a new GPU mesh
        t0 = time.perf_counter()
        ctx = amm.create_from_mesh(P.tess, P.conserved(), P.gamma, precision=prec, mesh_motion="lagrangian")
        amm.amm_sync(ctx)
        create = time.perf_counter() - t0

        def device_step():
            dt = float(amm.amm_timestep(ctx, CFL)[0])
            amm.amm_drift(ctx, dt)
            amm.amm_step(ctx, dt)
            amm.amm_retessellate(ctx)
            return dt

        t = device_step()                                                   # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            t += device_step()
        amm.amm_sync(ctx)
        dev = (time.perf_counter() - t0) / steps
        amm.amm_destroy(ctx)
        kh = 2
        t0 = time.perf_counter()
        moving.run(P, moving.LibraryBackend(amm, prec, "lagrangian"), steps=kh)
        host = (time.perf_counter() - t0) / kh
        res[prec] = {"device_s_per_step": dev, "host_driven_s_per_step": host, "speedup": host / dev,
                     "steps": steps, "sim_time": t, "context_creation_s": create}
    # the parts of one device step (FP32): mesh, step
    ctx = amm.create_from_mesh(P.tess, P.conserved(), P.gamma, precision="fp32", mesh_motion="lagrangian")
    dt = float(amm.amm_timestep(ctx, CFL)[0])
    amm.amm_drift(ctx, dt)
    amm.amm_step(ctx, dt)
    amm.amm_sync(ctx)
    t0 = time.perf_counter()
    amm.amm_retessellate(ctx)
    res["fp32"]["retessellate_s"] = time.perf_counter() - t0
    gd = torch.from_numpy(amm.amm_get_generators(ctx)).to("cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tess = amm.amm_tess_build(3, P.n_cells, gd.data_ptr(), P.tess.box)
    torch.cuda.synchronize()
    res["fp32"]["tessellation_s"] = time.perf_counter() - t0
    del tess
    from harness.tess import tessellate
    t0 = time.perf_counter()
    tessellate(amm.amm_get_generators(ctx), P.tess.box)
    res["fp32"]["host_tessellation_s"] = time.perf_counter() - t0
    amm.amm_destroy(ctx)
    clocks = sampler.stop()
    dev = res["fp32"]["device_s_per_step"]
    return {
        "metric": METRIC, "value": nf / dev, "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": 1,
        "ms_per_step": 1e3 * dev, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOADS["moving64"], "cells": P.n_cells, "faces": nf,
                   "step": "Courant step, drift, update, GPU re-tessellation (wall clock, host loop; the "
                           "context is created once, before the timed steps)"},
        "cycle": res,
        "gpu_launches": None,
        "clocks": clocks,
    }


def bench_sedov(args, g, world, rank, local):
    """The point explosion to t = 0.06: global steps against individual time
    steps, FP32 and FP64 forms; value = face fluxes per second of the FP32
    individual-step run, with the times to solution beside it."""
    import numpy as np
    from harness import ics
    amm, torch = g.amm, g.torch
    n = args.n or 64
    t_end, cycles = 0.06, 6
    P = ics.sedov(3, n)
    Q0 = P.conserved()
    nf = P.n_faces

    def radius_err(Q):
        rho = Q[:, 0] / P.tess.volume
        d = P.tess.points - P.meta["centre"]
        d -= np.round(d)
        r = np.linalg.norm(d, axis=1)
        edges = np.arange(0.0, 0.8, 0.5 / n)
        idx = np.digitize(r, edges)
        prof = np.array([rho[idx == i].mean() if np.any(idx == i) else 0.0 for i in range(1, len(edges))])
        i = int(np.argmax(prof))
        return 0.5 * (edges[i] + edges[i + 1]) / ics.sedov_radius(t_end) - 1.0

    def run_global(ctx):
        amm.amm_set_state(ctx, Q0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t, k = 0.0, 0
        while t < t_end * (1 - 1e-14):
            dt = min(float(amm.amm_timestep(ctx, CFL)[0]), t_end - t)
            amm.amm_step(ctx, dt)
            t += dt
            k += 1
        amm.amm_sync(ctx)
        return time.perf_counter() - t0, {"steps": k, "face_fluxes": k * nf}

    def run_individual(ctx):
        amm.amm_set_state(ctx, Q0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tot = {"substeps": 0, "face_fluxes": 0, "activations": 0, "deepest_bin": 0}
        for _ in range(cycles):
            st = amm.amm_advance_individual(ctx, CFL, t_end / cycles, 30, True)
            for key in ("substeps", "face_fluxes", "activations"):
                tot[key] += st[key]
            tot["deepest_bin"] = max(tot["deepest_bin"], st["deepest_bin"])
        amm.amm_sync(ctx)
        return time.perf_counter() - t0, tot

    sampler = ClockSampler(local)
    sampler.start()
    res = {}
    for prec in ("fp32", "fp64"):
        ctx = amm.create_from_mesh(P.tess, Q0, P.gamma, precision=prec, mesh_motion="eulerian",
                                   stream=g.stream.cuda_stream)
        if args.individual_host_loop:
            amm.amm_individual_host_loop(ctx, True)
        amm.amm_advance_individual(ctx, CFL, t_end / cycles, 30, True)   # warm-up (setup, first launches)
        res[prec] = {}
        for name, fn in (("global", run_global), ("individual", run_individual)):
            wall, cnt = fn(ctx)
            cnt.update({"wall_s": wall, "radius_rel_err": radius_err(amm.amm_get_state(ctx))})
            res[prec][name] = cnt
        res[prec]["speedup"] = res[prec]["global"]["wall_s"] / res[prec]["individual"]["wall_s"]
        res[prec]["flux_ratio"] = res[prec]["global"]["face_fluxes"] / res[prec]["individual"]["face_fluxes"]
        amm.amm_destroy(ctx)
    clocks = sampler.stop()
    ind = res["fp32"]["individual"]
    value = ind["face_fluxes"] / ind["wall_s"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": cycles, "warmup": 1,
        "ms_per_step": 1e3 * ind["wall_s"] / cycles, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS["sedov64"], "cells": P.n_cells, "faces": nf,
                   "step": "one cycle of individual time steps of length 0.01: one CUDA graph whose while node "
                           "runs the ticks on the device" + (" (here: ticks launched from the host)"
                                                             if args.individual_host_loop else ""),
                   "l2": "inputs and working set exceed L2 only in part: whole runs timed, not single steps"},
        "time_to_solution": res,
        "gpu_launches": 8 * ind["substeps"],
        "clocks": clocks,
    }
    if rank == 0 and not args.no_cpu:
        from oracle import oracle as O
        cores = host_threads()
        O.set_threads(cores)
        M = O.Mesh(P.tess)
        V, s_ = O.geometry(M)
        t0 = time.perf_counter()
        Q, k = Q0, 0
        while k < 2:
            W = O.primitives(M, Q, V, P.gamma)
            dt = O.timestep(M, W, V, None, P.gamma, CFL)[0]
            Q, _, _, rc = O.step(M, Q, P.gamma, "eulerian", dt=dt, geom=(V, s_))
            k += 1
        secs = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": k * nf / secs, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "cpu": cpu_model(),
                                "sample": "2 global oracle steps of the 64^3 explosion, %d host threads" % cores}
    return line


def reduce_replicas(torch, step_ms, faces, world, device):
    """N replicas, one per rank: the job's step time is the slowest rank's and
    its work the sum of the ranks' faces (weak scaling).  Returns (step_ms,
    faces of all ranks)."""
    if world <= 1:
        return step_ms, float(faces)
    t = torch.tensor([step_ms, float(faces)], dtype=torch.float64, device=device)
    mx = t.clone()
    torch.distributed.all_reduce(mx, op=torch.distributed.ReduceOp.MAX)
    torch.distributed.all_reduce(t)
    return float(mx[0].item()), float(t[1].item())


def state_and_failures(amm, ctx):
    """The state even after a numeric failure, with what failed: the Newton
    solves that hit the iteration cap, the non-positive cells and the boxes
    whose status word is set."""
    import numpy as np
    Q = np.empty((ctx.n, ctx.dim + 2))
    amm.lib().amm_get_state(ctx.handle, Q.ctypes.data)
    st = amm.amm_get_stats(ctx)
    boxes = np.nonzero(np.asarray(amm.amm_get_box_status(ctx)))[0].tolist()
    return Q, {"newton_cap_faces": st["newton_fail"], "nonpositive_cells": st["nonpositive_cells"],
               "boxes_flagged": boxes}


def bench_ensemble(args, g, world, rank, local):
    """64 boxes of uneven size advanced together: each timed step is one
    ensemble step (every box one step, its own Courant dt) of a 50-step run
    from the initial state; the footprint is far above L2, so no flush."""
    import numpy as np
    from harness import ics
    from oracle import oracle as O
    amm, torch = g.amm, g.torch
    E = ics.concat(ics.ensemble(64, seed=5 + rank))
    n, nf, nb = E.n_cells, E.n_faces, len(E.problems)
    Q0d = torch.from_numpy(E.Q).to("cuda")

    def make(prec):
        opt = amm.amm_default_options(prec, "eulerian", stream=g.stream.cuda_stream, entropy=True)
        ctx = amm.amm_create(3, E.points, E.cells, E.shift, E.area, E.centroid, E.box, E.Q, E.gamma, opt,
                             box_cells=E.box_cells, box_faces=E.box_faces)
        if prec == "fp32_learned":
            amm.amm_mlp_attach(ctx, g.proposal())
        return ctx

    def run(ctx, steps, warmup, profile):
        amm.amm_profile(ctx, profile)
        amm.amm_set_state_device(ctx, Q0d.data_ptr())
        amm.amm_advance(ctx, CFL, warmup, True)
        amm.amm_set_state_device(ctx, Q0d.data_ptr())
        amm.amm_reset_stats(ctx)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        with torch.cuda.stream(g.stream):
            ev[0].record(g.stream)
        kt = []
        for i in range(steps):
            amm.amm_advance(ctx, CFL, 1, True)
            with torch.cuda.stream(g.stream):
                ev[i + 1].record(g.stream)
            if profile:
                kt.append(amm.amm_get_kernel_times(ctx))
        torch.cuda.synchronize()
        ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
        ker = {k: statistics.median([d[k] for d in kt]) for k in kt[0]} if kt else None
        return ms, ker

    head = "fp32_learned"
    ctxs = {head: make(head)}
    tuning = g.tune(ctxs[head], args.tuning, 3)
    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        torch.distributed.barrier()
    ms, _ = run(ctxs[head], args.steps, args.warmup, False)
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    status = amm.amm_get_box_status(ctxs[head])
    stats = amm.amm_get_stats(ctxs[head])
    head_final, head_failures = state_and_failures(amm, ctxs[head])
    # both step modes of the same shapes: one cooperative launch per step,
    # and the four-kernel sequence (the autotuner keeps the faster)
    modes = {}
    for pm in (0, 1):
        amm.amm_set_tuning(ctxs[head], tuning["grad_lanes"], tuning["update_lanes"], tuning["flux_block"], pm)
        msm, _ = run(ctxs[head], min(args.steps, 20), 2, False)
        modes["persistent" if pm else "kernel_sequence"] = {"ms_per_step": statistics.mean(msm),
                                                            "value": nf / (statistics.mean(msm) * 1e-3)}
    amm.amm_set_tuning(ctxs[head], tuning["grad_lanes"], tuning["update_lanes"], tuning["flux_block"],
                       tuning["persistent"])
    _, ker = run(ctxs[head], min(args.steps, 20), 2, True)
    step_ms, faces_all = reduce_replicas(torch, statistics.mean(ms), nf, world, "cuda")
    value = faces_all / (step_ms * 1e-3)
    # per-phase times of the same shapes for the roofline (a persistent step
    # is one launch)
    if tuning["persistent"]:
        amm.amm_set_tuning(ctxs[head], tuning["grad_lanes"], tuning["update_lanes"], tuning["flux_block"], 0)
        _, ker = run(ctxs[head], min(args.steps, 20), 2, True)
        amm.amm_set_tuning(ctxs[head], tuning["grad_lanes"], tuning["update_lanes"], tuning["flux_block"], 1)
    kern = kernel_table(ker, n, nf, 4, True)   # static mesh
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOADS["ensemble"], "boxes": nb, "cells": n, "faces": nf,
                   "box_cells_min_max": [int(np.diff(E.box_cells).min()), int(np.diff(E.box_cells).max())],
                   "form": "fp32_learned (learned p* proposal, FP32 bulk, exact fixed-point flux sums)",
                   "l2": "footprint far above L2 (no flush); consecutive steps of one run",
                   "graph": "one captured CUDA graph per step", "parallelism": "replicas" if world > 1 else "1 GPU",
                   "step_mode": ("one persistent cooperative launch per step" if tuning["persistent"] else
                                 "kernel sequence per step (gradients, fluxes, update, totals); the persistent "
                                 "single launch is slower here, see step_modes"),
                   "tuning": tuning},
        "cells_per_s": n * (faces_all / nf) / (step_ms * 1e-3),
        "roofline": roofline(kern, nf, "learned_"),
        "kernels": kern,
        "gpu_launches": (1 if tuning["persistent"] else 4) * args.steps,
        "clocks": clocks,
        "boxes_flagged": int((np.asarray(status) != 0).sum()),
        "step_modes": modes,
        "entropy_kept_per_cell_update": stats["entropy_kept"] / float(n * args.steps),
        "newton_iters_per_face": stats["newton_iters"] / max(1, stats["faces"]),
    }
    if rank != 0 or args.no_extras:
        return line
    forms = {head: {"value": value, "ms_per_step": step_ms, "newton_iters_per_face": line["newton_iters_per_face"],
                    "training": g.train_stats}}
    finals = {head: head_final}
    forms[head]["failures"] = head_failures
    for prec in ("fp32", "fp64"):
        ctxs[prec] = make(prec)
        tp = g.tune(ctxs[prec], args.tuning, 2)
        msf, _ = run(ctxs[prec], args.steps, 2, False)
        st = amm.amm_get_stats(ctxs[prec])
        forms[prec] = {"value": nf / (statistics.mean(msf) * 1e-3), "ms_per_step": statistics.mean(msf),
                       "tuning": tp, "newton_iters_per_face": st["newton_iters"] / max(1, st["faces"])}
        finals[prec], forms[prec]["failures"] = state_and_failures(amm, ctxs[prec])
    for prec in forms:
        forms[prec]["vs_fp64"] = forms[prec]["value"] / forms["fp64"]["value"]
    # after the whole run: FP32 forms against the FP64 GPU form, per box
    ref = finals["fp64"]
    errs = {}
    for prec in (head, "fp32"):
        worst, per_box = 0.0, []
        skip = set(forms[prec]["failures"]["boxes_flagged"]) | set(forms["fp64"]["failures"]["boxes_flagged"])
        for b, Pb in enumerate(E.problems):
            if b in skip:
                continue
            s = slice(E.box_cells[b], E.box_cells[b + 1])
            Qb = E.Q[s]
            c2 = Pb.gamma * (Pb.gamma - 1) * (Qb[:, 4] / Qb[:, 0] - 0.5 * (Qb[:, 1:4] ** 2).sum(1) / Qb[:, 0] ** 2)
            fl = np.sqrt(np.mean(Qb * Qb, axis=0))
            fl[1:4] = np.sqrt(np.mean(Qb[:, 0] ** 2 * c2))
            e = parity_errors(finals[prec][s], ref[s], fl)
            per_box.append(e[1])
            worst = max(worst, e[0])
        errs[prec] = {"max": worst, "median_box_p999": float(np.median(per_box)) if per_box else None,
                      "boxes_compared": len(per_box)}
    line["after_%d_steps_vs_fp64_gpu" % args.steps] = errs
    if not args.no_cpu:
        # one step of the smallest boxes against the oracle (its own dt per box)
        order = np.argsort(np.diff(E.box_cells))[:4]
        cores = host_threads()
        O.set_threads(cores)
        t_cpu, faces_cpu, worst = 0.0, 0, {p: 0.0 for p in ctxs}
        outs, kept, flips = {}, {}, {p: 0 for p in ctxs}
        for prec, ctx in ctxs.items():
            amm.amm_reset_stats(ctx)
            amm.amm_set_state(ctx, E.Q)
            amm.amm_advance(ctx, CFL, 1, False)
            outs[prec] = amm.amm_get_state(ctx)
            kept[prec] = amm.amm_get_entropy(ctx)[1]
        for b in order:
            Pb = E.problems[b]
            s = slice(E.box_cells[b], E.box_cells[b + 1])
            M = O.Mesh(Pb.tess)
            geom = O.geometry(M)
            S0 = O.entropy_init(M, E.Q[s], geom[0], Pb.gamma)
            t0 = time.perf_counter()
            refb, _, kb, dt, _, rc = O.step_entropy(M, E.Q[s], S0, Pb.gamma, "eulerian", cfl=CFL, geom=geom)
            t_cpu += time.perf_counter() - t0
            faces_cpu += Pb.n_faces
            W0 = O.primitives(M, E.Q[s], geom[0], Pb.gamma)
            fl = floors(E.Q[s], W0, 3, Pb.gamma)
            for prec in ctxs:
                # cells whose switch decision differs (a value within rounding
                # of its threshold) are counted, not compared
                kg = kept[prec][s]
                same = kg == kb
                flips[prec] += int((~same).sum())
                e = np.abs(outs[prec][s] - refb) / np.maximum(np.abs(refb), fl)
                worst[prec] = max(worst[prec], float(e[same].max()))
        for prec in ctxs:
            forms[prec]["err_max_first_step_sampled_boxes"] = worst[prec]
            forms[prec]["switch_decisions_differing_from_oracle"] = flips[prec]
        line["cpu_baseline"] = {"value": faces_cpu / t_cpu, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "cpu": cpu_model(),
                                "sample": "one oracle step of the %d smallest boxes (%d faces), %d host threads"
                                          % (len(order), faces_cpu, cores)}
    # end to end: host state in, 1 ensemble step, host state out
    ke = max(3, min(args.steps, 20))
    e2e_s, nbytes = e2e_rate(g, ctxs[head], E.Q, ke)
    line["e2e"] = {"value": nf / e2e_s, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                   "ms_per_step": 1e3 * e2e_s, "steps": ke}
    line["forms"] = forms
    return line


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    world, rank, local = dist_env()
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    g = Gpu(local, args.proposal_epochs)
    if args.workload == "ensemble":
        line = bench_ensemble(args, g, world, rank, local)
    elif args.workload == "training":
        line = bench_train_workload(args, g, world, rank, local)
    elif args.workload == "sedov64":
        line = bench_sedov(args, g, world, rank, local)
    elif args.workload == "moving64":
        line = bench_moving(args, g, world, rank, local)
    else:
        line = bench_box(args, g, world, rank, local)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
