#!/usr/bin/env python
"""Benchmark of one moving-mesh MUSCL-Hancock update on GB300.

Workload: a 64^3 jittered lattice (+-0.2 spacing, seed 2) in a periodic unit
box, gamma = 5/3, rho = P = 1, a random-phase Gaussian velocity field with
P(k) ~ k^-4 on 2 <= k <= 8 at rms Mach 2, mesh generators moving with the
cells (Lagrangian); the Voronoi tessellation is built on the host before
timing.  One "step" is one pass of the whole hot path on the device:
gradients + limiter + Courant minimum, face velocities + fluxes (exact
Riemann), signed FP64 cell update + primitives + conservation sums, replayed
from a captured CUDA graph, with the time step kept on the device.

Metric: face-flux updates per second = faces x steps / device time.  The
headline value is the FP32 form (FP32 bulk, FP64 accumulation and sums);
the FP64 form is measured on the same workload and both are reported with
their error against the FP64 CPU oracle.  Between timed steps the state is
reset to the same input and the L2 is flushed (256 MiB write).

`--impl reference` times the FP64 CPU oracle instead (host cores, one
thread) on a sample of the same workload.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Voronoi face-flux updates/s on 1 GB300 (FP32/learned vs plain FP64, same error)"
UNIT = "face-flux updates/s"
CFL = 0.3
WORKLOAD = ("config-2 workload: 64^3 jittered lattice (+-0.2h, seed 2) in a periodic unit box, gamma=5/3, "
            "rho=P=1, Gaussian velocity field P(k)~k^-4 (2<=k<=8) at rms Mach 2, Lagrangian mesh motion, "
            "one MUSCL-Hancock step on the given tessellation")


def parse():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="amm", choices=["amm", "reference"])
    ap.add_argument("--n", type=int, default=64, help="lattice size per dimension")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline (profiling runs)")
    ap.add_argument("--no-extras", action="store_true", help="headline form only (profiling runs)")
    return ap.parse_args()


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


def source_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_0901_4107_gb300", "csrc")
    for fn in sorted(os.listdir(d)):
        if fn.endswith((".cu", ".cuh")):
            with open(os.path.join(d, fn), "rb") as f:
                h.update(fn.encode() + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, n, nf):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(p) as f:
            t = json.load(f)
    except Exception:
        return None
    if t.get("source_hash") != source_hash():
        return None
    k = t.get("kernels", {}).get(kernel)
    if not k:
        return None
    # scale by the units one launch processes if the capture was on another size
    return k["dram_bytes"] * (nf / k["faces"])


def algorithmic_bytes(kernel, n, nf, rb):
    """Bytes each kernel must move per launch (each array touched once; the
    gathered neighbour data counted once per cell).  rb = bytes of the bulk
    real type (4 FP32 form, 8 FP64 form)."""
    inc = 2 * nf                                  # cell->face incidences
    if kernel == "gradients":
        # W, P, cell geometry read; gradients written; CSR and offsets read;
        # face geometry (2 vectors of 4 reals) read once per face
        return n * (5 * rb + 4 * rb + 16 * rb + 4) + inc * 8 + nf * 8 * rb
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


def parity_errors(out, ref, Q0, W0, dim, gamma):
    import numpy as np
    fl = np.sqrt(np.mean(Q0 * Q0, axis=0))
    c = np.sqrt(gamma * W0[:, dim + 1] / W0[:, 0])
    fl[1:1 + dim] = np.sqrt(np.mean((Q0[:, 0] * c) ** 2))
    e = np.abs(out - ref) / np.maximum(np.abs(ref), fl)
    return float(e.max()), float(np.quantile(e, 0.999))


# ------------------------------------------------------------------ oracle arm
def oracle_rate(P, steps, budget_s=None):
    """Times full oracle steps (one host thread) of problem P; returns
    (faces/s, steps run, seconds, first-step output, its dt)."""
    from oracle import oracle as O
    M = O.Mesh(P.tess)
    geom = O.geometry(M)
    Q0 = P.conserved()
    t_all = 0.0
    first = None
    k = 0
    while k < steps:
        t0 = time.perf_counter()
        Qn, dt, cnt, rc = O.step(M, Q0, P.gamma, "lagrangian", cfl=CFL, geom=geom)
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
    # size the sample so warmup + steps stay within ~2 minutes of one core
    calib = ics.turbulent_3d(16, seed=2)
    r_cal, _, _, _ = oracle_rate(calib, 1)
    total = max(1, args.steps + args.warmup)
    faces_budget = 120.0 * r_cal / total
    n = int(max(8, min(args.n, round((faces_budget / 7.84) ** (1.0 / 3.0)))))
    P = ics.turbulent_3d(n, seed=2)
    if args.warmup:
        oracle_rate(P, args.warmup)
    rate, k, secs, _ = oracle_rate(P, args.steps)
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus, "steps": k,
        "warmup": args.warmup, "ms_per_step": 1e3 * secs / k, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_lattice": n, "cells": P.n_cells, "faces": P.n_faces},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "%d full oracle steps of the same recipe at %d^3 (%d faces)" % (k, n, P.n_faces)},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
def timed_form(amm, torch, ctx, Q0d, steps, warmup, stream, flush):
    """Event-timed steps of one context; state reset and L2 flushed between."""
    amm.amm_profile(ctx, True)
    for _ in range(warmup):
        amm.amm_set_state_device(ctx, Q0d.data_ptr())
        with torch.cuda.stream(stream):
            flush.fill_(1)
        amm.amm_advance(ctx, CFL, 1, True)
    torch.cuda.synchronize()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    kt = []
    t0 = time.perf_counter()
    for i in range(steps):
        amm.amm_set_state_device(ctx, Q0d.data_ptr())
        with torch.cuda.stream(stream):
            flush.fill_(i)
            ev0[i].record(stream)
        amm.amm_advance(ctx, CFL, 1, True)
        with torch.cuda.stream(stream):
            ev1[i].record(stream)
        kt.append(amm.amm_get_kernel_times(ctx))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    ker = {k: statistics.median([d[k] for d in kt]) for k in kt[0]}
    return ms, ker, wall


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    world, rank, local = dist_env()
    import numpy as np
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    from harness import ics
    from paper_0901_4107_gb300 import amm

    P = ics.turbulent_3d(args.n, seed=2 + rank)
    n, nf = P.n_cells, P.n_faces
    Q0 = P.conserved()
    stream = torch.cuda.Stream()
    Q0d = torch.from_numpy(Q0).to("cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device="cuda")   # 256 MiB
    torch.cuda.synchronize()

    def make(prec):
        return amm.create_from_mesh(P.tess, Q0, P.gamma, precision=prec, mesh_motion="lagrangian",
                                    stream=stream.cuda_stream)

    ctx32 = make("fp32")
    tuning = amm.amm_autotune(ctx32, CFL, reps=5)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.05)
    if world > 1:
        torch.distributed.barrier()
    ms32, ker32, wall32 = timed_form(amm, torch, ctx32, Q0d, args.steps, args.warmup, stream, flush)
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    step_ms = statistics.mean(ms32)
    if world > 1:
        t = torch.tensor([step_ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        step_ms = float(t.item())
        tot = torch.tensor([float(nf)], device="cuda")
        torch.distributed.all_reduce(tot)
        faces_all = float(tot.item())
    else:
        faces_all = float(nf)
    value = faces_all / (step_ms * 1e-3)

    hbm, peak_src = peaks()
    kern = {}
    for k, t in ker32.items():
        b = algorithmic_bytes(k, n, nf, 4)
        kern[k] = {"ms": t, "share": t / sum(ker32.values()), "algorithmic_bytes": b,
                   "gbs": (b / (t * 1e-3) / 1e9) if t > 0 else None}
    dom = max(ker32, key=lambda k: ker32[k])
    achieved = kern[dom]["gbs"]
    traffic = ncu_traffic(dom, n, nf)
    roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": traffic, "peak_source": peak_src + " hbm_gbs (copy bandwidth)",
            "algorithmic_bytes": kern[dom]["algorithmic_bytes"]}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": n, "faces": nf, "form": "fp32 (FP64 accumulation and sums)",
                   "l2": "flushed between timed steps (256 MiB write); state reset to the same input",
                   "graph": "one captured CUDA graph per step", "parallelism": "replicas" if world > 1 else "1 GPU",
                   "tuning": tuning},
        "cells_per_s": n * world / (step_ms * 1e-3),
        "roofline": roof,
        "kernels": kern,
        "gpu_launches": 4 * args.steps,
        "clocks": clocks,
    }
    if rank == 0 and not args.no_extras:
        from oracle import oracle as O
        forms = {"fp32": {"value": value, "ms_per_step": step_ms, "wall_s": wall32}}
        # FP64 form on the same workload
        ctx64 = make("fp64")
        amm.amm_autotune(ctx64, CFL, reps=2)
        k64 = max(3, min(args.steps, 200))
        ms64, ker64, wall64 = timed_form(amm, torch, ctx64, Q0d, k64, min(args.warmup, 5), stream, flush)
        forms["fp64"] = {"value": nf / (statistics.mean(ms64) * 1e-3), "ms_per_step": statistics.mean(ms64),
                         "steps": k64, "kernels_ms": ker64}
        # error of each form against the oracle on one step (oracle dt)
        if not args.no_cpu:
            rate, kcpu, secs, first = oracle_rate(P, 8, budget_s=12.0)
            ref, dt, geom = first
            M = O.Mesh(P.tess)
            W0 = O.primitives(M, Q0, geom[0], P.gamma)
            for name, ctx in (("fp32", ctx32), ("fp64", ctx64)):
                amm.amm_set_state(ctx, Q0)
                amm.amm_step(ctx, dt)
                emax, e999 = parity_errors(amm.amm_get_state(ctx), ref, Q0, W0, 3, P.gamma)
                forms[name].update({"err_max": emax, "err_p999": e999})
            line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": "%d full oracle steps of the workload (%d faces each), one host thread"
                                              % (kcpu, nf)}
        # FP32 learned form: proposal trained on the method's own face states
        # (harvested from the 2D shock tube and 3D turbulent boxes), then the
        # same timed loop
        from paper_0901_4107_gb300 import learned
        from harness import ics as _ics
        t_tr = time.perf_counter()
        net, tstats = learned.train_proposal(_ics, torch, small=False, epochs=4)
        tstats["train_seconds"] = time.perf_counter() - t_tr
        ctxl = make("fp32_learned")
        amm.amm_mlp_attach(ctxl, net)
        amm.amm_autotune(ctxl, CFL, reps=2)
        kl = max(3, min(args.steps, 500))
        msl, kerl, walll = timed_form(amm, torch, ctxl, Q0d, kl, min(args.warmup, 5), stream, flush)
        forms["fp32_learned"] = {"value": nf / (statistics.mean(msl) * 1e-3), "ms_per_step": statistics.mean(msl),
                                 "steps": kl, "kernels_ms": kerl, "training": tstats}
        # Newton iterations per face from the same input, each form
        for name, ctx in (("fp32", ctx32), ("fp32_learned", ctxl), ("fp64", ctx64)):
            amm.amm_set_state(ctx, Q0)
            amm.amm_reset_stats(ctx)
            amm.amm_advance(ctx, CFL, 1, False)
            s = amm.amm_get_stats(ctx)
            forms[name]["newton_iters_per_face"] = s["newton_iters"] / max(1, s["faces"])
            forms[name]["newton_hist"] = s["newton_hist"][:8]
        if not args.no_cpu:
            amm.amm_set_state(ctxl, Q0)
            amm.amm_step(ctxl, dt)
            emax, e999 = parity_errors(amm.amm_get_state(ctxl), ref, Q0, W0, 3, P.gamma)
            forms["fp32_learned"].update({"err_max": emax, "err_p999": e999})
        # end to end through the C ABI with pinned host buffers
        Qh = torch.from_numpy(Q0.copy()).pin_memory()
        Qo = torch.empty_like(Qh).pin_memory()
        ke = max(3, min(args.steps, 200))
        amm.amm_profile(ctx32, False)
        for _ in range(3):
            amm.amm_set_state(ctx32, Qh.numpy())
            amm.amm_advance(ctx32, CFL, 1, True)
            amm.amm_get_state(ctx32, Qo.numpy())
        t0 = time.perf_counter()
        for _ in range(ke):
            amm.amm_set_state(ctx32, Qh.numpy())
            amm.amm_advance(ctx32, CFL, 1, True)
            amm.amm_get_state(ctx32, Qo.numpy())
        e2e_s = (time.perf_counter() - t0) / ke
        line["e2e"] = {"value": nf / e2e_s, "unit": UNIT, "h2d_bytes_per_step": Q0.nbytes,
                       "d2h_bytes_per_step": Q0.nbytes, "ms_per_step": 1e3 * e2e_s, "steps": ke}
        line["forms"] = forms
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
