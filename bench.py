#!/usr/bin/env python
"""Benchmark of the GB300 FFT-Galerkin strain-gradient crystal-plasticity
increment: the 64^3-voxel, 100-grain Cu polycrystal in uniaxial tension to 5 %
in 50 increments (strain rate 1e-3 /s), FP64 throughout.

One step = one strain increment (Nye curl and hardening, Newton-CG
equilibrium with the local update and tangent, commit).  Metric:
voxel-iterations/s = voxels x conjugate-gradient mat-vecs / time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one rank per GPU) every rank runs an independent
replica (the increment does not shard); value = all ranks' voxel-iterations /
max-over-ranks time.  --impl reference times the FP64 CPU oracle on the same
workload (a timed slice of its increment per step, see oracle_slice(); with
--full every step is one whole oracle increment).  --fft-compare times the
hand-written FFT against cuFFT.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import rvegen  # noqa: E402

WORKLOAD = "cu64"
FP64_PEAK_GFLOPS = 152 * 4 * 2.070   # 152 SMs x 2 DFMA (4 flop) per clock x 2.07 GHz = 1258.6
# The oracle's own mix of work: conjugate-gradient iterations per local
# evaluation (local update with tangent on every voxel).  Measured from whole
# oracle increments of the 64^3 / 100-grain Cu workload itself: increments 2-5
# (past the first increment's elastic-plastic transition, as the timed
# increments are) took 5319 CG iterations over 30 evaluations (177, 186, 176
# and 167 per evaluation).  A timed slice of the oracle keeps this mix, so that
# its voxel-iterations/s is the one its whole increments reach.
ORACLE_CG_PER_EVAL = 177.3


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=47)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--graphs", type=int, default=1, choices=[0, 1],
                    help="replay chunks of CG iterations as captured CUDA graphs")
    ap.add_argument("--autotune", type=int, default=None, choices=[0, 1],
                    help="time candidate launch shapes at create (default: on for the sweep, off otherwise)")
    ap.add_argument("--sensitivity", action="store_true",
                    help="time the increments with and without d<P>/d(tau0, K, alpha, b) and report the ratio")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(rvegen.WORKLOADS) + ["sweep", "convergence"],
                    help="sweep: the 16-RVE grain-size sweep stepped together (rve_step_batch), with the "
                         "Hall-Petch fit; convergence: the grid and realisation study of the flow stress")
    ap.add_argument("--precision", default="f64", choices=["f64", "mixed"],
                    help="mixed: FP32 conjugate gradients with FP64 local update and residual")
    ap.add_argument("--full", action="store_true",
                    help="with --impl reference: every step is one whole oracle increment (no slice)")
    ap.add_argument("--fft-compare", action="store_true",
                    help="time the hand-written FFT against cuFFT (3 and 9 fields, 64^3 and 128^3, FP64 and FP32)")
    return ap.parse_args(argv)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ---------------------------------------------------------------- roofline
# FP64 operations of the local update, counted from the kernels' arithmetic
# (an FMA counts 2; constant Schmid-tensor entries 0 and +-1 folded).  k_local:
# per voxel set-up (frame rotation, trial elastic state) and P at the
# converged S (six 3x3 products), per residual evaluation, per Newton
# iteration (Jacobian with the stiffness applied once per column of the
# accumulated sum, LU, solve).  k_tangent: per voxel set-up, one evaluation,
# Jacobian and LU, the intermediate products, the strain-linear response to
# each of the six unit strains (solve, Schmid sum, five 3x3 products, F~ dQ)
# and the nine directions of dP/dF (Fe^T a and Fp^-T b, dE, H dE, the
# rank-one term and the rotation).  The k_tangent total, 7744, agrees with
# the FP64 operations ncu counts for the kernel (7771 per voxel).
CONST_SETUP, CONST_EVAL, CONST_ITER = 180.0 + 270.0, 500.0, 1442.0
TANGENT_FLOPS = 180.0 + 500.0 + 1230.0 + 146.0 + 180.0 + 6 * 522.0 + 9 * 264.0
CONST_BYTES = 364 + 216        # reads F, dF, Fp^-1, tauc, S, grain; writes S, dgam, P
TANGENT_BYTES = 364 + 648      # reads F, dF, Fp^-1, tauc, S, grain; writes K


def fft_models(n0, n1, n2, nf):
    """Algorithmic FP64 flops and bytes of one launch of each FFT pass over nf
    real fields (2.5 N log2 N per real and 5 N log2 N per complex transform;
    6 flops per spectrum value for the operator between the z passes)."""
    nvox = n0 * n1 * n2
    nkx = n0 // 2 + 1
    nspec = nkx * n1 * n2
    lg = math.log2
    fx = nf * n2 * n1 * 2.5 * n0 * lg(n0)
    fy = nf * n2 * nkx * 5.0 * n1 * lg(n1)
    fz = nf * nkx * n1 * 2 * 5.0 * n2 * lg(n2) + nf * nspec * 6.0
    return {"x": (fx, nf * nvox * 8 + nf * nspec * 16), "y": (fy, 2 * nf * nspec * 16),
            "z": (fz, 2 * nf * nspec * 16)}


def kernel_models(n0, n1, n2, local=None):
    """Algorithmic FP64 flops and bytes per launch of each kernel category.
    The fft_* categories count the three-field transforms of the projection
    (the CG loop, the residual); fft_curl counts all five passes of the
    nine-field Nye-curl transform, so its per-launch figure is a fifth of one
    curl.  `local` = (launches, local iterations, local evaluations) of the
    local update in the timed region, for its per-launch average."""
    nvox = n0 * n1 * n2
    f3 = fft_models(n0, n1, n2, 3)
    f9 = fft_models(n0, n1, n2, 9)
    # one curl = x, y, z (with the operator), y^-1, x^-1 passes over nine fields
    curl = [(2 * f9["x"][i] + 2 * f9["y"][i] + f9["z"][i]) / 5 for i in (0, 1)]
    return {
        "fft_x_r2c": f3["x"],
        "fft_y": f3["y"],
        "fft_y_inv": f3["y"],
        "fft_z_op": f3["z"],
        "fft_x_c2r": f3["x"],
        "fft_curl": (curl[0], curl[1]),
        "tangent_apply": (nvox * (162 + 18 + 18), nvox * (81 + 9 + 9 + 9 + 9) * 8),
        # divergence 9 -> 3 fields applied separably: per field a z pair, a y
        # pair and the x step (30 additions), and the means of the stress-
        # controlled components (5 under uniaxial tension)
        "stencil": (nvox * (30 + 5), nvox * (9 + 3) * 8),
        # gradient 3 -> 9 applied separably (per potential a z pair and
        # difference, three y sums, three x steps: 24 additions), the zero-mode
        # offsets of the stress-controlled components (5), and the fused
        # x += alpha p, r -= alpha q, r . r (27 FMA)
        "cg_update": (nvox * (24 + 5 + 27 * 2), nvox * (3 + 9 * 5) * 8),
        "tangent_build": (nvox * TANGENT_FLOPS, nvox * TANGENT_BYTES),
    } | ({"constitutive": ((local[0] * nvox * CONST_SETUP + local[1] * CONST_ITER
                            + local[2] * CONST_EVAL) / local[0], nvox * CONST_BYTES)}
         if local and local[0] else {})


# the FP32 conjugate-gradient kernels of the mixed path: half the bytes of the
# FP64 model, and their FP32 arithmetic is far below the FP32 peak, so HBM binds
FP32_CG = ("tangent_apply", "stencil", "cg_update", "fft_x_r2c", "fft_y", "fft_y_inv", "fft_z_op", "fft_x_c2r")



def rate(flops, nbytes, avg_s, peaks):
    """The bound of one launch (FP64 ALU or HBM, whichever needs more time at
    the peaks) and its achieved fraction of that bound."""
    t_alu = flops / (FP64_PEAK_GFLOPS * 1e9)
    t_hbm = nbytes / (peaks["hbm_gbs"] * 1e9)
    if t_alu >= t_hbm:
        ach = flops / avg_s / 1e9
        return dict(bound="alu", achieved=ach, peak=FP64_PEAK_GFLOPS, unit="GFLOP/s (FP64)",
                    frac=ach / FP64_PEAK_GFLOPS)
    ach = nbytes / avg_s / 1e9
    return dict(bound="hbm", achieved=ach, peak=peaks["hbm_gbs"], unit="GB/s", frac=ach / peaks["hbm_gbs"])


def roofline_all(stats, shape, peaks, local=None, prec=0):
    """Every timed category: launches, average launch time, share of kernel
    time, and its roofline fraction (algorithmic figures per launch over the
    event-timed average launch duration)."""
    models = kernel_models(*shape, local=local)
    if prec == 1:
        for k in FP32_CG:
            models[k] = (0.0, models[k][1] / 2)
    timed = {k: v for k, v in stats.items() if v[0] > 0 and v[1] > 0}
    total = sum(v[1] for v in timed.values())
    out = {}
    for k, (n, ms) in timed.items():
        avg_s = ms / n / 1e3
        e = {"launches": n, "avg_us": avg_s * 1e6, "share": ms / total}
        if k in models:
            flops, nbytes = models[k]
            e.update(rate(flops, nbytes, avg_s, peaks))
            e["algorithmic_flops"] = flops
            e["algorithmic_bytes"] = nbytes
        out[k] = e
    return out


def roofline(stats, shape, peaks, local=None, prec=0):
    """(dominant category by event time, its entry of roofline_all)."""
    allr = roofline_all(stats, shape, peaks, local=local, prec=prec)
    if not allr:
        return None, None
    dom = max(allr, key=lambda k: allr[k]["share"])
    return dom, allr[dom]


def measured_fp64_peak(smi_index):
    """The device's FP64 FMA rate, timed live (libbench_aux: chains of
    independent DFMA, 4 blocks of 256 threads per SM, best of 10 launches of
    about 20 ms), with the SM clock sampled meanwhile."""
    import ctypes
    from paper_1910_01946_gb300 import _build
    try:
        lib = ctypes.CDLL(_build.build_aux())
    except (OSError, RuntimeError):
        return None
    lib.aux_fp64_peak.restype = ctypes.c_int
    lib.aux_fp64_peak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double)]
    clocks = ClockSampler(smi_index)
    clocks.start()
    time.sleep(0.25)
    g, ms = ctypes.c_double(), ctypes.c_double()
    rc = lib.aux_fp64_peak(4, 8000, 10, ctypes.byref(g), ctypes.byref(ms))
    time.sleep(0.1)
    clocks.stop()
    if rc != 0:
        return None
    c = clocks.summary()
    return {"gflops": g.value, "launch_ms": ms.value, "sm_mhz": c["sm_mhz"], "samples": c["samples"],
            "how": "DFMA chains, 8 per thread, 4 x 256 threads per SM, best of 10 launches (libbench_aux)"}


def mixed_accuracy(pkg, rve, wl, gid, quat, mat, dev, a, P_hist):
    """The mixed-precision run against the FP64 path on the same increments:
    an FP64 handle steps through the warm-up and timed increments; the
    largest relative error of the macroscopic stress <P> over the timed
    increments, and of the per-voxel Cauchy stress and GND densities of the
    last increment (max |mixed - fp64| / max |fp64| over the field)."""
    mask = rvegen.UNIAXIAL_X_MASK
    ref = pkg.RVE(gid, quat, mat, wl.edge, device=dev, precision=0, own_stream=True, graphs=a.graphs)
    try:
        for _ in range(a.warmup):
            ref.step(wl.dFbar(), mask, np.zeros(9), wl.dt)
        perr = 0.0
        for k in range(a.steps):
            ref.step(wl.dFbar(), mask, np.zeros(9), wl.dt)
            Pr = ref.macro_stress()[0]
            perr = max(perr, float(np.abs(P_hist[k] - Pr).max() / np.abs(Pr).max()))
        out = {"macro_P_rel_err_max": perr}
        for name in ("SIGMA", "RHO_GND"):
            f, r = rve.field(name), ref.field(name)
            out[f"{name.lower()}_rel_err_max"] = float(np.abs(f - r).max() / np.abs(r).max())
        out["how"] = (f"FP64 handle stepped through the same {a.warmup} + {a.steps} increments; <P> compared at "
                      "every timed increment, sigma and rho_GND fields at the last")
        return out
    finally:
        ref.close()


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# kernels that lead the timed region, from one ncu capture of the 64^3
# workload; keyed by (category, precision).  Kernels changed since that
# capture have no entry (reported as null), as do other grid sizes.
TRAFFIC_SOURCE = "profiles/kernels_cu64.md"
TRAFFIC_64 = {
    ("tangent_apply", 0): 207.66e6 + 5.11e6,   # K : p reads its algorithmic 207.6 MB
    ("tangent_apply", 1): 103.84e6 + 3.36e6,   # TMA-staged FP32 apply (float K, r, p)
    ("constitutive", 0): 97.20e6 + 30.14e6,    # k_local (the same kernel in both precisions)
    ("constitutive", 1): 97.20e6 + 30.14e6,
    ("tangent_build", 0): 77.53e6 + 149.33e6,  # k_tangent, K written in FP64
    ("stencil", 0): 18.94e6,                   # k_div_rows (its writes stay in L2)
    ("stencil", 1): 9.49e6,                    # k_div_rows<float>
    ("cg_update", 0): 62.96e6 + 0.16e6,        # k_grad_rows<true>
    ("cg_update", 1): 31.49e6,                 # k_grad_rows<true, float>
}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d.get("hbm_gbs", 6800.0), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


# ---------------------------------------------------------------- CPU oracle
_ORACLE_CACHE = {}


def oracle_slice(wl, n_cg, seed=0):
    """A bounded slice of the FP64 CPU oracle's increment on the full
    workload, timed for real (wall clock on the host cores): the local update
    with tangent on a seeded subset of the voxels (whole grains, the last one
    cut to size) holding n_cg / ORACLE_CG_PER_EVAL of them, then n_cg
    conjugate-gradient iterations on the full grid.  The slice keeps the
    oracle's own mix of the two, so its rate nvox * n_cg / seconds is the
    voxel-iterations/s of the oracle's whole increments.  Two steps of the
    slice are its own scaffolding and run off the clock: tiling the subset's
    tangent over the grid, and the residual projection that starts the CG
    (a whole increment projects one residual per local evaluation, about 1 %
    of an evaluation's time).  The hardening (once per increment) is set up
    before the clock starts.  Returns (seconds, voxels evaluated, n_cg)."""
    from oracle import solver
    from oracle import spectral as sp
    key = wl.name
    if key not in _ORACLE_CACHE:
        gid, quat, mat = wl.inputs()
        o = solver.RVE(gid, quat, mat, wl.edge)
        _ORACLE_CACHE[key] = (o, o.hardening(), list(o.grains))
    o, (tauc, ell), grains = _ORACLE_CACHE[key]
    nv = o.F.shape[0]
    F = o.F + (wl.dFbar() * rvegen.UNIAXIAL_X_MASK).reshape(3, 3)
    rng = np.random.default_rng(seed)
    need = max(1, int(round(nv * n_cg / ORACLE_CG_PER_EVAL)))
    chosen, count = [], 0
    for gi in rng.permutation(len(grains)):
        if count >= need:
            break
        g = grains[gi]
        take = min(len(g["idx"]), need - count)
        chosen.append(g if take == len(g["idx"]) else dict(g, idx=g["idx"][:take]))
        count += take
    idx = np.concatenate([g["idx"] for g in chosen])
    o.opts.max_cg = n_cg
    o.opts.cg_tol = 1e-300
    o.grains = chosen
    try:
        t0 = time.perf_counter()
        P, K, S, M, dg, lit, lf = o.constitutive(F, tauc, o.S, wl.dt)
        t_local = time.perf_counter() - t0
    finally:
        o.grains = grains
    Kfull = np.resize(K[idx], (nv, 3, 3, 3, 3))
    R = o.flat(sp.project(o.field(np.resize(P[idx], (nv, 3, 3))), rvegen.UNIAXIAL_X_MASK, o.h))
    t0 = time.perf_counter()
    o.cg(Kfull, -R, rvegen.UNIAXIAL_X_MASK)
    t_cg = time.perf_counter() - t0
    return t_local + t_cg, len(idx), n_cg


def oracle_increments(wl, warmup, steps):
    """Whole increments of the FP64 CPU oracle, each timed for real: `warmup`
    untimed increments, then `steps` timed ones.  Returns (seconds of each
    timed increment, CG iterations of each, local evaluations of each)."""
    from oracle import solver
    gid, quat, mat = wl.inputs()
    o = solver.RVE(gid, quat, mat, wl.edge)
    n_eval = [0]
    evaluate = o.constitutive

    def counted(*args, **kw):
        n_eval[0] += 1
        return evaluate(*args, **kw)
    o.constitutive = counted
    secs, cgs, evals = [], [], []
    for k in range(warmup + steps):
        n_eval[0] = 0
        t0 = time.perf_counter()
        info = o.step(wl.dFbar(), rvegen.UNIAXIAL_X_MASK, np.zeros(9), wl.dt)
        el = time.perf_counter() - t0
        if not info.converged:
            raise RuntimeError(f"oracle increment {k} did not converge")
        if k >= warmup:
            secs.append(el)
            cgs.append(int(sum(info.cg_iters)))
            evals.append(n_eval[0])
    return secs, cgs, evals


def reduce_over_ranks(ms, units, device="cpu"):
    """Replicas: the job's time is the slowest rank's, its work the sum of all
    ranks' (weak scaling, no data exchange between ranks).  Returns
    (max ms, total units); a single process returns its own values."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(units)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------- main
def run_sensitivity(a):
    """Cost of the forward-mode sensitivities: the same increments timed with
    and without d<P>/d theta (one extra linear solve per parameter and
    increment), device-synchronised on both sides."""
    import torch
    import paper_1910_01946_gb300 as pkg
    from paper_1910_01946_gb300 import _build
    _build.build()
    pkg.load_library()
    prec = 1 if a.precision == "mixed" else 0
    wl = rvegen.WORKLOADS[a.workload]
    gid, quat, mat = wl.inputs()
    mask = rvegen.UNIAXIAL_X_MASK
    out = {}
    clocks = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
    clocks.start()
    for sens in (False, True):
        r = pkg.RVE(gid, quat, mat, wl.edge, own_stream=True, precision=prec, graphs=a.graphs)
        if sens:
            r.enable_sensitivity()
        for _ in range(a.warmup):
            r.step(wl.dFbar(), mask, np.zeros(9), wl.dt)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(r.stream)
        cg = 0
        for _ in range(a.steps):
            cg += r.step(wl.dFbar(), mask, np.zeros(9), wl.dt)["cg_iters_total"]
        ev1.record(r.stream)
        torch.cuda.synchronize()
        out[sens] = (ev0.elapsed_time(ev1) / a.steps, cg / a.steps,
                     r.stress_sensitivity()[:, 0, 0].tolist() if sens else None)
        r.close()
    clocks.stop()
    line = {"metric": "sensitivity cost: increment with d<P>/d(tau0, K, alpha, b) / increment alone",
            "value": out[True][0] / out[False][0], "unit": "x", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": out[True][0], "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == 0 else "f64 local update and residual, f32 conjugate gradients",
            "data": "synthetic",
            "config": {"workload": f"{wl.name}: {wl.n}^3 voxels, {wl.n_grains} grains, {wl.material}, "
                                   f"tension {wl.strain:.0%} in {wl.increments} increments, sensitivities to "
                                   "(tau0, K, alpha, b)", "voxels": wl.n ** 3},
            "clocks": clocks.summary(),
            "detail": {"ms_per_increment_forward": out[False][0], "ms_per_increment_with_sensitivities": out[True][0],
                       "newton_cg_iters_per_increment": out[False][1],
                       "dP11_dtheta_last_increment": out[True][2]}}
    print(json.dumps(line))


def run_sweep(a):
    """The batched grain-size sweep: 16 RVEs (32^3 .. 96^3, 8 .. 400 grains,
    Cu/Al/Ag/Ni) advanced together, each on its own stream.  Throughput is
    the sum over RVEs of voxels x CG iterations over the wall time of the
    batched increments (device synchronised on both sides)."""
    import torch
    import paper_1910_01946_gb300 as pkg
    from paper_1910_01946_gb300 import _build
    _build.build()
    pkg.load_library()
    prec = 1 if a.precision == "mixed" else 0
    wls = rvegen.sweep_workloads()
    rves = []
    for w in wls:
        gid, quat, mat = w.inputs()
        rves.append(pkg.RVE(gid, quat, mat, w.edge, own_stream=True, precision=prec, graphs=a.graphs,
                            autotune=1 if a.autotune is None else a.autotune))
    mask = rvegen.UNIAXIAL_X_MASK
    dF = [w.dFbar() for w in wls]
    dts = [w.dt for w in wls]
    curves = [[] for _ in wls]            # sigma_11 after every increment (host copies, no device work)

    def record():
        for c, r in zip(curves, rves):
            c.append(float(r.macro_stress()[1][0, 0]))

    for k in range(a.warmup):
        try:
            pkg.step_batch(rves, dF, mask, np.zeros(9), dts)
        except pkg.RVEError as e:
            print(json.dumps({"metric": "voxel-iterations/s", "error": f"warm-up increment {k}: {e}"}))
            raise
        record()
    for r in rves:
        r.profile(False)                 # reset the launch counters; no per-kernel events in the timed region
    torch.cuda.synchronize()
    clocks = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
    clocks.start()
    time.sleep(0.3)
    t0 = time.perf_counter()
    work, cg = 0.0, 0
    for k in range(a.steps):
        try:
            infos = pkg.step_batch(rves, dF, mask, np.zeros(9), dts)
        except pkg.RVEError as e:
            print(json.dumps({"metric": "voxel-iterations/s", "error": f"timed increment {k}: {e}"}))
            raise
        for w, i in zip(wls, infos):
            work += w.n ** 3 * i["cg_iters_total"]
            cg += i["cg_iters_total"]
        record()
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    clocks.stop()
    launches = sum(sum(v[0] for v in r.kernel_stats().values()) for r in rves)
    shapes = [r.tuning() for r in rves]
    for r in rves:
        r.close()
    rves = []
    torch.cuda.empty_cache()
    # Hall-Petch analysis (Sec. 3, Eq. SizeEffect2): the same sixteen RVEs with
    # the GND densities switched off give sigma_inf, the size-independent flow
    # stress of the same microstructure ("infinite grain size"), after the
    # same increments; per material the four grain sizes give C and x
    nsteps = a.warmup + a.steps
    inf_curves = [[] for _ in wls]
    base = []
    for w in wls:
        gid, quat, mat = w.inputs()
        mat.gnd_enabled = False
        base.append(pkg.RVE(gid, quat, mat, w.edge, own_stream=True, precision=prec, graphs=a.graphs))
    hp_error = None
    try:
        for k in range(nsteps):
            pkg.step_batch(base, dF, mask, np.zeros(9), dts)
            for c, r in zip(inf_curves, base):
                c.append(float(r.macro_stress()[1][0, 0]))
    except pkg.RVEError as e:
        hp_error = f"GND-off increment {len(inf_curves[0])}: {e}"
    for r in base:
        r.close()
    grain_m = [w.edge * (6.0 / (math.pi * w.n_grains)) ** (1 / 3) for w in wls]
    curve = [{"rve": w.name, "grain_um": round(1e6 * g, 2), "sigma11_MPa": c[-1],
              "sigma11_inf_MPa": ci[-1] if ci else None}
             for w, g, c, ci in zip(wls, grain_m, curves, inf_curves)]
    rho_i = rvegen.material("Cu").rho0_total
    fits = {"error": hp_error} if hp_error else {}
    for k_inc in ([] if hp_error else sorted({min(nsteps, max(1, round(nsteps / 2))), nsteps})):
        eps = wls[0].rate * wls[0].dt * k_inc
        for m in ("Cu", "Al", "Ag", "Ni"):
            js = [j for j, w in enumerate(wls) if w.material == m]
            f = hall_petch_fit([grain_m[j] for j in js], [curves[j][k_inc - 1] for j in js],
                               [inf_curves[j][k_inc - 1] for j in js], rho_i)
            fits[f"{m} at {eps:.1%}"] = None if f is None else {"C": round(f[0], 5), "x": round(f[1], 4)}
    line = {"metric": "voxel-iterations/s", "value": work / el, "unit": "voxel-iter/s", "n_gpus": 1,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * el / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == 0 else "f64 local update and residual, f32 conjugate gradients",
            "data": "synthetic",
            "config": {"workload": "grain-size sweep: 16 RVEs, edges {32,48,64,96}^3, 8-400 grains, Cu/Al/Ag/Ni, "
                                   "2 % tension in 20 increments, L = 100 um, batched (one stream per RVE)",
                       "voxels": int(sum(w.n ** 3 for w in wls))},
            "gpu_launches": launches, "clocks": clocks.summary(),
            "detail": {"cg_iters_per_increment_all_rves": cg / a.steps, "flow_stress": curve,
                       "hall_petch_fit": fits,
                       "hall_petch_how": "sigma_y/sigma_inf - 1 = C (D_g sqrt(rho_i))^-x (Eq. SizeEffect2), log-log "
                                         "least squares over the four grain sizes of each material; sigma_inf from "
                                         "the same RVEs with GND off; the paper's x = 0.59-0.74 is context, not a target",
                       "launch_shapes": shapes}}
    print(json.dumps(line))


def hall_petch_fit(d_m, sigma_y, sigma_inf, rho_i):
    """Eq. SizeEffect2 of the paper, sigma_y / sigma_inf - 1 = C (D_g sqrt(rho_i))^-x,
    fitted by linear least squares of log(sigma_y / sigma_inf - 1) against
    log(D_g sqrt(rho_i)) (grain sizes D_g in m, rho_i in m^-2).  Returns
    (C, x) or None when a point has no strengthening to take the log of."""
    d = np.asarray(d_m, dtype=np.float64)
    g = np.asarray(sigma_y, dtype=np.float64) / np.asarray(sigma_inf, dtype=np.float64) - 1.0
    if len(d) < 2 or np.any(g <= 0):
        return None
    A = np.stack([np.ones_like(d), -np.log(d * math.sqrt(rho_i))], axis=1)
    (logC, x), *_ = np.linalg.lstsq(A, np.log(g), rcond=None)
    return float(math.exp(logC)), float(x)


def run_fft_compare(a):
    """The hand-written batched 3-D real FFT against cuFFT on the same box:
    forward + inverse of 3 and 9 fields at 64^3 and 128^3, FP64 and FP32
    (the library's FP32 transform exists for 3 fields, the mixed-precision
    conjugate gradients).  Ours runs on a handle's own buffers with the
    operator that sits between its z passes (the inverse-Laplacian weight for
    3 fields, the Galerkin projection for 9); cuFFT runs plain D2Z + Z2D
    (R2C + C2R) plans.  CUDA-event device time per forward + inverse pair."""
    import ctypes
    import torch
    import paper_1910_01946_gb300 as pkg
    from paper_1910_01946_gb300 import _build
    _build.build()
    pkg.load_library()
    aux = ctypes.CDLL(_build.build_aux())
    aux.aux_cufft_time.restype = ctypes.c_int
    aux.aux_cufft_time.argtypes = [ctypes.c_int] * 6 + [ctypes.POINTER(ctypes.c_double)]
    rows = []
    clocks = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
    clocks.start()
    for n in (64, 128):
        reps = 50 if n == 64 else 20
        gid = np.zeros((n, n, n), dtype=np.int32)
        quat = np.array([[1.0, 0.0, 0.0, 0.0]])
        mat = rvegen.material("Cu")
        for prec in (0, 1):
            r = pkg.RVE(gid, quat, mat, 20e-6, own_stream=True, precision=prec)
            for nf in (3, 9):
                fp32 = prec == 1
                ours = r.time_fft(nf, fp32=fp32, reps=reps) if (nf == 3 or not fp32) else None
                ms = ctypes.c_double()
                rc = aux.aux_cufft_time(n, n, n, nf, int(fp32), reps, ctypes.byref(ms))
                cu = ms.value if rc == 0 else None
                rows.append({"grid": f"{n}^3", "fields": nf, "dtype": "f32" if fp32 else "f64",
                             "ours_us": None if ours is None else round(1e3 * ours, 2),
                             "cufft_us": None if cu is None else round(1e3 * cu, 2),
                             "ours_over_cufft": None if (ours is None or cu is None) else round(ours / cu, 3)})
            r.close()
            del r
            torch.cuda.empty_cache()
    clocks.stop()
    line = {"metric": "3-D real FFT forward + inverse, hand-written vs cuFFT", "unit": "us per pair",
            "higher_is_better": False, "n_gpus": 1, "data": "synthetic (zeros; FFT time does not depend on values)",
            "rows": rows, "clocks": clocks.summary(),
            "note": "ours includes the operator fused between the z passes; cuFFT is a comparison only "
                    "(libbench_aux.so), not linked into librve.so"}
    print(json.dumps(line))


def run_convergence(a):
    """Grid and realisation convergence of the flow stress (Sec. 2.2, the
    RVE-size paragraph: coarser grids and fewer grains gave about 4 % lower
    flow stress, realisations scattered by +-2 %).  Grid study: one seeded
    100-grain Cu microstructure (the same Voronoi seeds) sampled at N^3 =
    32^3, 48^3, 64^3, 96^3; realisations: five seeds at 64^3.  Tension to 1 %
    in 10 increments, FP64 unless --precision mixed.  Reports the
    final <sigma_11> and the differences."""
    import torch
    import paper_1910_01946_gb300 as pkg
    from paper_1910_01946_gb300 import _build
    _build.build()
    pkg.load_library()
    prec = 0 if a.precision == "f64" else 1
    mask = rvegen.UNIAXIAL_X_MASK
    t0 = time.perf_counter()

    def flow_stress(wl):
        gid, quat, mat = wl.inputs()
        r = pkg.RVE(gid, quat, mat, wl.edge, own_stream=True, precision=prec)
        try:
            for _ in range(wl.increments):
                r.step(wl.dFbar(), mask, np.zeros(9), wl.dt)
            return float(r.macro_stress()[1][0, 0])
        finally:
            r.close()
            torch.cuda.empty_cache()

    grid = {}
    for n in (32, 48, 64, 96):
        grid[n] = flow_stress(rvegen.Workload(f"conv{n}", n, 100, "Cu", 0.01, 10, seed=1500))
    real = [flow_stress(rvegen.Workload(f"real{s}", 64, 100, "Cu", 0.01, 10, seed=1600 + s)) for s in range(5)]
    ref = grid[96]
    line = {"metric": "flow stress convergence (grid and realisations)", "unit": "MPa", "n_gpus": 1,
            "data": "synthetic", "dtype": "f64" if prec == 0 else "f64 local update and residual, f32 conjugate gradients",
            "config": {"workload": "Cu, 100 seeded Voronoi grains, mean grain 20 um, tension to 1 % in 10 increments; "
                                   "grid: seed 1500 sampled at 32/48/64/96^3; realisations: seeds 1600-1604 at 64^3"},
            "grid_sigma11_MPa": {f"{n}^3": round(v, 4) for n, v in grid.items()},
            "grid_rel_diff_vs_96": {f"{n}^3": round(v / ref - 1, 5) for n, v in grid.items()},
            "realisations_sigma11_MPa": [round(v, 4) for v in real],
            "realisation_mean_MPa": round(float(np.mean(real)), 4),
            "realisation_rel_std": round(float(np.std(real, ddof=1) / np.mean(real)), 5),
            "realisation_rel_range": round(float((max(real) - min(real)) / np.mean(real)), 5),
            "seconds": round(time.perf_counter() - t0, 1),
            "paper_context": "about 4 % between N = 75 / 100 grains and N = 100 / 200 grains; +-2 % scatter"}
    print(json.dumps(line))


def main():
    a = parse()
    if a.fft_compare:
        return run_fft_compare(a)
    if a.workload == "convergence":
        return run_convergence(a)
    if a.workload == "sweep":
        return run_sweep(a)
    if a.sensitivity:
        return run_sensitivity(a)
    wl = rvegen.WORKLOADS[a.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    nvox = wl.n ** 3
    config = {"workload": f"{wl.name}: {wl.n}^3 voxels, {wl.n_grains} seeded Voronoi grains, {wl.material}, "
                          f"uniaxial tension {wl.strain:.0%} in {wl.increments} increments at {wl.rate:g}/s",
              "voxels": nvox, "grains": wl.n_grains, "dt_s": wl.dt,
              "l2": "inputs larger than L2 (working set ~1 GB: tangent fields 2 x 170 MB)",
              "parallelism": f"replicas x{a.gpus}"}

    if a.impl == "reference":
        if world > 1 and rank != 0:
            return
        if a.full:
            secs, cgs, evals = oracle_increments(wl, a.warmup, a.steps)
            el = sum(secs)
            value = nvox * sum(cgs) / el
            sample = (f"{a.steps} whole oracle increments (after {a.warmup} untimed), each timed: "
                      f"{sum(cgs) / a.steps:.0f} CG iterations and {sum(evals) / a.steps:.1f} local "
                      f"evaluations per increment, {el / a.steps:.1f} s per increment")
            ms = 1e3 * el / a.steps
        else:
            # every step a real slice of 6 CG iterations and its share of the
            # local update (about 1.5 s on 8 cores at 64^3), warm-up slices untimed
            n_cg = 6
            secs = []
            for k in range(a.warmup + a.steps):
                t, nsub, _ = oracle_slice(wl, n_cg, seed=k)
                if k >= a.warmup:
                    secs.append(t)
            el = sum(secs)
            value = nvox * n_cg * a.steps / el
            ms = 1e3 * el / a.steps
            sample = (f"per step: a timed slice of the oracle's increment on the full grid, {n_cg} CG "
                      f"iterations and the local update with tangent on about {nsub} voxels (the oracle's "
                      f"own mix of {ORACLE_CG_PER_EVAL:g} CG iterations per local evaluation)")
        line = {"impl": "reference", "metric": "voxel-iterations/s", "value": value, "unit": "voxel-iter/s",
                "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
                "cpu_baseline": {"value": value, "unit": "voxel-iter/s", "cores": cpu_cores(), "kind": "oracle",
                                 "sample": sample},
                "e2e": {"value": value, "unit": "voxel-iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        if a.full:
            line["detail"] = {"seconds_per_increment": secs, "cg_iters": cgs, "local_evals": evals,
                              "cg_iters_per_local_eval": sum(cgs) / max(1, sum(evals))}
        print(json.dumps(line))
        return

    import torch
    import paper_1910_01946_gb300 as pkg
    from paper_1910_01946_gb300 import _build

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    if rank == 0:
        _build.build()
    if world > 1:
        dist.barrier()
    pkg.load_library()
    peaks = load_peaks()
    gid, quat, mat = wl.inputs()
    mask = rvegen.UNIAXIAL_X_MASK
    Pbar = np.zeros(9)
    dev = torch.device("cuda", local_rank)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()

    # ---- device-resident run (inputs already on the GPU)
    prec = 1 if a.precision == "mixed" else 0
    # a stream of the library's own: the CG chunks are replayed as CUDA graphs,
    # which the legacy default stream cannot capture
    rve = pkg.RVE(gid, quat, mat, wl.edge, device=dev, precision=prec, own_stream=True, graphs=a.graphs,
                  autotune=a.autotune or 0)
    stream = rve.stream
    for _ in range(a.warmup):
        rve.step(wl.dFbar(), mask, Pbar, wl.dt)
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    smi_index = vis.split(",")[local_rank] if vis else str(local_rank)
    clocks = ClockSampler(smi_index)
    clocks.start()
    time.sleep(0.3)
    barrier()
    # the timed increments run without per-kernel events, which would sit
    # between kernels and serialise their launches; the same increments are
    # then replayed from a checkpoint with events on for the per-kernel times
    ckpt = rve.checkpoint()
    rve.profile(False)                   # launch counting stays on
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    cg_total, newton_total, evals = 0, 0, 0
    local_iters, local_evals = 0, 0
    P_hist = []
    for _ in range(a.steps):
        info = rve.step(wl.dFbar(), mask, Pbar, wl.dt)
        if prec == 1:
            P_hist.append(rve.macro_stress()[0])     # host read after the step's own synchronisation
        cg_total += info["cg_iters_total"]
        newton_total += info["newton_iters"]
        local_iters += info["local_iters_total"]
        local_evals += info["local_evals_total"]
    ev1.record(stream)
    barrier()
    clocks.stop()
    ms = ev0.elapsed_time(ev1)
    launches_timed = int(sum(v[0] for v in rve.kernel_stats().values()))
    P_macro, sig_macro = rve.macro_stress()
    rve.restore(ckpt)
    rve.profile(True)
    cg_replay = 0
    for _ in range(a.steps):
        cg_replay += rve.step(wl.dFbar(), mask, Pbar, wl.dt)["cg_iters_total"]
    stats = rve.kernel_stats()
    rve.profile(False)
    evals = stats["constitutive"][0]
    # per-kernel events cost the replay time between kernels; the ratio says by
    # how much the summed event times exceed the plain timed region
    replay_over_timed = sum(v[1] for v in stats.values()) / ms if ms > 0 else None
    ms_max, cg_all = reduce_over_ranks(ms, cg_total, device=dev)
    value = nvox * cg_all / (ms_max / 1e3)
    launches = launches_timed
    shapes = rve.tuning()
    accuracy = None
    if prec == 1 and rank == 0:
        accuracy = mixed_accuracy(pkg, rve, wl, gid, quat, mat, dev, a, P_hist)
    rve.close()
    del rve
    torch.cuda.empty_cache()
    fp64_peak = measured_fp64_peak(smi_index) if rank == 0 else None

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not a.no_e2e:
        sig_h = torch.empty((9, nvox), dtype=torch.float64).pin_memory()
        gnd_h = torch.empty((12, nvox), dtype=torch.float64).pin_memory()
        load_h = torch.empty(9 + 9, dtype=torch.float64).pin_memory().numpy()
        r2 = pkg.RVE(gid, quat, mat, wl.edge, device=dev, precision=prec, own_stream=True, graphs=a.graphs,
                     autotune=a.autotune or 0)
        cg2 = 0
        h2d = 9 * 8 + 9 + 9 * 8
        d2h = sig_h.numel() * 8 + gnd_h.numel() * 8 + 2 * 9 * 8

        def e2e_step():
            load_h[:9] = wl.dFbar()
            load_h[9:] = Pbar
            info = r2.step(load_h[:9], mask, load_h[9:], wl.dt)
            pkg.rve_get_fields(r2.h, pkg.FIELDS["SIGMA"][0], sig_h.data_ptr(), sig_h.numel() * 8, 0)
            pkg.rve_get_fields(r2.h, pkg.FIELDS["RHO_GND"][0], gnd_h.data_ptr(), gnd_h.numel() * 8, 0)
            r2.macro_stress()
            return info

        for _ in range(a.warmup):
            e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            cg2 += e2e_step()["cg_iters_total"]
        barrier()
        el = time.perf_counter() - t0
        el_max, cg2_all = reduce_over_ranks(el, cg2, device=dev)
        e2e = {"value": nvox * cg2_all / el_max, "unit": "voxel-iter/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": 1e3 * el_max / a.steps,
               "path": "rve_step with host load arrays + rve_get_fields(SIGMA, RHO_GND) to pinned host + macro stress"}
        r2.close()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    loc = (evals, local_iters, local_evals)
    by_kernel = roofline_all(stats, (wl.n, wl.n, wl.n), peaks, local=loc, prec=prec)
    dom, roof = roofline(stats, (wl.n, wl.n, wl.n), peaks, local=loc, prec=prec)
    roof_line = None
    if roof is not None and "bound" in roof:
        traffic = TRAFFIC_64.get((dom, prec)) if wl.n == 64 else None
        roof_line = {"bound": roof["bound"], "achieved": roof["achieved"], "peak": roof["peak"], "unit": roof["unit"],
                     "frac": roof["frac"], "traffic": traffic,
                     "traffic_source": ("stored figure from one ncu capture of this kernel at 64^3 "
                                        f"({TRAFFIC_SOURCE})") if traffic else None,
                     "kernel": dom, "launches": roof["launches"],
                     "avg_us": roof["avg_us"], "share_of_kernel_time": roof["share"],
                     "peak_source": "FP64: derived 152 SM x 4 flop/clk x 2070 MHz" if roof["bound"] == "alu"
                     else f"HBM: MEASURED_PEAKS.json ({peaks['source']})"}
        if roof["bound"] == "alu" and fp64_peak:
            roof_line["fp64_peak_measured"] = fp64_peak
            roof_line["frac_of_measured_fp64"] = roof["achieved"] / fp64_peak["gflops"]
    cpu = None
    if not a.no_cpu_baseline:
        n_cg = max(2, int(round(24 * (64 ** 3) / nvox)))     # about 10-20 s of CPU work
        t, nsub, _ = oracle_slice(wl, n_cg)
        cpu = {"value": nvox * n_cg / t, "unit": "voxel-iter/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": f"a timed slice of the oracle's increment on the full grid: {n_cg} CG iterations and "
                         f"the local update with tangent on {nsub} voxels ({t:.1f} s; the oracle's own mix of "
                         f"{ORACLE_CG_PER_EVAL:g} CG iterations per local evaluation)"}
    line = {"metric": "voxel-iterations/s", "value": value, "unit": "voxel-iter/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == 0 else "f64 local update and residual, f32 conjugate gradients",
            "data": "synthetic", "config": config,
            "e2e": e2e, "gpu_launches": launches, "roofline": roof_line, "cpu_baseline": cpu,
            "clocks": clocks.summary(),
            "detail": {"cuda_graphs": bool(a.graphs), "launch_shapes": shapes,
                       "kernel_times": "per-kernel CUDA events over a replay of the timed increments from a "
                                       f"checkpoint ({cg_replay} CG iterations, {cg_total} in the timed run)",
                       "voxel_increments_per_s": world * nvox * a.steps / (ms_max / 1e3),
                       "cg_iters_per_increment": cg_total / a.steps,
                       "newton_iters_per_increment": newton_total / a.steps,
                       "local_evals_per_increment": evals / a.steps,
                       "local_newton_iters_per_voxel_eval": local_iters / max(1, evals * nvox),
                       "local_residual_evals_per_voxel_eval": local_evals / max(1, evals * nvox),
                       "macro_P11_MPa": float(P_macro[0, 0]), "macro_sigma11_MPa": float(sig_macro[0, 0]),
                       "kernels_ms": {k: round(v[1], 3) for k, v in stats.items()},
                       "kernels_launches": {k: v[0] for k, v in stats.items()},
                       "kernel_event_time_over_timed_region": replay_over_timed,
                       "roofline_by_kernel": {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv)
                                                  for kk, vv in v.items()} for k, v in by_kernel.items()}}}
    if accuracy is not None:
        line["accuracy_vs_fp64"] = accuracy
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
