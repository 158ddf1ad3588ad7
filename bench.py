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
workload (a bounded sample per step, see oracle_sample()).
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
# per-increment counts of the GPU path on this workload (local evaluations,
# CG iterations), used to compose the CPU oracle's time per increment
REF_EVALS_PER_INC = 6.0
REF_CG_PER_INC = 500.0


def parse():
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
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(rvegen.WORKLOADS) + ["sweep"],
                    help="sweep: the 16-RVE grain-size sweep stepped together (rve_step_batch)")
    ap.add_argument("--precision", default="f64", choices=["f64", "mixed"],
                    help="mixed: FP32 conjugate gradients with FP64 local update and residual")
    return ap.parse_args()


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
# iteration (Jacobian, LU, solve).  k_tangent: per voxel set-up, one
# evaluation, Jacobian and LU, the intermediate products, and the nine
# directions of dP/dF.
CONST_SETUP, CONST_EVAL, CONST_ITER = 180.0 + 270.0, 500.0, 1532.0
TANGENT_FLOPS = 180.0 + 500.0 + 1320.0 + 146.0 + 180.0 + 9 * 780.0
CONST_BYTES = 364 + 216        # reads F, dF, Fp^-1, tauc, S, grain; writes S, dgam, P
TANGENT_BYTES = 364 + 648      # reads F, dF, Fp^-1, tauc, S, grain; writes K


def kernel_models(n0, n1, n2, local=None):
    """Algorithmic FP64 flops and bytes per launch of each kernel category
    (FFTs: 2.5 N log2 N per real and 5 N log2 N per complex transform).
    `local` = (launches, local iterations, local evaluations) of the local
    update in the timed region, for its per-launch average."""
    nvox = n0 * n1 * n2
    nkx = n0 // 2 + 1
    nspec = nkx * n1 * n2
    lg = math.log2
    fx = 9 * n2 * n1 * 2.5 * n0 * lg(n0)
    fy = 9 * n2 * nkx * 5.0 * n1 * lg(n1)
    fz = 9 * nkx * n1 * 2 * 5.0 * n2 * lg(n2) + 9 * nspec * 6.0
    return {
        "fft_x_r2c": (fx, 9 * nvox * 8 + 9 * nspec * 16),
        "fft_y": (fy, 2 * 9 * nspec * 16),
        "fft_z_op": (fz, 2 * 9 * nspec * 16),
        "fft_x_c2r": (fx, 9 * nvox * 8 + 9 * nspec * 16),
        "tangent_apply": (nvox * (162 + 18 + 18), nvox * (81 + 9 + 9 + 9 + 9) * 8),
        # tiled divergence 9 -> 3 fields: per field a z-pair sum and 3 corner-sum
        # additions, 2 row additions per row, and the means of the stress-
        # controlled components (5 under uniaxial tension)
        "stencil": (nvox * (9 * 4 + 6 + 5), nvox * (9 + 3) * 8),
        # tiled gradient 3 -> 9 (z-pair sum and difference, 3 x 3 corner sums),
        # zero-mode offsets, fused x += alpha p, r -= alpha q, r . r (27 FMA)
        "cg_update": (nvox * (6 + 27 + 9 + 27 * 2), nvox * (3 + 9 * 5) * 8),
        "tangent_build": (nvox * TANGENT_FLOPS, nvox * TANGENT_BYTES),
    } | ({"constitutive": ((local[0] * nvox * CONST_SETUP + local[1] * CONST_ITER
                            + local[2] * CONST_EVAL) / local[0], nvox * CONST_BYTES)}
         if local and local[0] else {})


# the FP32 conjugate-gradient kernels of the mixed path: half the bytes of the
# FP64 model, and their FP32 arithmetic is far below the FP32 peak, so HBM binds
FP32_CG = ("tangent_apply", "stencil", "cg_update", "fft_x_r2c", "fft_y", "fft_z_op", "fft_x_c2r")


def roofline(stats, shape, peaks, local=None, prec=0):
    models = kernel_models(*shape, local=local)
    if prec == 1:
        for k in FP32_CG:
            models[k] = (0.0, models[k][1] / 2)
    timed = {k: v for k, v in stats.items() if v[0] > 0 and v[1] > 0}
    if not timed:
        return None, None
    dom = max(timed, key=lambda k: timed[k][1])
    n, ms = timed[dom]
    avg_s = ms / n / 1e3
    out = {"kernel": dom, "launches": n, "avg_us": avg_s * 1e6, "share": ms / sum(v[1] for v in timed.values())}
    if dom in models:
        flops, nbytes = models[dom]
        t_alu = flops / (FP64_PEAK_GFLOPS * 1e9)
        t_hbm = nbytes / (peaks["hbm_gbs"] * 1e9)
        if t_alu >= t_hbm:
            ach = flops / avg_s / 1e9
            out.update(bound="alu", achieved=ach, peak=FP64_PEAK_GFLOPS, unit="GFLOP/s (FP64)", frac=ach / FP64_PEAK_GFLOPS)
        else:
            ach = nbytes / avg_s / 1e9
            out.update(bound="hbm", achieved=ach, peak=peaks["hbm_gbs"], unit="GB/s", frac=ach / peaks["hbm_gbs"])
        out["algorithmic_flops"] = flops
        out["algorithmic_bytes"] = nbytes
    return dom, out


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# kernels that lead the timed region, from one ncu capture of the 64^3
# workload; keyed by (category, precision).  Kernels changed since that
# capture have no entry (reported as null), as do other grid sizes.
TRAFFIC_64 = {
    ("tangent_apply", 0): 207.66e6 + 5.10e6,   # K : p reads its algorithmic 207.6 MB
    ("tangent_apply", 1): 103.84e6 + 3.53e6,   # TMA-staged FP32 apply (float K, r, p)
    ("constitutive", 0): 98.92e6 + 50.16e6,    # k_local (the same kernel in both precisions)
    ("constitutive", 1): 98.92e6 + 50.16e6,
    ("tangent_build", 0): 78.10e6 + 211.22e6,  # k_tangent, K written in FP64
    ("stencil", 0): 18.94e6,                   # k_div (its writes stay in L2)
    ("cg_update", 0): 62.95e6 + 0.11e6,        # k_grad_t<true>
}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d.get("hbm_gbs", 6800.0), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


# ---------------------------------------------------------------- CPU oracle
def oracle_sample(wl, frac=0.08, n_cg=2, seed=0):
    """Bounded sample of the FP64 CPU oracle on the workload: the local update
    with tangent on a seeded subset of grains holding about `frac` of the
    voxels, and n_cg conjugate-gradient iterations on the full grid.  Returns
    the composed seconds per increment for REF_EVALS_PER_INC local
    evaluations and REF_CG_PER_INC CG iterations, and the sample's own CPU
    seconds."""
    from oracle import solver
    from oracle import spectral as sp
    gid, quat, mat = wl.inputs()
    o = solver.RVE(gid, quat, mat, wl.edge)
    nv = gid.size
    t0 = time.perf_counter()
    tauc, ell = o.hardening()
    t_hard = time.perf_counter() - t0
    F = o.F + (wl.dFbar() * rvegen.UNIAXIAL_X_MASK).reshape(3, 3)
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(o.grains))
    chosen, count = [], 0
    for gi in order:
        chosen.append(o.grains[gi])
        count += len(o.grains[gi]["idx"])
        if count >= frac * nv:
            break
    keep = o.grains
    o.grains = chosen
    idx = np.concatenate([g["idx"] for g in chosen])
    t0 = time.perf_counter()
    P, K, S, M, dg, lit, lf = o.constitutive(F, tauc, o.S, wl.dt)
    t_eval = (time.perf_counter() - t0) / len(idx)
    o.grains = keep
    Kfull = np.resize(K[idx], (nv, 3, 3, 3, 3))
    R = o.flat(sp.project(o.field(np.resize(P[idx], (nv, 3, 3))), rvegen.UNIAXIAL_X_MASK, o.h))
    o.opts.max_cg = n_cg
    o.opts.cg_tol = 1e-300
    t0 = time.perf_counter()
    o.cg(Kfull, -R, rvegen.UNIAXIAL_X_MASK)
    t_cg = (time.perf_counter() - t0) / n_cg
    per_inc = REF_EVALS_PER_INC * nv * t_eval + REF_CG_PER_INC * t_cg + t_hard
    sample_s = t_hard + t_eval * len(idx) + t_cg * n_cg
    return per_inc, sample_s, len(idx), t_eval, t_cg


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
    for k in range(a.warmup):
        try:
            pkg.step_batch(rves, dF, mask, np.zeros(9), dts)
        except pkg.RVEError as e:
            print(json.dumps({"metric": "voxel-iterations/s", "error": f"warm-up increment {k}: {e}"}))
            raise
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
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    clocks.stop()
    launches = sum(sum(v[0] for v in r.kernel_stats().values()) for r in rves)
    curve = [{"rve": w.name, "grain_um": round(w.edge * 1e6 * (6.0 / (math.pi * w.n_grains)) ** (1 / 3), 2),
              "sigma11_MPa": float(r.macro_stress()[1][0, 0])} for w, r in zip(wls, rves)]
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
                       "launch_shapes": [r.tuning() for r in rves]}}
    for r in rves:
        r.close()
    print(json.dumps(line))


def main():
    a = parse()
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
        times = []
        samp = None
        for k in range(a.warmup + a.steps):
            per_inc, sample_s, nsub, t_eval, t_cg = oracle_sample(wl, frac=0.02, n_cg=1, seed=k)
            if k >= a.warmup:
                times.append(per_inc)
                samp = (sample_s, nsub)
        ms = 1e3 * statistics.mean(times)
        value = nvox * REF_CG_PER_INC / (ms / 1e3)
        line = {"impl": "reference", "metric": "voxel-iterations/s", "value": value, "unit": "voxel-iter/s",
                "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
                "cpu_baseline": {"value": value, "unit": "voxel-iter/s", "cores": cpu_cores(), "kind": "oracle",
                                 "sample": f"per step: oracle local update + tangent on {samp[1]} voxels and 1 CG "
                                           f"iteration on the full grid ({samp[0]:.1f} s), composed to "
                                           f"{REF_EVALS_PER_INC:g} evaluations + {REF_CG_PER_INC:g} CG iterations "
                                           "per increment"},
                "e2e": {"value": value, "unit": "voxel-iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
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
    for _ in range(a.steps):
        info = rve.step(wl.dFbar(), mask, Pbar, wl.dt)
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
    ms_max, cg_all = reduce_over_ranks(ms, cg_total, device=dev)
    value = nvox * cg_all / (ms_max / 1e3)
    launches = launches_timed
    shapes = rve.tuning()
    rve.close()
    del rve
    torch.cuda.empty_cache()

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
    dom, roof = roofline(stats, (wl.n, wl.n, wl.n), peaks, local=(evals, local_iters, local_evals), prec=prec)
    roof_line = None
    if roof is not None and "bound" in roof:
        roof_line = {"bound": roof["bound"], "achieved": roof["achieved"], "peak": roof["peak"], "unit": roof["unit"],
                     "frac": roof["frac"],
                     "traffic": TRAFFIC_64.get((dom, prec)) if wl.n == 64 else None,
                     "kernel": dom, "launches": roof["launches"],
                     "avg_us": roof["avg_us"], "share_of_kernel_time": roof["share"],
                     "peak_source": "FP64: derived 152 SM x 4 flop/clk x 2070 MHz" if roof["bound"] == "alu"
                     else f"HBM: MEASURED_PEAKS.json ({peaks['source']})"}
    cpu = None
    if not a.no_cpu_baseline:
        per_inc, sample_s, nsub, t_eval, t_cg = oracle_sample(wl)
        evals_per_inc = evals / a.steps
        cg_per_inc = cg_total / a.steps
        t_inc = evals_per_inc * nvox * t_eval + cg_per_inc * t_cg
        cpu = {"value": nvox * cg_per_inc / t_inc, "unit": "voxel-iter/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": f"oracle local update + tangent on {nsub} voxels ({t_eval * 1e6:.0f} us/voxel) and 2 CG "
                         f"iterations on the full grid ({t_cg:.2f} s each), {sample_s:.1f} s in all; composed with "
                         f"this run's {evals_per_inc:.1f} evaluations and {cg_per_inc:.0f} CG iterations per increment"}
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
                       "kernels_launches": {k: v[0] for k, v in stats.items()}}}
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
