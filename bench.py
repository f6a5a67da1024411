#!/usr/bin/env python3
"""Throughput of the matrix-free TPFA conjugate-gradient solve on GB300.

One step = one full solve of the paper-scale workload through the C ABI:
transmissibilities + diagonal (tpfa_build_trans), right-hand side
(tpfa_build_rhs), and cg_solve to the FP64-checked relative residual (inner
FP32 CG sweeps, FP64 residual, refinement).  Metric: cell-updates/s =
cells x CG iterations / time (the paper's Gcell/s definition, Table III).

Workload (synthetic, seeded): 1024 x 1024 x 256 cells, ln K ~ N(0, 1.5^2)
drawn per (i, j, floor(k/8)) (8-cell vertical layer correlation),
accumulation diagonal d = 1e-3, injector/producer (q = +-1) at opposite
corners, no Dirichlet cells, CG to relative residual 1e-6.

--impl reference times the CPU FP64 oracle (CSR assembly + textbook CG) on
a bounded sample of the same workload recipe.

Multi-GPU: the solve does not shard here (replicas only): each rank solves
its own copy; value = all ranks' cell-updates / max rank time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2408_03452_gb300 import synth  # noqa: E402

METRIC = "TPFA-CG cell-updates/s"
UNIT = "cell-updates/s"
# algorithmic DRAM bytes per cell of one fused CG sweep: read r, p, q, x and
# the 16-byte coefficient record, write r, p, q, x (FP32)
SWEEP_BYTES_PER_CELL = 48
# algorithmic DRAM bytes per cell of one operator application: read p and the
# 16-byte coefficient record, write A p
APPLY_BYTES_PER_CELL = 24
FALLBACK_HBM_GBS = 6800.0
# nominal HBM3e bandwidth of one GB300 (the north star's "~8 TB/s"), for a
# second roofline fraction beside the measured copy peak
NOMINAL_HBM_GBS = 8000.0
LEARNED_METRIC = "U-Net FCG cell-iterations/s"
LEARNED_FCG_M = 2  # retained directions of flexible CG in the learned workload
LEARNED_LEVELS = 2  # the network runs on the 2^levels coarser grid
LEARNED_UNIT = "cell-iterations/s"
# useful FLOPs per cell of one U-Net application (true layer shapes: 2->16,
# 16->16 and 16->1 at full resolution, 16->32 and 32->16 at 1/8, 32->64 and
# 64->32 at 1/64 of the cells; 2*27*cin*cout per layer and cell)
UNET_FLOP_PER_CELL = 2 * 27 * (2 * 16 + 16 * 16 + 16 * 1 + (16 * 32 + 32 * 16) / 8
                               + (32 * 64 + 64 * 32) / 64)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nx", type=int, default=1024)
    ap.add_argument("--ny", type=int, default=1024)
    ap.add_argument("--nz", type=int, default=256)
    ap.add_argument("--n-inst", type=int, default=96, help="ensemble size (--workload ensemble)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--compare-single", action="store_true",
                    help="ensemble: also time the instances solved one after another")
    ap.add_argument("--workload", default="paper",
                    choices=["paper", "channelized", "ensemble", "table3", "learned"],
                    help="paper: 1024x1024x256 layered lognormal, wells, CG to 1e-6 (default); "
                         "channelized: 256^3 sigma-2 background + 1e4 channels, Dirichlet x "
                         "ends, refined to 1e-10 (the mixed-precision configuration)")
    ap.add_argument("--epochs", type=int, default=12, help="learned: training epochs")
    ap.add_argument("--n-real", type=int, default=50, help="learned: training realizations")
    ap.add_argument("--snaps", type=int, default=40, help="learned: pairs per realization")
    ap.add_argument("--inner", default="f32", choices=["f32", "bf16"],
                    help="coefficient records of the inner CG sweeps")
    ap.add_argument("--precond", type=int, default=0, help="0: plain CG (Alg. 1); 1: Jacobi")
    ap.add_argument("--tol", type=float, default=None)
    ap.add_argument("--maxit", type=int, default=200000)
    ap.add_argument("--allow-notconv", action="store_true",
                    help="record solves that stop at maxit instead of failing")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=1,
                    help="solves timed end to end with host buffers (0 = skip)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-ttt", action="store_true",
                    help="paper workload: skip the time-to-1e-8 solver comparison")
    ap.add_argument("--window", type=int, default=1,
                    help="paper workload: also time the oracle on the full grid (a 10-iteration "
                         "window) when host memory allows (0 = skip)")
    ap.add_argument("--tile-vy", type=int, default=0)
    ap.add_argument("--tile-zc", type=int, default=-1)
    ap.add_argument("--stages", type=int, default=0)
    ap.add_argument("--loop", type=int, default=0,
                    help="0: CUDA-graph while loop; 1: host-polled graph chunks")
    ap.add_argument("--sweep", type=int, default=0,
                    help="CG sweep kernel: 0 automatic, 1 cp.async-staged, 2 TMA-staged")
    ap.add_argument("--tma-tile", type=int, default=-1, help="tile of the TMA-staged sweep")
    ap.add_argument("--probe-iters", type=int, default=0,
                    help="profiling aid: build the workload, run one solve capped at this many "
                         "CG iterations (host-polled chunks of 4), print its info, no timing")
    ap.add_argument("--probe-apply", type=int, default=0,
                    help="profiling aid: build the workload's records, run this many operator "
                         "applications (tpfa_apply, or tpfa_apply_bf16 with --inner bf16) with "
                         "p'Ap, print the tiling, no timing")
    return ap.parse_args()


def workload_desc(a):
    solver = ("plain CG" if a.precond == 0 else "Jacobi-preconditioned CG") + \
        (", FP32 records" if a.inner == "f32" else ", BF16 records")
    if a.workload == "ensemble":
        return (f"batched ensemble of {a.n_inst} TPFA problems, sizes uniform over "
                f"{{48x48x24, 64x64x32, 96x96x48, 128x128x64}}, lnK~N(0,s^2) with s~U(0.5,2.5) "
                f"per instance, Dirichlet end layers on a random axis (p_hi~U(0.5,2), p_lo=0), "
                f"{solver}, each refined to FP64 relative residual {a.tol:g}, one batched sweep "
                f"launch per iteration")
    if a.workload == "channelized":
        return (f"channelized TPFA pressure solve {a.nx}x{a.ny}x{a.nz}, lnK~N(0,2^2) background "
                f"plus 8 sinusoidal channels 1e4x more permeable, Dirichlet p=1/0 on the x end "
                f"layers, {solver} refined to FP64 relative residual {a.tol:g}")
    return (f"paper-scale TPFA pressure solve {a.nx}x{a.ny}x{a.nz}, lnK~N(0,1.5^2) per "
            f"(i,j,k//8), d=1e-3, well pair q=+-1 at opposite corners, no Dirichlet, "
            f"{solver} to FP64-checked relative residual {a.tol:g}")


def finish_args(a):
    if a.workload in ("channelized", "learned") and (a.nx, a.ny, a.nz) == (1024, 1024, 256):
        a.nx = a.ny = a.nz = 256
    if a.tol is None:
        a.tol = {"channelized": 1e-10, "ensemble": 1e-8, "learned": 1e-8}.get(a.workload, 1e-6)
    return a


# ----------------------------------------------------------------------------
# CPU oracle leg
# ----------------------------------------------------------------------------

SAMPLE = (256, 256, 128)
SAMPLE_CHANNELS = (64, 64, 64)


def oracle_step(O, iters, workload="paper"):
    """Oracle on a bounded sample of the same recipe: assemble the CSR of a
    256x256x128 block (64^3 for the channelized recipe), build the
    right-hand side, run `iters` CG iterations (Jacobi PCG on the
    channelized recipe, whose plain CG barely moves), evaluate the FP64
    residual.  Returns cell-updates done."""
    if workload == "learned":
        return oracle_fcg_step(iters)
    if workload == "channelized":
        nx, ny, nz = SAMPLE_CHANNELS
        w = synth.channelized(seed=0, n=nx)
        g = O.Grid(nx, ny, nz)
        A = O.assemble(g, w["K"], w["mask"], 0.0)
        b = O.rhs(g, w["K"], w["mask"], None, w["pD"])
        x, st, it, _ = O.pcg_jacobi(A, b, tol=0.0, maxit=iters)
        float(np.linalg.norm(b - A.matvec(x)))
        return nx * ny * nz * it
    nx, ny, nz = SAMPLE
    K = synth.lognormal_field(nx, ny, nz, 1.5, 0, layer=8)
    idx, val = synth.well_pair(nx, ny, nz)
    q = synth.dense_sources(nx * ny * nz, idx, val)
    g = O.Grid(nx, ny, nz)
    A = O.assemble(g, K, None, 1e-3)
    b = O.rhs(g, K, None, q, None)
    x, st, it, _ = O.cg(A, b, tol=0.0, maxit=iters)
    r = b - A.matvec(x)
    float(np.linalg.norm(r))
    return nx * ny * nz * it


SAMPLE_LEARNED = 32


def oracle_fcg_step(iters, params=None):
    """Oracle flexible CG with the Jacobi-blended U-Net (on the 2^LEARNED_LEVELS
    coarser grid) on a 32^3 lognormal
    (sigma 1.5) realization with Dirichlet x ends: CSR assembly, RHS, `iters`
    FCG iterations.  params: flat parameter vector (default: He
    initialisation of the oracle).  Returns cell-iterations done."""
    from oracle import oracle as O
    from oracle import unet_oracle as U
    n = SAMPLE_LEARNED
    K = synth.lognormal_field(n, n, n, 1.5, 5)
    mask, pD = synth.dirichlet_faces(n, n, n, "x", 1.0, 0.0)
    g = O.Grid(n, n, n)
    A = O.assemble(g, K, mask)
    b = O.rhs(g, K, mask, None, pD)
    if params is None:
        p = U.init_params(0)
    else:
        p, off = {}, 0
        for i, (name, cin, cout) in enumerate(U.LAYERS):
            nw = 27 * cin * cout
            p[name] = params[off:off + nw].reshape(27, cout, cin).astype(np.float64)
            p["b%d" % i] = params[off + nw:off + nw + cout].astype(np.float64)
            off += nw + cout
    lnk = np.log(K).reshape(1, n, n, n)
    dinv = 1.0 / np.asarray(A.dense().diagonal()) if n ** 3 <= 4096 else None
    if dinv is None:
        diag = np.zeros(n ** 3)
        for i in range(n ** 3):
            lo, hi = A.rowptr[i], A.rowptr[i + 1]
            j = np.nonzero(A.cols[lo:hi] == i)[0]
            diag[i] = A.vals[lo + j[0]]
        dinv = 1.0 / diag

    def precond(r):
        u = U.precondition_coarse(p, r.reshape(1, n, n, n), lnk, LEARNED_LEVELS).reshape(-1)
        return U.jacobi_blend(u, r, dinv, A.matvec)[0]

    _, it, _ = U.fcg(A.matvec, b, precond, 0.0, iters)
    return n ** 3 * it


def oracle_sample_iters(O, target_s=12.0, workload="paper"):
    """Iterations for one oracle step of about target_s: the solver's iterations
    take about 60% of it, the sample's setup (generation, CSR assembly) the rest.
    The per-iteration cost is timed on the solver alone (the setup varies by
    more than a few iterations cost)."""
    per = oracle_iteration_s(O, workload)
    return max(5, min(int(0.6 * target_s / per), 100000))


def oracle_iteration_s(O, workload="paper"):
    """Seconds per iteration of the oracle's solver on the sample of `workload`
    (the solver timed alone, 10 and 30 iterations)."""
    if workload == "learned":
        t = time.perf_counter()
        oracle_fcg_step(3)
        t3 = time.perf_counter() - t
        t = time.perf_counter()
        oracle_fcg_step(13)
        return max((time.perf_counter() - t - t3) / 10, 1e-4)
    if workload == "channelized":
        nx, ny, nz = SAMPLE_CHANNELS
        w = synth.channelized(seed=0, n=nx)
        g = O.Grid(nx, ny, nz)
        A = O.assemble(g, w["K"], w["mask"], 0.0)
        b = O.rhs(g, w["K"], w["mask"], None, w["pD"])
        solve = O.pcg_jacobi
    else:
        nx, ny, nz = SAMPLE
        K = synth.lognormal_field(nx, ny, nz, 1.5, 0, layer=8)
        idx, val = synth.well_pair(nx, ny, nz)
        q = synth.dense_sources(nx * ny * nz, idx, val)
        g = O.Grid(nx, ny, nz)
        A = O.assemble(g, K, None, 1e-3)
        b = O.rhs(g, K, None, q, None)
        solve = O.cg
    t = time.perf_counter()
    solve(A, b, tol=0.0, maxit=10)
    t10 = time.perf_counter() - t
    t = time.perf_counter()
    solve(A, b, tol=0.0, maxit=30)
    return max((time.perf_counter() - t - t10) / 20, 1e-6)


def sample_desc(workload):
    if workload == "learned":
        n = SAMPLE_LEARNED
        return f"{n}x{n}x{n} lognormal (sigma 1.5) realization, U-Net FCG with the Jacobi blend"
    s = SAMPLE_CHANNELS if workload == "channelized" else SAMPLE
    return f"{s[0]}x{s[1]}x{s[2]} block of the same recipe"


def metric_unit(workload):
    if workload == "learned":
        return LEARNED_METRIC, LEARNED_UNIT
    return METRIC, UNIT


def oracle_cores(workload):
    # the C oracle runs its rows on all host threads (OpenMP); the learned-
    # preconditioner oracle runs numpy matrix products (BLAS threads)
    if workload == "learned":
        return os.cpu_count()
    from oracle import oracle as O
    return O.threads()


def mem_available_gb():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) / 1e6
    except OSError:
        pass
    return 0.0


def oracle_window_estimate(w, iters=10):
    """The oracle on the full benchmark grid: CSR assembly of all cells, the
    right-hand side, then a window of `iters` CG iterations, timed.  A full
    oracle solve at this size would take hours; the per-iteration time of the
    window is reported as an estimate of its rate."""
    from oracle import oracle as O
    nx, ny, nz = w["nx"], w["ny"], w["nz"]
    n = nx * ny * nz
    need_gb = n * (7 * 16 + 8 + 7 * 8) / 1e9 + 4
    have = mem_available_gb()
    if have < need_gb:
        return {"skipped": f"needs about {need_gb:.0f} GB of host memory, {have:.0f} GB available"}
    O.build()
    g = O.Grid(nx, ny, nz)
    t = time.perf_counter()
    A = O.assemble(g, w["K"], None, w["d"])
    q = synth.dense_sources(n, w["src_idx"], w["src_val"])
    b = O.rhs(g, w["K"], None, q, None)
    t_asm = time.perf_counter() - t
    t = time.perf_counter()
    _, _, it, _ = O.cg(A, b, tol=0.0, maxit=iters)
    t_cg = time.perf_counter() - t
    del A, b, q
    return {"kind": "estimate", "grid": [nx, ny, nz], "iterations": it,
            "value": n * it / t_cg, "unit": UNIT, "s_per_iteration": t_cg / max(it, 1),
            "assembly_and_rhs_s": t_asm, "cores": O.threads(),
            "what": f"oracle CSR CG on the full grid: a window of {it} iterations of the solve, "
                    f"timed after assembly; the per-iteration rate stands for the whole solve"}


def cpu_baseline(target_s=12.0, workload="paper"):
    from oracle import oracle as O
    O.build()
    iters = oracle_sample_iters(O, target_s, workload)
    t = time.perf_counter()
    units = oracle_step(O, iters, workload)
    dt = time.perf_counter() - t
    what = "FCG" if workload == "learned" else "CG"
    how = "numpy" if workload == "learned" else "C with OpenMP"
    if workload == "channelized":
        what = "Jacobi PCG"
    return {"value": units / dt, "unit": metric_unit(workload)[1], "cores": oracle_cores(workload),
            "kind": "oracle",
            "sample": f"{sample_desc(workload)}: CSR assembly, RHS, {iters} {what} iterations, "
                      f"FP64; {how}, {dt:.1f} s"}


def run_reference(a, rank, world):
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    iters = oracle_sample_iters(O, 10.0, a.workload)
    for _ in range(a.warmup):
        oracle_step(O, iters, a.workload)
    times, units = [], 0
    for _ in range(a.steps):
        t = time.perf_counter()
        units += oracle_step(O, iters, a.workload)
        times.append(time.perf_counter() - t)
    tot = sum(times)
    val = units / tot
    metric, unit = metric_unit(a.workload)
    what = "FCG" if a.workload == "learned" else "CG"
    sample = (f"each step: {sample_desc(a.workload)}, CSR assembly, RHS, {iters} {what} "
              f"iterations, FP64")
    print(json.dumps({
        "impl": "reference", "metric": metric, "value": val, "unit": unit, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * tot / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_desc(a), "sample": sample},
        "cpu_baseline": {"value": val, "unit": unit, "cores": oracle_cores(a.workload),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------
# GPU leg
# ----------------------------------------------------------------------------

def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        v = float(json.load(open(p))["hbm_gbs"])
        return v, "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_traffic(record, cells):
    """DRAM bytes of one launch of a TMA-staged kernel over `cells` cells from
    a committed ncu summary under profiles/ (bytes per cell of a smaller
    capture with the same 128-plane runs, times the cells), if it was taken on
    the current kernel source; else None."""
    src = os.path.join(ROOT, "paper_2408_03452_gb300", "csrc", "sweep_tma.cu")
    prof = os.path.join(ROOT, "profiles", record)
    try:
        rec = json.load(open(prof))
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        if rec.get("source_sha256_16") != h:
            return None
        return rec["dram_bytes_per_cell"] * cells
    except Exception:
        return None


def sweep_traffic(nx, ny, nz):
    """The CG sweep (TMA-staged, FP32 records, plain CG)."""
    return kernel_traffic("cg_sweep_traffic.json", nx * ny * nz)


# Table III of the paper (Section V.C): grid, CG iterations, CS-2 and A100
# times of the whole CG solve (Alg. 1), in seconds.  Context, not targets.
TABLE3 = [((200, 200, 922), 226, 0.0251, 2.8021), ((400, 400, 922), 225, 0.0337, 5.6343),
          ((600, 600, 922), 225, 0.0423, 11.8380), ((750, 600, 922), 225, 0.0456, 16.3473),
          ((750, 800, 922), 225, 0.0500, 20.9367), ((750, 950, 922), 225, 0.0532, 22.9128),
          ((750, 994, 922), 225, 0.0542, 23.1879)]


def run_table3(a, dev, rank):
    """Weak-scaling sweep over the paper's Table III grids (nz = 922): the
    paper-scale recipe (layered lognormal, d = 1e-3, corner wells) on each
    grid, 225 CG iterations as in the table, timed with CUDA events
    (coefficient build, right-hand side, the iterations and the FP64 check)."""
    import torch
    from paper_2408_03452_gb300 import tpfa
    rows = []
    for (nx, ny, nz), it_paper, cs2_s, a100_s in TABLE3:
        n = nx * ny * nz
        w = synth.paper_scale(seed=a.seed, nx=nx, ny=ny, nz=nz)
        K = torch.from_numpy(w["K"]).to(dev)
        si, sv = torch.from_numpy(w["src_idx"]).to(dev), torch.from_numpy(w["src_val"]).to(dev)
        del w
        with tpfa.Context(nx, ny, nz, device=dev) as ctx:
            ctx.set_option("precond", a.precond)
            coef = torch.empty((n, 4), dtype=torch.float32, device=dev)
            coef64 = torch.empty((n, 4), dtype=torch.float64, device=dev)
            b = torch.empty(n, dtype=torch.float64, device=dev)
            x = torch.empty(n, dtype=torch.float64, device=dev)
            times = []
            for rep in range(1 + max(a.steps, 1)):
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                ctx.build_trans(K, None, None, 1e-3, coef=coef, coef64=coef64)
                ctx.build_rhs(K, None, None, None, si, sv, b=b)
                x.zero_()
                _, info = ctx.cg_solve(coef, coef64, b, x=x, tol=1e-30, maxit=225, check=False)
                e1.record()
                torch.cuda.synchronize()
                if rep > 0:  # the first run is a warm-up
                    times.append(e0.elapsed_time(e1) / 1e3)
            t = sum(times) / len(times)
            rows.append({"grid": [nx, ny, nz], "cells": n, "iters": info["iters"],
                         "time_s": t, "gcell_s": n * info["iters"] / t / 1e9,
                         "sweep_ms": info["inner_ms"] / max(info["iters"], 1),
                         "paper_cs2_s": cs2_s, "paper_a100_s": a100_s,
                         "paper_iters": it_paper})
        del K, coef, coef64, b, x
        torch.cuda.empty_cache()
    if rank == 0:
        last = rows[-1]
        print(json.dumps({
            "metric": METRIC, "value": last["cells"] * last["iters"] / last["time_s"],
            "unit": UNIT, "n_gpus": 1, "steps": a.steps, "warmup": 1,
            "ms_per_step": 1e3 * last["time_s"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "Table III weak-scaling grids (nz = 922) with the paper-scale "
                                   "recipe, 225 CG iterations each, "
                                   + ("plain CG" if a.precond == 0 else "Jacobi PCG")},
            "sweep": rows}))


def measured_tensor_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(p))["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def time_conv(tpfa, dev, n, cin, cout, reps=10):
    """CUDA-event time of one tensor-core convolution launch on an n^3
    haloed BF16 volume (random data, ReLU epilogue)."""
    import torch
    V = tpfa.halo_voxels(n, n, n)
    x = torch.zeros((n + 2, n + 2, n + 2, cin), dtype=torch.bfloat16, device=dev)
    x[1:-1, 1:-1, 1:-1] = torch.rand((n, n, n, cin), device=dev, dtype=torch.float32).to(torch.bfloat16)
    y = torch.zeros((V, cout), dtype=torch.bfloat16, device=dev)
    w = (torch.rand((27, cout, cin), device=dev) - 0.5).to(torch.bfloat16)
    b = torch.zeros(cout, dtype=torch.float32, device=dev)
    xs = x.reshape(V, cin)
    for _ in range(3):
        tpfa.conv3d_bf16(xs, w, y, (n, n, n, 1), cin, cout, bias=b, flags=tpfa.CONV_RELU)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        tpfa.conv3d_bf16(xs, w, y, (n, n, n, 1), cin, cout, bias=b, flags=tpfa.CONV_RELU)
    e1.record(stream)
    tpfa.net_status(dev)
    return e0.elapsed_time(e1) / reps


def time_to_1e8(dev, seed=0, n=256, tol=1e-8, ensemble=True, maxit=200000):
    """The metric's comparison of solvers by time to an FP64 relative residual
    of 1e-8, on one GPU, on a held-out n^3 lognormal (sigma 1.5) realization
    with Dirichlet x ends: plain CG (Alg. 1), Jacobi PCG, Jacobi PCG on BF16
    records (mixed precision) and flexible CG with the U-Net preconditioner
    (trained first, untimed, at 64^3), each run once untimed and once timed
    (CUDA events inside the call); with ensemble=True the same comparison on
    the batched 96-instance ensemble."""
    import torch
    from paper_2408_03452_gb300 import learned, tpfa
    t0 = time.perf_counter()
    ds = learned.make_dataset(50, 40, 64)
    P, hist = learned.train(ds, epochs=12, batch=16, lr=1e-3, levels=LEARNED_LEVELS)
    train_s = time.perf_counter() - t0
    n_pairs = len(ds.real)
    del ds
    torch.cuda.empty_cache()
    ctx = tpfa.Context(n, n, n, device=dev)
    ctx.set_option("fcg_m", LEARNED_FCG_M)
    pr = learned.Problem(ctx, 777001 + seed, n, 1.5)
    Kh, mh, _ = learned.realization(777001 + seed, n, 1.5)
    c16 = ctx.build_trans_bf16(torch.from_numpy(Kh).to(dev), torch.from_numpy(mh).to(dev))
    del Kh, mh
    nn = n >> LEARNED_LEVELS
    net = tpfa.UNet(nn, nn, nn, device=dev)
    net.set_params(P)
    x = torch.zeros(n ** 3, dtype=torch.float64, device=dev)

    def fcg():
        x.zero_()
        return ctx.fcg_solve(pr.coef, pr.coef64, pr.b, net=net, lnk=pr.lnk, x=x, tol=tol,
                             maxit=maxit)[1]

    def cg(precond, coef):
        def run():
            ctx.set_option("precond", precond)
            x.zero_()
            info = ctx.cg_solve(coef, pr.coef64, pr.b, x=x, tol=tol, maxit=maxit)[1]
            ctx.set_option("precond", 0)
            return info
        return run

    out = {"grid": [n, n, n], "tol": tol,
           "workload": f"held-out {n}^3 lognormal sigma-1.5 realization, Dirichlet x ends",
           "time_s": {}, "iters": {}, "rel_res_fp64": {}, "converged": {}}
    for name, fn in (("plain_cg", cg(0, pr.coef)), ("jacobi_pcg", cg(1, pr.coef)),
                     ("jacobi_pcg_bf16_records", cg(1, c16)), ("unet_fcg", fcg)):
        fn()
        info = fn()
        out["time_s"][name] = info["total_ms"] / 1e3
        out["iters"][name] = info["iters"]
        out["rel_res_fp64"][name] = info["rel_res_fp64"]
        out["converged"][name] = info["code"] == tpfa.OK
    out["chosen"] = "unet_fcg"
    out["speedup_vs_plain_cg"] = {k: out["time_s"]["plain_cg"] / v for k, v in out["time_s"].items()}
    out["training"] = {"pairs": n_pairs, "seconds": train_s, "final_val_loss": hist["val_loss"][-1],
                       "jacobi_loss": hist["jacobi_loss"], "untimed": True}
    ctx.close()
    del pr, net, x, c16
    torch.cuda.empty_cache()
    if ensemble:
        e = learned.evaluate_ensemble(P, seed=seed, levels=LEARNED_LEVELS, fcg_m=LEARNED_FCG_M,
                                      tol=tol)
        out["ensemble"] = {k: e[k] for k in ("instances", "cells", "sizes")}
        for k in ("plain_cg_batched", "jacobi_pcg_batched", "unet_fcg_batched"):
            out["ensemble"][k] = {"s": e[k]["s"], "iters_min_max": e[k]["iters_min_max"],
                                  "rel_res_fp64_max": e[k]["rel_res_fp64_max"],
                                  "code": e[k]["code"]}
        # the chosen form for the ensemble: a network trained (untimed) on the
        # ensemble's own distribution (sigma ~ U(0.5, 2.5), Dirichlet ends on a
        # random axis), same budget as the 64^3 network
        t1 = time.perf_counter()
        ds = learned.make_dataset(50, 40, 64, mixed=True)
        P_mix, hist_mix = learned.train(ds, epochs=12, batch=16, lr=1e-3, levels=LEARNED_LEVELS)
        mix_s = time.perf_counter() - t1
        del ds
        torch.cuda.empty_cache()
        em = learned.evaluate_ensemble(P_mix, seed=seed, levels=LEARNED_LEVELS,
                                       fcg_m=LEARNED_FCG_M, tol=tol, solvers=("unet_fcg_batched",))
        k = "unet_fcg_batched"
        out["ensemble"]["unet_fcg_batched_ensemble_trained"] = {
            "s": em[k]["s"], "iters_min_max": em[k]["iters_min_max"],
            "rel_res_fp64_max": em[k]["rel_res_fp64_max"], "code": em[k]["code"],
            "training": {"seconds": mix_s, "final_val_loss": hist_mix["val_loss"][-1],
                         "untimed": True}}
        out["ensemble"]["chosen"] = "unet_fcg_batched_ensemble_trained"
        out["ensemble"]["speedup_vs_plain_cg"] = {
            k: out["ensemble"]["plain_cg_batched"]["s"] / out["ensemble"][k]["s"]
            for k in ("plain_cg_batched", "jacobi_pcg_batched", "unet_fcg_batched",
                      "unet_fcg_batched_ensemble_trained")}
    return out


def channelized_steps(a, dev, n=64):
    """GPU iterates after each FP64 refinement step on an n^3 grid of the
    channelized recipe, with BF16 records and with FP32 records (Jacobi inner
    CG both): one refinement step per call, each call continuing from the
    previous iterate (which is what the refinement loop does)."""
    import torch
    from paper_2408_03452_gb300 import tpfa
    w = synth.channelized(seed=a.seed, n=n)
    runs = {}
    with tpfa.Context(n, n, n, device=dev) as ctx:
        ctx.set_option("precond", 1)
        ctx.set_option("max_outer", 1)
        K, mask, pD = (torch.from_numpy(w[k]).to(dev) for k in ("K", "mask", "pD"))
        coef, coef64 = ctx.build_trans(K, mask, None, 0.0)
        c16 = ctx.build_trans_bf16(K, mask, None, 0.0)
        b = ctx.build_rhs(K, mask, None, pD)
        for name, inner in (("bf16_records", c16), ("fp32_records", coef)):
            x = torch.zeros(n ** 3, dtype=torch.float64, device=dev)
            steps = []
            for _ in range(40):
                x, info = ctx.cg_solve(inner, coef64, b, x=x, tol=a.tol, maxit=a.maxit, check=False)
                steps.append({"x": x.cpu().numpy().copy(), "inner_iters": info["iters"],
                              "rel_res_fp64": info["rel_res_fp64"]})
                if info["code"] != tpfa.NOTCONV:
                    break
            runs[name] = steps
    return {"n": n, "w": w, "runs": runs, "tol": a.tol}


def refinement_errors(sg):
    """CPU-baseline leg of the channelized workload: the oracle's FP64
    solution of the same grid (Jacobi PCG to 1e-13) and the error of every
    GPU refinement step against it."""
    from oracle import oracle as O
    O.build()
    n, w = sg["n"], sg["w"]
    g = O.Grid(n, n, n)
    t = time.perf_counter()
    A = O.assemble(g, w["K"], w["mask"], 0.0)
    b = O.rhs(g, w["K"], w["mask"], None, w["pD"])
    xr, st, it, rel = O.pcg_jacobi(A, b, tol=1e-13)
    dt = time.perf_counter() - t
    nr = float(np.linalg.norm(xr))
    out = {"grid": [n, n, n], "tol": sg["tol"],
           "oracle": {"solver": "FP64 Jacobi PCG to 1e-13", "iters": it, "status": st,
                      "rel_res": rel, "seconds": dt, "cores": O.threads()}}
    for name, steps in sg["runs"].items():
        out[name] = [{"step": k + 1, "inner_iters": s_["inner_iters"],
                      "rel_res_fp64": s_["rel_res_fp64"],
                      "rel_err_vs_oracle": float(np.linalg.norm(s_["x"] - xr)) / nr}
                     for k, s_ in enumerate(steps)]
    return out


def run_learned(a, dev, rank, local, barrier):
    """Learned-preconditioner workload.  Setup (untimed): 50 lognormal
    (sigma 1.5) 64^3 realizations x 40 pairs (r_k, e_k) from plain-CG iterates,
    Adam on the blended A-norm loss with the network on the 4x coarser grid.
    Step: a held-out n^3 realization solved to FP64 relative residual tol by
    flexible CG with z = D^-1 r + c P^2 net(R^2 r, R^2 ln K).  Plain CG and Jacobi
    PCG on the same system are timed beside it."""
    import torch
    from paper_2408_03452_gb300 import learned, tpfa
    n = a.nx
    t0 = time.perf_counter()
    ds = learned.make_dataset(a.n_real, a.snaps, 64)
    P, hist = learned.train(ds, epochs=a.epochs, batch=16, lr=1e-3, levels=LEARNED_LEVELS)
    train_s = time.perf_counter() - t0
    n_pairs = len(ds.real)
    del ds
    torch.cuda.empty_cache()
    ctx = tpfa.Context(n, n, n, device=dev)
    ctx.set_option("fcg_m", LEARNED_FCG_M)
    pr = learned.Problem(ctx, 777001 + a.seed, n, 1.5)
    nn = n >> LEARNED_LEVELS  # the network runs on the 2^levels coarser grid
    net = tpfa.UNet(nn, nn, nn, device=dev)
    net.set_params(P)
    x = torch.zeros(n ** 3, dtype=torch.float64, device=dev)

    def fcg():
        x.zero_()
        _, info = ctx.fcg_solve(pr.coef, pr.coef64, pr.b, net=net, lnk=pr.lnk, x=x, tol=a.tol,
                                maxit=a.maxit)
        if info["code"] != tpfa.OK:
            raise RuntimeError(f"fcg_solve returned {info}")
        return info

    def cg(precond):
        ctx.set_option("precond", precond)
        x.zero_()
        _, info = ctx.cg_solve(pr.coef, pr.coef64, pr.b, x=x, tol=a.tol, maxit=a.maxit)
        ctx.set_option("precond", 0)
        return info

    for _ in range(a.warmup):
        fcg()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0.record(stream)
    infos = [fcg() for _ in range(a.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / a.steps
    iters = infos[-1]["iters"]
    cg(0)
    plain = cg(0)
    cg(1)
    jac = cg(1)
    # further held-out realizations (untimed by the step clock): learned vs Jacobi
    others = []
    for k in range(1, 4):
        pk = learned.Problem(ctx, 777001 + a.seed + 1000 * k, n, 1.5)
        x.zero_()
        _, fi = ctx.fcg_solve(pk.coef, pk.coef64, pk.b, net=net, lnk=pk.lnk, x=x, tol=a.tol,
                              maxit=a.maxit)
        ctx.set_option("precond", 1)
        x.zero_()
        _, ji = ctx.cg_solve(pk.coef, pk.coef64, pk.b, x=x, tol=a.tol, maxit=a.maxit)
        ctx.set_option("precond", 0)
        others.append({"seed": 777001 + a.seed + 1000 * k,
                       "unet_fcg": {"iters": fi["iters"], "s": fi["total_ms"] / 1e3,
                                    "rel_res_fp64": fi["rel_res_fp64"], "code": fi["code"],
                                    "fell_back": fi["fell_back"]},
                       "jacobi_pcg": {"iters": ji["iters"], "s": ji["total_ms"] / 1e3}})
        del pk
    # the batched form: the uneven 96-instance ensemble, with the same network
    # and with one trained on the ensemble's own distribution (sigma ~ U(0.5,
    # 2.5), Dirichlet ends on a random axis, p_hi ~ U(0.5, 2))
    ensemble = learned.evaluate_ensemble(P, seed=a.seed, levels=LEARNED_LEVELS,
                                         fcg_m=LEARNED_FCG_M, tol=a.tol)
    t1 = time.perf_counter()
    ds_mix = learned.make_dataset(a.n_real, a.snaps, 64, mixed=True)
    P_mix, hist_mix = learned.train(ds_mix, epochs=a.epochs, batch=16, lr=1e-3,
                                    levels=LEARNED_LEVELS)
    mix_s = time.perf_counter() - t1
    del ds_mix
    torch.cuda.empty_cache()
    ens_mix = learned.evaluate_ensemble(P_mix, seed=a.seed, levels=LEARNED_LEVELS,
                                        fcg_m=LEARNED_FCG_M, tol=a.tol)
    ensemble["unet_fcg_batched_mixed_training"] = dict(
        ens_mix["unet_fcg_batched"], training_s=mix_s,
        final_val_loss=hist_mix["val_loss"][-1], jacobi_loss=hist_mix["jacobi_loss"])
    apply = learned.apply_bench(nn, 10)
    conv_ms = time_conv(tpfa, dev, nn, 16, 16)
    # the operator application: two per FCG iteration, the largest kernel time
    pv = torch.rand(n ** 3, dtype=torch.float32, device=dev)
    av = torch.empty_like(pv)
    for _ in range(3):
        ctx.apply(pr.coef, pv, av)
    stream = torch.cuda.current_stream(dev)
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e2.record(stream)
    for _ in range(10):
        ctx.apply(pr.coef, pv, av)
    e3.record(stream)
    torch.cuda.synchronize()
    apply_ms = e2.elapsed_time(e3) / 10
    if rank == 0:
        cells = n ** 3
        tpeak, tkind = measured_tensor_peak()
        hpeak, hkind = measured_hbm_peak()
        flop = 2 * 27 * 16 * 16 * nn ** 3
        achieved = flop / (conv_ms / 1e3) / 1e12
        out = {
            "metric": LEARNED_METRIC, "value": cells * iters / (ms / 1e3), "unit": LEARNED_UNIT,
            "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16-net/f32-fcg/f64-refine", "data": "synthetic",
            "config": {
                "workload": (f"learned preconditioner: U-Net trained at 64^3 on {n_pairs} plain-CG "
                             f"pairs, applied on the {2 ** LEARNED_LEVELS}x coarser grid inside flexible CG "
                             f"(m = {LEARNED_FCG_M}, "
                             f"Jacobi blend) on a held-out {n}^3 lognormal sigma-1.5 "
                             f"realization with Dirichlet x ends, FP64 relative residual "
                             f"{a.tol:g}"),
                "time_to_tol_s": {"unet_fcg": ms / 1e3, "plain_cg": plain["total_ms"] / 1e3,
                                  "jacobi_pcg": jac["total_ms"] / 1e3},
                "iters": {"unet_fcg": iters, "plain_cg": plain["iters"],
                          "jacobi_pcg": jac["iters"]},
                "rel_res_fp64": {"unet_fcg": infos[-1]["rel_res_fp64"],
                                 "plain_cg": plain["rel_res_fp64"],
                                 "jacobi_pcg": jac["rel_res_fp64"]},
                "fell_back": infos[-1]["fell_back"],
                "other_realizations": others,
                "ensemble": ensemble,
                "unet_apply_ms": apply["apply_ms"], "unet_grid": [nn, nn, nn],
                "unet_flop_per_cell": UNET_FLOP_PER_CELL,
                "training": {"pairs": n_pairs, "epochs": a.epochs, "steps": hist["steps"],
                             "seconds": train_s, "final_train_loss": hist["epoch_loss"][-1],
                             "final_val_loss": hist["val_loss"][-1],
                             "jacobi_loss": hist["jacobi_loss"]},
                "l2": "inputs larger than L2 (no flush needed)"},
            "roofline": {"kernel": "operator application A p (tpfa_apply, two per FCG "
                                   "iteration)", "bound": "hbm",
                         "apply_kernel": ("TMA-staged" if ctx.tiling(2)["kernel"] == 2
                                          else "cp.async-staged"),
                         "achieved": APPLY_BYTES_PER_CELL * cells / (apply_ms / 1e3) / 1e9,
                         "peak": hpeak, "unit": "GB/s",
                         "frac": APPLY_BYTES_PER_CELL * cells / (apply_ms / 1e3) / 1e9 / hpeak,
                         "peak_source": hkind, "bytes_per_cell": APPLY_BYTES_PER_CELL,
                         "launch_ms": apply_ms,
                         "traffic": (kernel_traffic("apply_tma_traffic.json", cells)
                                     if ctx.tiling(2)["kernel"] == 2 else None)},
            "roofline_network": {"kernel": f"tensor-core 3x3x3 convolution 16->16 on the "
                                           f"network's finest level ({nn}^3)",
                                 "bound": "tensor", "achieved": achieved, "peak": tpeak,
                                 "unit": "TFLOP/s", "frac": achieved / tpeak,
                                 "peak_source": tkind, "flop_per_launch": flop,
                                 "launch_ms": conv_ms},
            "gpu_launches": int(sum(i["kernel_launches"] for i in infos)),
            "clocks": clk,
        }
        if not a.no_cpu:
            out["cpu_baseline"] = cpu_baseline(workload="learned")
        print(json.dumps(out))


def run_ensemble(a, dev, rank, world, local, barrier):
    """Batched-ensemble step: build + batched CG solve of every instance."""
    import torch
    from paper_2408_03452_gb300 import autotune, tpfa

    ens = synth.ensemble(seed=a.seed, n_inst=a.n_inst)
    grids = [(w["nx"], w["ny"], w["nz"]) for w in ens]
    cells = [w["nx"] * w["ny"] * w["nz"] for w in ens]
    host = {k: torch.from_numpy(np.concatenate([w[k] for w in ens])).pin_memory()
            for k in ("K", "mask", "pD")}
    inp = {k: v.to(dev) for k, v in host.items()}
    with tpfa.BatchContext(grids) as bc0:
        coef, coef64 = bc0.build_trans(inp["K"], inp["mask"], None, 0.0)
        b = bc0.build_rhs(inp["K"], inp["mask"], None, inp["pD"])
        bc0.set_option("precond", a.precond)
        zc_auto = bc0.zc
    shape = ({"sweep": 0, "tile": 0, "zc": zc_auto} if a.no_autotune else
             autotune.tune_batch(grids, coef, coef64, b, tol=a.tol, maxit=a.maxit,
                                 precond=a.precond))
    zc = shape["zc"]
    bc = tpfa.BatchContext(grids, zc=zc, device=dev)
    bc.set_option("precond", a.precond)
    bc.set_option("sweep", shape["sweep"])
    bc.set_option("tma_tile", shape["tile"])
    x = torch.empty(bc.n, dtype=torch.float64, device=dev)

    def step(d):
        c, c64 = bc.build_trans(d["K"], d["mask"], None, 0.0)
        rhs = bc.build_rhs(d["K"], d["mask"], None, d["pD"])
        x.zero_()
        _, per, tot = bc.cg_solve(c, c64, rhs, x=x, tol=a.tol, maxit=a.maxit)
        if tot["code"] not in ((0, 1) if a.allow_notconv else (0,)):
            raise RuntimeError(f"cg_solve_batch returned {tot}")
        return per, tot

    for _ in range(a.warmup):
        step(inp)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0.record(stream)
    res = [step(inp) for _ in range(a.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    units = sum(sum(c * p["iters"] for c, p in zip(cells, per)) for per, _ in res)
    inner_ms = sum(t["inner_ms"] for _, t in res)
    launches = sum(2 * len(ens) + t["kernel_launches"] for _, t in res)  # builds + solve

    e2e = None
    if a.e2e_steps > 0:
        x_host = torch.empty(bc.n, dtype=torch.float64).pin_memory()
        dev_in = {k: torch.empty_like(v) for k, v in inp.items()}
        barrier()
        torch.cuda.synchronize()
        e2 = torch.cuda.Event(enable_timing=True)
        e3 = torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        e2e_units = 0
        for _ in range(a.e2e_steps):
            for k, v in host.items():
                dev_in[k].copy_(v, non_blocking=True)
            per, _ = step(dev_in)
            e2e_units += sum(c * p["iters"] for c, p in zip(cells, per))
            x_host.copy_(x, non_blocking=True)
        e3.record(stream)
        torch.cuda.synchronize()
        barrier()
        e2e = (e2e_units, e2.elapsed_time(e3))

    single_ms = None
    if a.compare_single:
        torch.cuda.synchronize()
        e4 = torch.cuda.Event(enable_timing=True)
        e5 = torch.cuda.Event(enable_timing=True)
        e4.record(stream)
        for i, w in enumerate(ens):
            with tpfa.Context(*grids[i], device=dev) as ctx:
                ctx.set_option("precond", a.precond)
                o0, o1 = bc.offsets[i], bc.offsets[i + 1]
                c, c64 = ctx.build_trans(inp["K"][o0:o1], inp["mask"][o0:o1], None, 0.0)
                rhs = ctx.build_rhs(inp["K"][o0:o1], inp["mask"][o0:o1], None, inp["pD"][o0:o1])
                ctx.cg_solve(c, c64, rhs, tol=a.tol, maxit=a.maxit)
        e5.record(stream)
        torch.cuda.synchronize()
        single_ms = e4.elapsed_time(e5)

    ms_max, units_all, e2e_ms_max, e2e_units_all = combine_ranks(
        ms, units, e2e[1] if e2e else 0.0, e2e[0] if e2e else 0.0, dev)
    if rank == 0:
        per, tot = res[-1]
        peak, peak_kind = measured_hbm_peak()
        achieved = SWEEP_BYTES_PER_CELL * units / a.steps / (inner_ms / a.steps / 1e3) / 1e9
        out = {
            "metric": METRIC, "value": units_all / (ms_max / 1e3), "unit": UNIT,
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms_max / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_desc(a), "instances": len(ens),
                       "cells": int(sum(cells)), "tol": a.tol,
                       "parallelism": f"replicas{world}",
                       "precond": ["none", "jacobi"][a.precond],
                       "zc_per_size": {f"{g[0]}x{g[1]}x{g[2]}": z for g, z in zip(grids, zc)},
                       "sweep_kernel": ["TMA-staged", "cp.async-staged"][shape["sweep"]],
                       "tma_tile": shape["tile"],
                       "autotuned": not a.no_autotune,
                       "iters_min_max": [min(p["iters"] for p in per), max(p["iters"] for p in per)],
                       "time_to_tol_s": ms / 1e3 / a.steps,
                       "rel_res_fp64_max": tot["rel_res_fp64"],
                       "single_solves_s": None if single_ms is None else single_ms / 1e3,
                       "l2": "inputs larger than L2 (no flush needed)"},
            "roofline": {"kernel": "batched cg sweep", "bound": "hbm", "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_source": peak_kind, "bytes_per_cell": SWEEP_BYTES_PER_CELL,
                         "traffic": None},
            "gpu_launches": launches,
            "clocks": clk,
        }
        if e2e:
            out["e2e"] = {"value": e2e_units_all / (e2e_ms_max / 1e3), "unit": UNIT,
                          "h2d_bytes_per_step": int(sum(v.numel() * v.element_size()
                                                        for v in host.values())),
                          "d2h_bytes_per_step": int(bc.n * 8), "steps": a.e2e_steps}
        if not a.no_cpu:
            out["cpu_baseline"] = cpu_baseline(workload="paper")
        print(json.dumps(out))
    bc.close()


def cell_updates_per_s(cells, iterations, ms):
    """The paper's throughput definition (Table III): cells x iterations / time."""
    return cells * iterations / (ms / 1e3)


def combine_ranks(ms, iters, e2e_ms, e2e_iters, device):
    """Whole-job figures over the replicas: the slowest rank's time and the
    sum of every rank's iterations.  One process per GPU; without an
    initialised process group this is the identity."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms, iters, e2e_ms, e2e_iters
    t = torch.tensor([ms, iters, e2e_ms, e2e_iters], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return tmax[0].item(), t[1].item(), tmax[2].item(), t[3].item()


def main():
    a = finish_args(parse())
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank, world)
        return

    import torch
    import torch.distributed as dist
    from paper_2408_03452_gb300 import tpfa

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    if a.workload == "table3":
        run_table3(a, dev, rank)
        return
    if a.workload == "ensemble":
        run_ensemble(a, dev, rank, world, local, barrier)
        if world > 1:
            dist.destroy_process_group()
        return
    if a.workload == "learned":
        run_learned(a, dev, rank, local, barrier)
        if world > 1:
            dist.destroy_process_group()
        return

    nx, ny, nz = a.nx, a.ny, a.nz
    n = nx * ny * nz
    if a.workload == "channelized":
        if not (nx == ny == nz):
            raise SystemExit("the channelized workload is cubic: give nx = ny = nz")
        w = synth.channelized(seed=a.seed, n=nx)
    else:
        w = synth.paper_scale(seed=a.seed, nx=nx, ny=ny, nz=nz)
    # host inputs (pinned) and their device copies
    host = {"K": torch.from_numpy(w["K"]).pin_memory(),
            "si": torch.from_numpy(w["src_idx"]).pin_memory(),
            "sv": torch.from_numpy(w["src_val"]).pin_memory()}
    if w["mask"] is not None:
        host["mask"] = torch.from_numpy(w["mask"]).pin_memory()
        host["pD"] = torch.from_numpy(w["pD"]).pin_memory()
    d0 = w["d"]
    inp = {k: v.to(dev) for k, v in host.items()}

    ctx = tpfa.Context(nx, ny, nz, device=dev)
    if a.tile_vy:
        ctx.set_option("tile_vy", a.tile_vy)
    if a.stages:
        ctx.set_option("stages", a.stages)
    if a.tile_zc >= 0:
        ctx.set_option("tile_zc", a.tile_zc)
    ctx.set_option("loop", a.loop)
    ctx.set_option("sweep", a.sweep)
    if a.tma_tile >= 0:
        ctx.set_option("tma_tile", a.tma_tile)
    ctx.set_option("precond", a.precond)
    coef = torch.empty((n, 4), dtype=torch.float32, device=dev)
    coef64 = torch.empty((n, 4), dtype=torch.float64, device=dev)
    coef16 = torch.empty((n, 4), dtype=torch.int16, device=dev) if a.inner == "bf16" else None
    b = torch.empty(n, dtype=torch.float64, device=dev)
    x = torch.empty(n, dtype=torch.float64, device=dev)

    def build(d):
        ctx.build_trans(d["K"], d.get("mask"), None, d0, coef=coef, coef64=coef64)
        if coef16 is not None:
            ctx.build_trans_bf16(d["K"], d.get("mask"), None, d0, coef16=coef16)
        ns = d["si"].numel()
        ctx.build_rhs(d["K"], d.get("mask"), None, d.get("pD"), d["si"] if ns else None,
                      d["sv"] if ns else None, b=b)
        x.zero_()
        return coef16 if coef16 is not None else coef

    def step(d):
        inner = build(d)
        _, info = ctx.cg_solve(inner, coef64, b, x=x, tol=a.tol, maxit=a.maxit)
        if info["code"] not in ((0, 1) if a.allow_notconv else (0,)):
            raise RuntimeError(f"cg_solve returned {info}")
        return info

    builds_per_step = 3 + (1 if coef16 is not None else 0)
    K = inp["K"]

    if a.probe_apply > 0:
        inner = build(inp)
        pv = torch.rand(ctx.n, dtype=torch.float32, device=dev)
        av = torch.empty_like(pv)
        pAp = torch.zeros(1, dtype=torch.float64, device=dev)
        fn = ctx.apply_bf16 if coef16 is not None else ctx.apply
        for _ in range(a.probe_apply):
            fn(inner, pv, Ap=av, pAp=pAp)
        torch.cuda.synchronize()
        print(json.dumps({"probe_apply": a.probe_apply, "pAp": pAp.item(),
                          "tiling": ctx.tiling(3 if coef16 is not None else 2)}))
        ctx.close()
        return

    if a.probe_iters > 0:
        ctx.set_option("loop", 1)
        ctx.set_option("chunk", 4)
        inner = build(inp)
        _, info = ctx.cg_solve(inner, coef64, b, x=x, tol=a.tol, maxit=a.probe_iters, check=False)
        torch.cuda.synchronize()
        print(json.dumps({"probe": info}))
        ctx.close()
        return

    for _ in range(a.warmup):
        step(inp)
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0.record(stream)
    infos = [step(inp) for _ in range(a.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    iters = sum(i["iters"] for i in infos)
    launches = sum(builds_per_step + i["kernel_launches"] for i in infos)
    inner_ms = sum(i["inner_ms"] for i in infos)

    # end to end through the public API with host buffers: H2D of the step's
    # inputs, the solve, D2H of the solution
    e2e = None
    if a.e2e_steps > 0:
        x_host = torch.empty(n, dtype=torch.float64).pin_memory()
        dev_in = {k: torch.empty_like(v) for k, v in inp.items()}
        barrier()
        torch.cuda.synchronize()
        e2 = torch.cuda.Event(enable_timing=True)
        e3 = torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        e2e_iters = 0
        for _ in range(a.e2e_steps):
            for k, v in host.items():
                dev_in[k].copy_(v, non_blocking=True)
            info = step(dev_in)
            e2e_iters += info["iters"]
            x_host.copy_(x, non_blocking=True)
        e3.record(stream)
        torch.cuda.synchronize()
        barrier()
        e2e = (e2e_iters, e2.elapsed_time(e3))

    ms_max, iters_all, e2e_ms_max, e2e_iters_all = combine_ranks(
        ms, iters, e2e[1] if e2e else 0.0, e2e[0] if e2e else 0.0, dev)
    tiling = ctx.tiling(1 if coef16 is not None else 0)

    # beside the timed steps (their clock has stopped): the metric's
    # time-to-1e-8 comparison, and for the mixed-precision workload the
    # other record type and the per-refinement-step errors
    extras, steps_gpu = {}, None
    if rank == 0 and a.workload == "paper" and not a.no_ttt:
        extras["time_to_1e8"] = time_to_1e8(dev, a.seed)
    if rank == 0 and a.workload == "channelized":
        other = "f32" if a.inner == "bf16" else "bf16"
        oc = coef if other == "f32" else ctx.build_trans_bf16(K, inp.get("mask"), None, d0)
        cmp = {}
        for rep in range(2):
            x.zero_()
            _, oi = ctx.cg_solve(oc, coef64, b, x=x, tol=a.tol, maxit=a.maxit, check=False)
        cmp[other + "_records"] = {"time_to_tol_s": oi["total_ms"] / 1e3, "iters": oi["iters"],
                                   "refinements": oi["outer"], "rel_res_fp64": oi["rel_res_fp64"],
                                   "converged": oi["code"] == 0,
                                   "sweep_ms": oi["inner_ms"] / max(oi["iters"], 1)}
        extras["other_records"] = cmp
        if not a.no_cpu:
            steps_gpu = channelized_steps(a, dev)

    if rank == 0:
        value = cell_updates_per_s(n, iters_all, ms_max)
        peak, peak_kind = measured_hbm_peak()
        sweep_ms = inner_ms / max(iters, 1)
        # BF16 records save 8 B/cell; with Jacobi they need the 4 B/cell M^-1 array
        bpc = SWEEP_BYTES_PER_CELL - (8 if coef16 is not None else 0) + \
            (4 if coef16 is not None and a.precond else 0)
        algo = bpc * n
        achieved = algo / (sweep_ms / 1e3) / 1e9
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if coef16 is None else "bf16-coef/f32", "data": "synthetic",
            "config": {"workload": workload_desc(a), "nx": nx, "ny": ny, "nz": nz,
                       "tol": a.tol, "parallelism": f"replicas{world}",
                       "inner": a.inner, "precond": ["none", "jacobi"][a.precond],
                       "l2": "inputs larger than L2 (no flush needed)",
                       "iters_per_solve": iters / a.steps,
                       "time_to_tol_s": ms / 1e3 / a.steps,
                       "rel_res_fp64": infos[-1]["rel_res_fp64"],
                       "converged": all(i["code"] == 0 for i in infos),
                       "refinements": infos[-1]["outer"]},
            "roofline": {"kernel": "cg sweep (fused CG iteration)", "bound": "hbm",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": peak_kind,
                         "nominal_peak": NOMINAL_HBM_GBS,
                         "frac_nominal": achieved / NOMINAL_HBM_GBS,
                         "sweep_kernel": ["", "cp.async-staged", "TMA-staged"][tiling["kernel"]],
                         "tiling": tiling,
                         "bytes_per_cell": bpc, "sweep_ms": sweep_ms,
                         "traffic": (sweep_traffic(nx, ny, nz)
                                     if (coef16 is None and a.precond == 0 and tiling["kernel"] == 2)
                                     else None)},
            "gpu_launches": launches,
        }
        if e2e:
            out["e2e"] = {"value": n * e2e_iters_all / (e2e_ms_max / 1e3), "unit": UNIT,
                          "h2d_bytes_per_step": int(sum(v.numel() * v.element_size()
                                                        for v in host.values())),
                          "d2h_bytes_per_step": int(n * 8), "steps": a.e2e_steps}
        out["clocks"] = clk
        if extras:
            out["config"].update(extras)
        if not a.no_cpu:
            out["cpu_baseline"] = cpu_baseline(workload=a.workload)
            if a.workload == "paper" and a.window:
                out["cpu_baseline"]["full_grid_window"] = oracle_window_estimate(w)
            if a.workload == "channelized" and steps_gpu is not None:
                out["config"]["refinement_steps"] = refinement_errors(steps_gpu)
        print(json.dumps(out))
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
