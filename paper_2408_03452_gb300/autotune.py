"""Autotuner for the z-run length of batched sweeps.

The sweep tiles each instance into warps of 30 x 4 columns marching through
runs of zc planes.  Long runs re-read fewer halo planes; short runs give more
warps (better occupancy and load balance for small instances).  The best
choice depends on the mix of instance sizes and on how long each instance
keeps iterating (near the end of a batched solve only the slowest instances
run, and they need short runs to fill the GPU), so it is measured on the
real solve: first one common zc for the whole batch, then each size class on
its own (halved or doubled while the others stay fixed).  Each candidate is
timed with CUDA events over a complete batched solve to the target
tolerance.  Results can be cached in a JSON file keyed by the device name and
the size mix.
"""
from __future__ import annotations

import json
import os

import torch

from . import tpfa

CANDIDATES = (4, 8, 16, 32, 64, 128)


def _time_batch(grids, zc, coef, coef64, b, tol, maxit, precond):
    with tpfa.BatchContext(grids, zc=zc) as bc:
        bc.set_option("precond", precond)
        x = torch.zeros(bc.n, dtype=torch.float64, device=coef.device)
        bc.cg_solve(coef, coef64, b, x=x, tol=tol, maxit=maxit, check=False)  # warm up
        x.zero_()
        _, _, tot = bc.cg_solve(coef, coef64, b, x=x, tol=tol, maxit=maxit, check=False)
        return tot["total_ms"]


def _key(grids, precond, tol):
    sizes = sorted({tuple(g[:3]) for g in grids})
    counts = {s: sum(1 for g in grids if tuple(g[:3]) == s) for s in sizes}
    name = torch.cuda.get_device_name()
    return json.dumps([name, precond, tol, [[list(s), counts[s]] for s in sizes]])


def tune(grids, coef, coef64, b, tol=1e-8, maxit=100000, precond=0, cache=None, log=None):
    """Per-instance zc for a batch (list of ints).  grids: list of (nx, ny, nz)
    tuples; coef, coef64, b: the batch's concatenated records and rhs; the
    candidates are compared on the time of the whole solve to `tol`."""
    key = _key(grids, precond, tol)
    if cache and os.path.exists(cache):
        try:
            db = json.load(open(cache))
            if key in db:
                by = {tuple(k): v for k, v in db[key]["zc"]}
                return [by[tuple(g[:3])] for g in grids]
        except (OSError, ValueError, KeyError):
            pass
    classes = sorted({tuple(g[:3]) for g in grids})
    timings = {}

    def run(assign):
        zc = [assign[tuple(g[:3])] for g in grids]
        t = _time_batch(grids, zc, coef, coef64, b, tol, maxit, precond)
        timings[json.dumps(sorted((list(k), v) for k, v in assign.items()))] = t
        if log:
            log(f"zc {assign} -> {t:.2f} ms per solve")
        return t

    best_t, best = None, None
    for z in CANDIDATES:
        assign = {c: z for c in classes}
        t = run(assign)
        if best_t is None or t < best_t:
            best_t, best = t, dict(assign)
    for c in classes:
        for z in (best[c] // 2, best[c] * 2):
            if z < 1 or z > 256:
                continue
            trial = dict(best)
            trial[c] = z
            t = run(trial)
            if t < best_t:
                best_t, best = t, trial
    if cache:
        try:
            db = json.load(open(cache)) if os.path.exists(cache) else {}
        except (OSError, ValueError):
            db = {}
        db[key] = {"zc": [[list(k), v] for k, v in best.items()], "ms_per_solve": best_t}
        tmp = cache + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1)
        os.replace(tmp, cache)
    return [best[tuple(g[:3])] for g in grids]
