"""Autotuner for the tiling of batched sweeps.

The batched CG sweep tiles each instance into blocks that march through runs
of zc planes.  Long runs re-read fewer halo planes; short runs give more
blocks (better occupancy and load balance for small instances).  The TMA-
staged sweep also has a tile shape (compute warps x rows per warp x stages,
`tpfa.OPTIONS["tma_tile"]`), and the cp.async-staged sweep is the
alternative kernel.  The best choice depends on the mix of instance sizes and
on how long each instance keeps iterating (near the end of a batched solve
only the slowest instances run, and they need short runs to fill the GPU),
so it is measured on the real solve:
  1. one common zc for the whole batch (TMA sweep, tile 0);
  2. at that zc, the other tile shapes (plain CG; the Jacobi variant has one)
     and the cp.async sweep;
  3. each size class on its own, halved or doubled while the others stay
     fixed.
Each candidate is timed with CUDA events over a complete batched solve to the
target tolerance.  Results can be cached in a JSON file keyed by the device
name, the preconditioner, the tolerance and the size mix.
"""
from __future__ import annotations

import json
import os

import torch

from . import tpfa

CANDIDATES = (4, 8, 16, 32, 64, 128)
TMA_TILES = (0, 1, 2, 3)


def _time_batch(grids, zc, coef, coef64, b, tol, maxit, precond, sweep=0, tile=0):
    with tpfa.BatchContext(grids, zc=zc) as bc:
        bc.set_option("precond", precond)
        bc.set_option("sweep", sweep)
        bc.set_option("tma_tile", tile)
        x = torch.zeros(bc.n, dtype=torch.float64, device=coef.device)
        bc.cg_solve(coef, coef64, b, x=x, tol=tol, maxit=maxit, check=False)  # warm up
        x.zero_()
        _, _, tot = bc.cg_solve(coef, coef64, b, x=x, tol=tol, maxit=maxit, check=False)
        return tot["total_ms"]


def _key(grids, precond, tol, what):
    sizes = sorted({tuple(g[:3]) for g in grids})
    counts = {s: sum(1 for g in grids if tuple(g[:3]) == s) for s in sizes}
    name = torch.cuda.get_device_name()
    return json.dumps([name, precond, tol, [[list(s), counts[s]] for s in sizes]] +
                      ([what] if what else []))


def _load(cache, key):
    if cache and os.path.exists(cache):
        try:
            return json.load(open(cache)).get(key)
        except (OSError, ValueError):
            return None
    return None


def _store(cache, key, rec):
    if not cache:
        return
    try:
        db = json.load(open(cache)) if os.path.exists(cache) else {}
    except (OSError, ValueError):
        db = {}
    db[key] = rec
    tmp = cache + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(db, f, indent=1)
    os.replace(tmp, cache)


def tune_batch(grids, coef, coef64, b, tol=1e-8, maxit=100000, precond=0, cache=None, log=None,
               kernels=True):
    """Tiling of a batch: {"sweep": 0 (TMA) or 1 (cp.async), "tile": TMA tile,
    "zc": per-instance z-run, "ms_per_solve": time of the chosen one}.
    grids: list of (nx, ny, nz); coef, coef64, b: the batch's concatenated
    records and right-hand side.  kernels=False keeps the default kernel and
    tile and tunes zc only."""
    key = _key(grids, precond, tol, "kernels" if kernels else "")
    hit = _load(cache, key)
    if hit is not None:
        try:
            by = {tuple(k): v for k, v in hit["zc"]}
            return {"sweep": int(hit.get("sweep", 0)), "tile": int(hit.get("tile", 0)),
                    "zc": [by[tuple(g[:3])] for g in grids],
                    "ms_per_solve": hit.get("ms_per_solve")}
        except (KeyError, TypeError, ValueError):
            pass
    classes = sorted({tuple(g[:3]) for g in grids})

    def run(assign, sweep, tile):
        zc = [assign[tuple(g[:3])] for g in grids]
        t = _time_batch(grids, zc, coef, coef64, b, tol, maxit, precond, sweep=sweep, tile=tile)
        if log:
            log(f"sweep {sweep} tile {tile} zc {assign} -> {t:.2f} ms per solve")
        return t

    best_t, best, bs, bt = None, None, 0, 0
    for z in CANDIDATES:
        assign = {c: z for c in classes}
        t = run(assign, 0, 0)
        if best_t is None or t < best_t:
            best_t, best = t, dict(assign)
    if kernels:
        shapes = [(0, tl) for tl in (TMA_TILES[1:] if not precond else ())] + [(1, 0)]
        for sw, tl in shapes:
            t = run(best, sw, tl)
            if t < best_t:
                best_t, bs, bt = t, sw, tl
    for c in classes:
        for z in (best[c] // 2, best[c] * 2):
            if z < 1 or z > 256:
                continue
            trial = dict(best)
            trial[c] = z
            t = run(trial, bs, bt)
            if t < best_t:
                best_t, best = t, trial
    _store(cache, key, {"zc": [[list(k), v] for k, v in best.items()], "sweep": bs, "tile": bt,
                        "ms_per_solve": best_t})
    return {"sweep": bs, "tile": bt, "zc": [best[tuple(g[:3])] for g in grids],
            "ms_per_solve": best_t}


def tune(grids, coef, coef64, b, tol=1e-8, maxit=100000, precond=0, cache=None, log=None):
    """Per-instance zc for a batch (list of ints), default kernel and tile
    (the search of tune_batch without step 2)."""
    return tune_batch(grids, coef, coef64, b, tol, maxit, precond, cache, log, kernels=False)["zc"]
