"""Learned preconditioner: training pairs from plain CG, training of the
U-Net with the A-norm loss and Adam, and evaluation inside flexible CG.

Every numerical step runs in the library's kernels through the C ABI
(tpfa.py); torch only holds the buffers and gathers samples into batches.

Training data.  For each lognormal realization (ln K ~ N(0, sigma^2) i.i.d.
per cell, Dirichlet p = 1 / 0 on the x = 0 / x = n-1 layers) plain CG is run
once to tol (x*) and then stopped after k iterations for a geometric range
of k; each stop gives the pair (r_k, e_k) = (b - A x_k, x* - x_k), which
satisfies A e_k = r_k -- the residuals plain CG itself generates (k = 0 gives
(b, x*)).

The network output u enters the preconditioner as the Jacobi blend
z = D^-1 r + c u with the A-norm-optimal weight c (flexible CG in the
library).  By default the network runs on the 4x coarser grid,
u = P^2 net(R^2 r, R^2 ln K) (levels = 2): Jacobi takes the high frequencies,
the network the smooth error CG is slow on, at 1/64 of the full-grid cost.  Loss: the A-norm error of that blend relative to ||e||_A,
  min_c ||D^-1 r + c u - e||_A^2 / ||e||_A^2 = (w'Aw - (u's)^2 / (u'Au)) / (e'Ae),
w = e - D^-1 r, s = A w = r - A D^-1 r, per sample, summed over the batch
(Adam is invariant to a constant factor).  Minimising over the weight makes
the loss blind to the scale of u, as CG is to the scale of its
preconditioner; without it an untrained network is driven to u = 0, because
e = A^-1 r is orders of magnitude larger than r.
"""
from __future__ import annotations

import json
import time

import numpy as np
import torch

from . import synth, tpfa

LAYERS = [(2, 16), (16, 32), (32, 64), (64, 32), (32, 16), (16, 16), (16, 1)]
STREAM_INIT = 40


def init_params(seed: int) -> torch.Tensor:
    """He-style initial weights N(0, 2/(27 cin)) from the counter-based
    generator, zero biases, in the library's flat layout."""
    flat = []
    for i, (cin, cout) in enumerate(LAYERS):
        nw = 27 * cout * cin
        w = synth.normal(seed, STREAM_INIT + i, np.arange(nw)) * np.sqrt(2.0 / (27 * cin))
        flat += [w, np.zeros(cout)]
    p = np.concatenate(flat).astype(np.float32)
    if p.size != tpfa.unet_param_count():
        raise RuntimeError("parameter layout does not match the library")
    return torch.from_numpy(p)


STREAM_TRAIN_MIX = 41


def realization(seed: int, n: int, sigma: float, axis: str = "x", p_hi: float = 1.0):
    K = synth.lognormal_field(n, n, n, sigma, seed)
    mask, pD = synth.dirichlet_faces(n, n, n, axis, p_hi, 0.0)
    return K, mask, pD


def mixed_draw(seed: int, sigma_range=(0.5, 2.5)):
    """sigma ~ U(sigma_range), Dirichlet axis from {x, y, z}, p_hi ~ U(0.5, 2):
    the distribution the batched ensemble draws its instances from."""
    u = synth.uniform(seed, STREAM_TRAIN_MIX, np.arange(3, dtype=np.uint64))
    sigma = sigma_range[0] + (sigma_range[1] - sigma_range[0]) * float(u[0])
    return sigma, "xyz"[min(int(u[1] * 3), 2)], 0.5 + 1.5 * float(u[2])


class Problem:
    """One realization on the GPU: coefficients, right-hand side, ln K."""

    def __init__(self, ctx: tpfa.Context, seed: int, n: int, sigma: float, axis: str = "x",
                 p_hi: float = 1.0):
        dev = ctx.device
        K, mask, pD = realization(seed, n, sigma, axis, p_hi)
        Kd = torch.from_numpy(K).to(dev)
        md = torch.from_numpy(mask).to(dev)
        self.coef, self.coef64 = ctx.build_trans(Kd, md)
        self.b = ctx.build_rhs(Kd, md, pD=torch.from_numpy(pD).to(dev))
        self.lnk = tpfa.log_perm(Kd)


class Dataset:
    def __init__(self, n: int):
        self.n = n
        self.R, self.E, self.S, self.eae, self.wAw, self.real = [], [], [], [], [], []
        self.problems: list[Problem] = []

    def finish(self):
        n = self.n
        # ln K on the 2x, 4x and 8x coarser grids
        self.lnk_l = [None]
        cur = [pr.lnk for pr in self.problems]
        for l in range(1, 4):
            m = n >> (l - 1)
            cur = [tpfa.restrict2(c, (m, m, m, 1)) for c in cur]
            self.lnk_l.append(torch.stack(cur))
        self.R = torch.stack(self.R)
        self.E = torch.stack(self.E)
        self.S = torch.stack(self.S)
        self.eae = torch.cat(self.eae)
        self.wAw = torch.cat(self.wAw)
        self.real = np.asarray(self.real)
        self.lnk = torch.stack([p.lnk for p in self.problems])


def make_dataset(n_real=50, snaps=40, n=64, sigma=1.5, seed=1000, tol=1e-10, log=None,
                 mixed=False):
    """n_real realizations x snaps pairs (r_k, e_k) from plain CG.  mixed:
    each realization draws sigma, the Dirichlet axis and p_hi as the batched
    ensemble does (mixed_draw) instead of sigma with Dirichlet x ends."""
    ctx = tpfa.Context(n, n, n)
    ctx.set_option("precond", 0)
    ds = Dataset(n)
    ds.ctx = ctx
    t0 = time.perf_counter()
    for q in range(n_real):
        if mixed:
            pr = Problem(ctx, seed + q, n, *mixed_draw(seed + q))
        else:
            pr = Problem(ctx, seed + q, n, sigma)
        ds.problems.append(pr)
        xs, info = ctx.cg_solve(pr.coef, pr.coef64, pr.b, tol=tol, maxit=100000)
        if info["code"] != tpfa.OK:
            raise RuntimeError(f"training solve did not converge: {info}")
        caps = np.unique(np.geomspace(1, 0.9 * info["iters"], snaps - 1).astype(int))
        ks = [0] + [int(k) for k in caps]
        while len(ks) < snaps:  # small iteration counts: repeat late snapshots
            ks.append(int(caps[-1]))
        for k in ks[:snaps]:
            if k == 0:
                r64, e64 = pr.b, xs
            else:
                xk, _ = ctx.cg_solve(pr.coef, pr.coef64, pr.b, tol=1e-14, maxit=k, check=False)
                r64 = ctx.residual64(pr.coef64, pr.b, xk)
                e64 = xs - xk
            r, e = r64.float(), e64.float()
            eae = torch.zeros(1, dtype=torch.float64, device=ctx.device)
            ctx.apply(pr.coef, e, pAp=eae)
            wAw = torch.zeros(1, dtype=torch.float64, device=ctx.device)
            s = ctx.jacobi_split(pr.coef, r, e=e, wAw=wAw)
            ds.R.append(r)
            ds.E.append(e)
            ds.S.append(s)
            ds.eae.append(eae)
            ds.wAw.append(wAw)
            ds.real.append(q)
        if log:
            log(f"realization {q}: {info['iters']} CG iterations, {len(ks[:snaps])} pairs, "
                f"{time.perf_counter() - t0:.1f} s")
    ds.finish()
    return ds


def restrict_to(v, n, batch, levels, scale=0.125):
    """levels applications of the 2x restriction to batch samples of n^3."""
    for l in range(levels):
        m = n >> l
        v = tpfa.restrict2(v, (m, m, m, batch), scale=scale)
    return v


def prolong_from(v, n, batch, levels):
    """levels applications of the nearest prolongation, ending on n^3."""
    for l in range(levels, 0, -1):
        m = n >> (l - 1)
        v = tpfa.prolong2(v, (m, m, m, batch))
    return v


def train(ds: Dataset, epochs=12, batch=16, lr=1e-3, seed=0, holdout=0.1, levels=2, log=None):
    """Adam on the blended A-norm loss.  levels: the network runs on the 2^levels
    coarser grid, u = P^l net(R^l r, R^l ln K) (R: 2x2x2 mean, P: nearest
    prolongation; the gradient passes back through P^T = 8 R per level).
    Returns (params, history dict)."""
    dev = ds.R.device
    n = ds.n
    N = n ** 3
    ctx = ds.ctx
    nreal = len(ds.problems)
    n_val = max(1, int(round(holdout * nreal)))
    val_real = set(range(nreal - n_val, nreal))
    idx_train = np.array([i for i in range(len(ds.real)) if ds.real[i] not in val_real])
    idx_val = np.array([i for i in range(len(ds.real)) if ds.real[i] in val_real])
    nn = n >> levels
    net = tpfa.UNet(nn, nn, nn, ns=batch, train=True, device=dev)
    P = init_params(seed).to(dev)
    M = torch.zeros_like(P)
    V = torch.zeros_like(P)
    G = torch.empty(batch * N, dtype=torch.float32, device=dev)
    q = torch.empty(N, dtype=torch.float32, device=dev)
    stats = torch.zeros((batch, 2), dtype=torch.float64, device=dev)
    hist = {"epoch_loss": [], "val_loss": [], "seconds": [], "levels": levels,
            "jacobi_loss": float((ds.wAw / ds.eae).mean().item())}
    t = 0
    t0 = time.perf_counter()

    def batch_loss(idx, backward):
        nonlocal t
        Rb = ds.R[idx].reshape(-1)
        Sb = ds.S[idx].reshape(-1)
        if levels > 0:
            Lb = ds.lnk_l[levels][ds.real[idx]].reshape(-1)
            Z = prolong_from(net.forward(restrict_to(Rb, n, batch, levels), Lb), n, batch, levels)
        else:
            Lb = ds.lnk[ds.real[idx]].reshape(-1)
            Z = net.forward(Rb, Lb)
        for j, s in enumerate(idx):
            ctx.anorm_loss_grad(ds.problems[ds.real[s]].coef, Z[j * N:(j + 1) * N],
                                Sb[j * N:(j + 1) * N], ds.eae[s:s + 1], q, G[j * N:(j + 1) * N],
                                stats[j])
        if backward:
            grad = net.backward(restrict_to(G, n, batch, levels, scale=1.0) if levels > 0 else G)
            t += 1
            tpfa.adam_step(P, grad, M, V, t, lr)
        st = stats[:len(idx)]
        return ((ds.wAw[idx] - st[:, 0] ** 2 / st[:, 1]) / ds.eae[idx]).sum().item()

    for ep in range(epochs):
        perm = np.random.default_rng(seed + 7919 * (ep + 1)).permutation(idx_train)
        tot, cnt = 0.0, 0
        for st in range(0, len(perm) - batch + 1, batch):
            net.set_params(P)
            tot += batch_loss(perm[st:st + batch], True)
            cnt += batch
        net.set_params(P)
        vt, vc = 0.0, 0
        for st in range(0, len(idx_val) - batch + 1, batch):
            vt += batch_loss(idx_val[st:st + batch], False)
            vc += batch
        tpfa.net_status(dev)
        hist["epoch_loss"].append(tot / max(cnt, 1))
        hist["val_loss"].append(vt / max(vc, 1))
        hist["seconds"].append(time.perf_counter() - t0)
        if log:
            log(f"epoch {ep}: train {hist['epoch_loss'][-1]:.4g} val {hist['val_loss'][-1]:.4g} "
                f"({hist['seconds'][-1]:.1f} s, {t} steps)")
    hist["steps"] = t
    return P, hist


def evaluate(P, n=256, sigma=1.5, seed=777001, tol=1e-8, maxit=200000, levels=2, fcg_m=2,
             log=None):
    """Plain CG, Jacobi PCG and U-Net FCG on one held-out realization."""
    ctx = tpfa.Context(n, n, n)
    pr = Problem(ctx, seed, n, sigma)
    out = {"grid": [n, n, n], "sigma": sigma, "seed": seed, "tol": tol}

    def rec(name, info):
        out[name] = {"iters": int(info["iters"]), "seconds": info["total_ms"] / 1e3,
                     "rel_res_fp64": info["rel_res_fp64"], "code": int(info["code"])}
        if "fell_back" in info:
            out[name]["fell_back"] = bool(info["fell_back"])
        if log:
            log(f"{name}: {out[name]}")

    ctx.set_option("precond", 0)
    _, info = ctx.cg_solve(pr.coef, pr.coef64, pr.b, tol=tol, maxit=maxit)
    rec("plain_cg", info)
    ctx.set_option("precond", 1)
    _, info = ctx.cg_solve(pr.coef, pr.coef64, pr.b, tol=tol, maxit=maxit)
    rec("jacobi_pcg", info)
    ctx.set_option("precond", 0)
    nn = n >> levels
    net = tpfa.UNet(nn, nn, nn, device=ctx.device)
    net.set_params(P.to(ctx.device))
    ctx.set_option("fcg_m", fcg_m)
    _, info = ctx.fcg_solve(pr.coef, pr.coef64, pr.b, net=net, lnk=pr.lnk, tol=tol, maxit=maxit)
    rec("unet_fcg", info)
    out["unet_apply_ms"] = apply_bench(nn, 10)["apply_ms"]
    out["levels"] = levels
    return out


def net_grid(shape, levels: int):
    """(l, grid) of the network for instances of `shape`: the coarsest level
    l <= levels with extents divisible by 2^l, and the network's grid, the
    2^l coarser grid with each extent rounded up to a multiple of 4 (the
    extra cells are zero padding; two poolings need multiples of 4).  At
    l = 0 no padding is allowed.  None when no level fits."""
    for l in range(levels, -1, -1):
        f = 1 << l
        if any(d % f for d in shape):
            continue
        c = [d // f for d in shape]
        if l == 0 and any(v % 4 for v in c):
            continue
        return l, tuple((v + 3) // 4 * 4 for v in c)
    return None


def ensemble_problem(P, seed: int = 0, n_inst: int = 96, levels: int = 2):
    """The ensemble of synth.ensemble on one batch object, with one network
    (parameters P) per size class on its grid from net_grid.  Returns
    (batch, coef, coef64, b, lnk, nets, net_of, grids, levels per size)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    ens = synth.ensemble(seed=seed, n_inst=n_inst)
    grids = [(w["nx"], w["ny"], w["nz"]) for w in ens]

    def cat(k):
        return torch.from_numpy(np.concatenate([w[k] for w in ens])).to(dev)

    K, mask, pD = cat("K"), cat("mask"), cat("pD")
    bc = tpfa.BatchContext(grids, device=dev)
    coef, coef64 = bc.build_trans(K, mask, None, 0.0)
    b = bc.build_rhs(K, mask, None, pD)
    lnk = tpfa.log_perm(K)
    del K, mask, pD
    classes = sorted(set(grids))
    nets, idx, lv = [], {}, {}
    for g in classes:
        ng = net_grid(g, levels)
        lv["%dx%dx%d" % g] = None if ng is None else {"level": ng[0], "net_grid": list(ng[1])}
        if ng is None:
            continue
        u = tpfa.UNet(*ng[1], ns=sum(gi == g for gi in grids), device=dev)
        u.set_params(P.to(dev))
        idx[g] = len(nets)
        nets.append(u)
    net_of = [idx.get(g, -1) for g in grids]
    return bc, coef, coef64, b, lnk, nets, net_of, grids, lv


def evaluate_ensemble(P, seed: int = 0, n_inst: int = 96, levels: int = 2, fcg_m: int = 2,
                      tol: float = 1e-8, maxit: int = 200000, log=None,
                      solvers=("unet_fcg_batched", "jacobi_pcg_batched", "plain_cg_batched")) -> dict:
    """The batched ensemble of synth.ensemble (uneven sizes, sigma ~ U(0.5, 2.5),
    Dirichlet ends on a random axis) solved to tol three ways on one batch
    object: flexible CG with the Jacobi-blended U-Net (one network per size
    class, on the coarsest suitable grid up to 2^levels coarser), Jacobi PCG
    and plain CG (cg_solve_batch).  Each solver runs once untimed, then once
    timed with CUDA events."""
    dev = torch.device("cuda", torch.cuda.current_device())
    bc, coef, coef64, b, lnk, nets, net_of, grids, lv = ensemble_problem(P, seed, n_inst, levels)
    classes = sorted(set(grids))
    bc.set_option("fcg_m", fcg_m)
    x = torch.zeros(bc.n, dtype=torch.float64, device=dev)

    def fcg():
        x.zero_()
        return bc.fcg_solve(coef, coef64, b, nets=nets, net_of=net_of, lnk=lnk, x=x, tol=tol,
                            maxit=maxit)[1:]

    def cg(precond):
        def run():
            bc.set_option("precond", precond)
            x.zero_()
            return bc.cg_solve(coef, coef64, b, x=x, tol=tol, maxit=maxit)[1:]
        return run

    out = {"instances": n_inst, "cells": bc.n, "tol": tol, "fcg_m": fcg_m,
           "sizes": {"%dx%dx%d" % g: sum(gi == g for gi in grids) for g in classes},
           "levels_per_size": lv}
    for name, fn in (("unet_fcg_batched", fcg), ("jacobi_pcg_batched", cg(1)),
                     ("plain_cg_batched", cg(0))):
        if name not in solvers:
            continue
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        per, tot = fn()
        e1.record()
        torch.cuda.synchronize()
        its = [p["iters"] for p in per]
        out[name] = {"s": e0.elapsed_time(e1) / 1e3, "iters_min_max": [min(its), max(its)],
                     "iters_sum": int(sum(its)), "rel_res_fp64_max": tot["rel_res_fp64"],
                     "code": int(tot["code"]), "kernel_launches": int(tot["kernel_launches"])}
        by = {}
        for g in classes:
            gi = [it for it, gg in zip(its, grids) if gg == g]
            by["%dx%dx%d" % g] = [min(gi), max(gi)]
        out[name]["iters_by_size"] = by
        if name == "unet_fcg_batched":
            out[name]["fell_back"] = int(sum(p["fell_back"] for p in per))
        if log:
            log(f"{name}: {out[name]}")
    bc.close()
    return out


def ensemble_bench(iters: int = 12, seed: int = 0, levels: int = 2, fcg_m: int = 2) -> dict:
    """Two batched flexible-CG solves of the 96-instance ensemble capped at
    `iters` iterations (initial weights; the cost of an iteration does not
    depend on them): a profiling target."""
    bc, coef, coef64, b, lnk, nets, net_of, _, _ = ensemble_problem(init_params(seed), seed,
                                                                     96, levels)
    bc.set_option("fcg_m", fcg_m)
    tot = None
    for _ in range(2):
        _, per, tot = bc.fcg_solve(coef, coef64, b, nets=nets, net_of=net_of, lnk=lnk, tol=1e-12,
                                   maxit=iters, check=False)
    bc.close()
    return {"instances": 96, "iters": iters, "ms_per_iter": tot["inner_ms"] / iters,
            "launches_per_iter": tot["kernel_launches"] / iters}


def apply_bench(n: int, reps: int = 10, seed: int = 0) -> dict:
    """Time M(r) on an n^3 grid (initial weights; the cost does not depend on them)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    net = tpfa.UNet(n, n, n, device=dev)
    net.set_params(init_params(seed).to(dev))
    r = torch.from_numpy(synth.uniform_field(n ** 3, seed).astype(np.float32)).to(dev)
    lnk = tpfa.log_perm(torch.from_numpy(realization(seed, n, 1.5)[0]).to(dev))
    z = torch.empty_like(r)
    for _ in range(2):
        net.forward(r, lnk, z)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        net.forward(r, lnk, z)
    e1.record()
    tpfa.net_status(dev)
    return {"grid": n, "reps": reps, "apply_ms": e0.elapsed_time(e1) / reps}


def fcg_bench(n: int, levels: int = 2, iters: int = 12, seed: int = 0) -> dict:
    """Two flexible-CG solves capped at `iters` iterations (initial weights; the
    cost of an iteration does not depend on them): a profiling target."""
    dev = torch.device("cuda", torch.cuda.current_device())
    ctx = tpfa.Context(n, n, n, device=dev)
    ctx.set_option("fcg_m", 2)
    pr = Problem(ctx, 777001 + seed, n, 1.5)
    nn = n >> levels
    net = tpfa.UNet(nn, nn, nn, device=dev)
    net.set_params(init_params(seed).to(dev))
    info = None
    for _ in range(2):
        _, info = ctx.fcg_solve(pr.coef, pr.coef64, pr.b, net=net, lnk=pr.lnk, tol=1e-12,
                                maxit=iters, check=False)
    return {"grid": n, "levels": levels, "iters": info["iters"],
            "ms_per_iter": info["inner_ms"] / max(info["iters"], 1)}


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="train and evaluate the U-Net preconditioner")
    ap.add_argument("--n-real", type=int, default=50)
    ap.add_argument("--snaps", type=int, default=40)
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--epochs", type=int, default=12)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--eval-n", type=int, default=256)
    ap.add_argument("--save", default=None, help="write the trained parameters (.npy)")
    ap.add_argument("--levels", type=int, default=2,
                    help="the network runs on the 2^levels coarser grid (0 to 3)")
    ap.add_argument("--apply-bench", type=int, default=0,
                    help="only time preconditioner applications on an N^3 grid")
    ap.add_argument("--fcg-bench", type=int, default=0,
                    help="only run two flexible-CG solves capped at --iters iterations on an "
                         "N^3 problem with the network on the 2^levels coarser grid")
    ap.add_argument("--iters", type=int, default=12)
    ap.add_argument("--ensemble-bench", action="store_true",
                    help="only run two batched flexible-CG solves of the 96-instance ensemble "
                         "capped at --iters iterations")
    ap.add_argument("--ensemble", action="store_true",
                    help="also solve the 96-instance batched ensemble with the trained network "
                         "(fcg_solve_batch) against batched Jacobi PCG and plain CG")
    ap.add_argument("--reps", type=int, default=10)
    a = ap.parse_args(argv)
    log = lambda m: print(m, flush=True)  # noqa: E731
    if a.apply_bench:
        print(json.dumps(apply_bench(a.apply_bench, a.reps)))
        return
    if a.ensemble_bench:
        print(json.dumps(ensemble_bench(a.iters, levels=a.levels)))
        return
    if a.fcg_bench:
        print(json.dumps(fcg_bench(a.fcg_bench, a.levels, a.iters)))
        return
    ds = make_dataset(a.n_real, a.snaps, a.n, log=log)
    P, hist = train(ds, a.epochs, a.batch, a.lr, levels=a.levels, log=log)
    if a.save:
        np.save(a.save, P.cpu().numpy())
    res = evaluate(P, n=a.eval_n, levels=a.levels, log=log)
    res["train"] = hist
    if a.ensemble:
        res["ensemble"] = evaluate_ensemble(P, levels=a.levels, log=log)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
