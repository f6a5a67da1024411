"""Batched ensembles: many grids solved in one sweep launch per iteration.

Each instance's solution is checked by the oracle's FP64 residual; with the
same warp tiling, an instance solved inside a batch is bit-identical to the
same problem solved alone (same per-cell arithmetic, same partial sums in the
same order, same refinement decisions)."""
import numpy as np
import pytest
import torch

from paper_2408_03452_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03452_gb300 import build, tpfa
    build.build()
    return tpfa


def _instances():
    shapes = [(24, 20, 12), (7, 5, 3), (33, 17, 9), (1, 1, 1), (40, 3, 30), (16, 16, 16)]
    out = []
    for i, (nx, ny, nz) in enumerate(shapes):
        u = synth.uniform(50 + i, 2, np.arange(3))
        axis = "xyz"[i % 3]
        K = synth.lognormal_field(nx, ny, nz, 0.5 + 2.0 * u[0], 100 + i)
        mask, pD = synth.dirichlet_faces(nx, ny, nz, axis, 0.5 + 1.5 * u[1], 0.0)
        out.append(dict(nx=nx, ny=ny, nz=nz, K=K, mask=mask, pD=pD))
    # an instance whose right-hand side is zero (p^D = 0 everywhere)
    nx, ny, nz = 9, 8, 7
    K = synth.lognormal_field(nx, ny, nz, 1.0, 7)
    mask, pD = synth.dirichlet_faces(nx, ny, nz, "y", 0.0, 0.0)
    out.append(dict(nx=nx, ny=ny, nz=nz, K=K, mask=mask, pD=pD))
    return out


def _cat(insts, key):
    return torch.from_numpy(np.concatenate([w[key] for w in insts])).cuda()


def _batch_solve(tp, insts, tol, zc=None, precond=0, sweep=0):
    grids = [(w["nx"], w["ny"], w["nz"]) for w in insts]
    with tp.BatchContext(grids, zc=zc) as bc:
        bc.set_option("precond", precond)
        bc.set_option("sweep", sweep)
        K, mask, pD = _cat(insts, "K"), _cat(insts, "mask"), _cat(insts, "pD")
        coef, coef64 = bc.build_trans(K, mask, None, 0.0)
        b = bc.build_rhs(K, mask, None, pD)
        x, per, total = bc.cg_solve(coef, coef64, b, tol=tol)
        torch.cuda.synchronize()
        xs = [x[bc.offsets[i]:bc.offsets[i + 1]].cpu().numpy() for i in range(len(insts))]
        return xs, per, total, bc.zc


def _single_solve(tp, w, tol, zc, precond=0, sweep=0):
    with tp.Context(w["nx"], w["ny"], w["nz"]) as ctx:
        ctx.set_option("tile_vy", 4)
        ctx.set_option("stages", 4)
        ctx.set_option("tile_zc", zc)
        ctx.set_option("precond", precond)
        ctx.set_option("sweep", sweep)
        K, mask, pD = (torch.from_numpy(w[k]).cuda() for k in ("K", "mask", "pD"))
        coef, coef64 = ctx.build_trans(K, mask, None, 0.0)
        b = ctx.build_rhs(K, mask, None, pD)
        x, info = ctx.cg_solve(coef, coef64, b, tol=tol)
        torch.cuda.synchronize()
        return x.cpu().numpy(), info


@pytest.mark.parametrize("sweep", [0, 1], ids=["tma", "cpasync"])
@pytest.mark.parametrize("precond", [0, 1])
def test_batch_matches_oracle_and_single_solves(tp, oracle_mod, precond, sweep):
    """Both batched sweeps (TMA-staged, the default, and cp.async-staged)."""
    O = oracle_mod
    insts = _instances()
    xs, per, total, zc = _batch_solve(tp, insts, 1e-8, precond=precond, sweep=sweep)
    assert total["code"] == 0, (total, per)
    for i, w in enumerate(insts):
        g = O.Grid(w["nx"], w["ny"], w["nz"])
        assert per[i]["status"] == 0, per[i]
        assert O.rel_residual(g, w["K"], w["mask"], 0.0, None, w["pD"], xs[i]) <= 1e-8 * 1.001
        xi, info = _single_solve(tp, w, 1e-8, zc[i], precond, sweep)
        assert np.array_equal(xs[i], xi), i
        assert per[i]["iters"] == info["iters"], i
    # the zero right-hand side instance: x = 0 without iterating
    assert per[-1]["iters"] == 0 and np.all(xs[-1] == 0)
    # instances converge after different numbers of iterations
    assert len({p["iters"] for p in per[:-1]}) > 1


@pytest.mark.parametrize("sweep", [0, 1], ids=["tma", "cpasync"])
def test_batch_explicit_tiling_and_loose_tolerance(tp, oracle_mod, sweep):
    O = oracle_mod
    insts = _instances()[:4]
    xs, per, total, zc = _batch_solve(tp, insts, 1e-6, zc=[1, 2, 3, 1], sweep=sweep)
    assert zc == [1, 2, 3, 1]
    assert total["code"] == 0
    for i, w in enumerate(insts):
        g = O.Grid(w["nx"], w["ny"], w["nz"])
        assert O.rel_residual(g, w["K"], w["mask"], 0.0, None, w["pD"], xs[i]) <= 1e-6 * 1.001


def test_batch_rejects_bad_grids(tp):
    with pytest.raises(tp.TpfaError):
        tp.BatchContext([(4, 4, 4), (0, 3, 3)])
    with pytest.raises(tp.TpfaError):
        tp.BatchContext([(4, 4, 4)], zc=[-1])


@pytest.mark.parametrize("tile", [1, 2, 3])
def test_batch_tma_tiles(tp, oracle_mod, tile):
    """The other tiles of the TMA-staged batched sweep (plain CG)."""
    O = oracle_mod
    insts = _instances()
    grids = [(w["nx"], w["ny"], w["nz"]) for w in insts]
    with tp.BatchContext(grids) as bc:
        bc.set_option("tma_tile", tile)
        K, mask, pD = _cat(insts, "K"), _cat(insts, "mask"), _cat(insts, "pD")
        coef, coef64 = bc.build_trans(K, mask, None, 0.0)
        b = bc.build_rhs(K, mask, None, pD)
        x, per, total = bc.cg_solve(coef, coef64, b, tol=1e-8)
        torch.cuda.synchronize()
        assert total["code"] == 0, (total, per)
        for i, w in enumerate(insts):
            xi = x[bc.offsets[i]:bc.offsets[i + 1]].cpu().numpy()
            g = O.Grid(w["nx"], w["ny"], w["nz"])
            assert O.rel_residual(g, w["K"], w["mask"], 0.0, None, w["pD"], xi) <= 1e-8 * 1.001
