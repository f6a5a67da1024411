"""The TMA-staged CG sweep against the CPU FP64 oracle and the cp.async sweep.

The two sweeps apply the same per-cell arithmetic in the same order (Alg. 1
with the Eq. 6 operator); they differ in how planes reach shared memory and
in the grouping of the dot products' partial sums.  Expected values come from
the oracle:
  * iterates: x_k after k CG iterations (one inner solve capped at k) against
    the oracle's FP64 CG iterate x_k, relative 2-norm <= 1e-4 for k <= 8
    (FP32 vectors against FP64; on some fields FP32 CG itself drifts away
    from the FP64 iterates after about ten iterations: a numpy emulation of
    FP32 CG on the 100 x 30 x 41 wells case below differs from FP64 by 1e-7 at
    k = 8, 1.5e-5 at k = 10 and 8e-3 at k = 12, and the two sweeps, whose dot
    products are summed in different orders, then differ by 5e-3 as well);
    the two sweeps' iterates agree to 1e-5 for k <= 8 (same per-cell
    arithmetic);
  * solves: the oracle's FP64 residual of the GPU solution <= tol, for every
    tile choice, both loop modes, ragged x / y tiles and z-runs, any nx.
"""
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


def _case(shape, seed, kind):
    nx, ny, nz = shape
    n = nx * ny * nz
    if kind == "dirx":
        K = synth.lognormal_field(nx, ny, nz, 1.0, seed)
        mask, pD = synth.dirichlet_faces(nx, ny, nz, "x", 1.0, 0.0)
        return dict(K=K, mask=mask, pD=pD, d=0.0, q=None)
    K = synth.lognormal_field(nx, ny, nz, 1.5, seed, layer=4)
    idx, val = synth.well_pair(nx, ny, nz)
    return dict(K=K, mask=None, pD=None, d=1e-3, q=synth.dense_sources(n, idx, val))


def _dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()


def tiling(tp, ctx, which=0):
    return ctx.tiling(which)


def _solve(tp, shape, c, tol, maxit, opts):
    with tp.Context(*shape) as ctx:
        for k, v in opts.items():
            ctx.set_option(k, v)
        K, mask = _dev(c["K"]), _dev(c["mask"])
        coef, coef64 = ctx.build_trans(K, mask, None, c["d"])
        b = ctx.build_rhs(K, mask, _dev(c["q"]), _dev(c["pD"]))
        x, info = ctx.cg_solve(coef, coef64, b, tol=tol, maxit=maxit, check=False)
        torch.cuda.synchronize()
        t = tiling(tp, ctx)
        return x.cpu().numpy(), info, t


def test_tiling_selection(tp):
    for shape in ((64, 20, 9), (66, 20, 9), (65, 20, 9)):
        nx = shape[0]
        with tp.Context(*shape) as ctx:
            assert tiling(tp, ctx)["kernel"] == 2                                # FP32 records
            assert tiling(tp, ctx, 1)["kernel"] == (2 if nx % 2 == 0 else 1)     # BF16 records
            assert tiling(tp, ctx, 2)["kernel"] == (2 if nx % 4 == 0 else 1)     # tpfa_apply
            assert tiling(tp, ctx, 3)["kernel"] == (2 if nx % 4 == 0 else 1)     # tpfa_apply_bf16
            ctx.set_option("precond", 1)
            assert tiling(tp, ctx)["kernel"] == 2
            assert tiling(tp, ctx, 1)["kernel"] == (2 if nx % 4 == 0 else 1)     # BF16 Jacobi
            ctx.set_option("precond", 0)
            ctx.set_option("sweep", 1)
            assert tiling(tp, ctx)["kernel"] == 1
            assert tiling(tp, ctx, 2)["kernel"] == 1
            ctx.set_option("sweep", 2)
            t = tiling(tp, ctx)
            assert t["kernel"] == 2 and t["warps"] == 4 and t["vy"] == 4 and t["stages"] == 4
            nbx = (nx + 31) // 32
            for tile, (w, vy, st) in enumerate([(4, 4, 4), (4, 4, 3), (8, 4, 3), (4, 2, 6)]):
                ctx.set_option("tma_tile", tile)
                t = tiling(tp, ctx)
                assert (t["warps"], t["vy"], t["stages"]) == (w, vy, st)
                assert t["blocks"] == nbx * ((20 + w * vy - 1) // (w * vy)) * ((9 + t["zc"] - 1) // t["zc"])
                if nx % 2 == 0:  # BF16 records always use tile 0
                    t16 = tiling(tp, ctx, 1)
                    assert (t16["warps"], t16["vy"], t16["stages"]) == (4, 4, 4)
            with pytest.raises(tp.TpfaError):
                ctx.set_option("tma_tile", 4)
            if nx % 2 != 0:
                with pytest.raises(tp.TpfaError):
                    tiling(tp, ctx, 1)  # TMA requested, BF16 records, odd nx


def test_tma_sweep_refused_where_it_cannot_run(tp):
    """BF16 records with an odd nx have row strides that are not multiples of
    16 bytes: a requested TMA sweep is refused, the automatic choice falls
    back to the cp.async sweep."""
    shape = (65, 8, 8)
    c = _case(shape, 1, "wells")
    with tp.Context(*shape) as ctx:
        K = _dev(c["K"])
        coef, coef64 = ctx.build_trans(K, None, None, 1e-3)
        c16 = ctx.build_trans_bf16(K, None, None, 1e-3)
        b = ctx.build_rhs(K, None, _dev(c["q"]), None)
        ctx.set_option("sweep", 2)
        with pytest.raises(tp.TpfaError):
            ctx.cg_solve(c16, coef64, b, tol=1e-8)
        ctx.set_option("sweep", 0)
        _, info = ctx.cg_solve(c16, coef64, b, tol=1e-8)
        assert info["code"] == 0


ITER_SHAPES = [((32, 32, 32), "dirx"), ((36, 17, 9), "wells"), ((4, 4, 4), "dirx"),
               ((100, 30, 41), "wells"), ((64, 1, 7), "wells"), ((33, 17, 9), "dirx"),
               ((95, 33, 20), "wells")]


@pytest.mark.parametrize("shape,kind", ITER_SHAPES)
def test_cg_iterates_match_oracle(tp, oracle_mod, shape, kind):
    """x_k of the TMA sweep and of the cp.async sweep against the oracle's
    FP64 CG iterate and against each other, k = 1, 2, 5, 8."""
    O = oracle_mod
    c = _case(shape, 2, kind)
    g = O.Grid(*shape)
    A = O.assemble(g, c["K"], c["mask"], c["d"])
    b = O.rhs(g, c["K"], c["mask"], c["q"], c["pD"])
    H = 8
    _, _, _, _, hist = O.cg(A, b, tol=0.0, maxit=H, history=H)
    for k in (1, 2, 5, 8):
        xs = {}
        for sweep in (1, 2):
            x, info, t = _solve(tp, shape, c, 1e-30, k, {"sweep": sweep, "max_outer": 1})
            assert t["kernel"] == sweep
            assert info["iters"] == k, info
            ref = hist[k - 1]
            err = np.linalg.norm(x - ref) / np.linalg.norm(ref)
            assert err <= 1e-4, (k, sweep, err)
            xs[sweep] = x
        assert np.linalg.norm(xs[1] - xs[2]) <= 1e-5 * np.linalg.norm(xs[1]), k


SOLVE_SHAPES = [(32, 32, 32), (36, 17, 9), (4, 4, 4), (100, 30, 41), (64, 1, 7), (8, 50, 130),
                (4, 1, 1), (128, 16, 3), (7, 5, 3), (1, 1, 1), (61, 1, 1), (1, 1, 40), (95, 33, 20),
                (2, 40, 3)]


@pytest.mark.parametrize("shape", SOLVE_SHAPES)
@pytest.mark.parametrize("tile", [0, 1, 2, 3])
def test_tma_solve_matches_oracle(tp, oracle_mod, shape, tile):
    O = oracle_mod
    kind = "dirx" if shape[0] > 2 and shape[0] % 8 == 0 else "wells"
    c = _case(shape, 3, kind)
    x, info, t = _solve(tp, shape, c, 1e-8, 400000, {"sweep": 2, "tma_tile": tile})
    assert t["kernel"] == 2
    assert info["code"] == 0, info
    g = O.Grid(*shape)
    assert O.rel_residual(g, c["K"], c["mask"], c["d"], c["q"], c["pD"], x) <= 1e-8 * 1.001


@pytest.mark.parametrize("zc", [1, 7, 64, 200])
@pytest.mark.parametrize("loop", [0, 1])
def test_tma_z_runs_and_loop_modes(tp, oracle_mod, zc, loop):
    """Forced z-run lengths (1 plane, a ragged 7, 64, one run longer than
    the grid) in both loop modes; the default plan is covered above."""
    O = oracle_mod
    shape = (40, 20, 70)
    c = _case(shape, 4, "wells")
    x, info, t = _solve(tp, shape, c, 1e-8, 400000, {"sweep": 2, "tile_zc": zc, "loop": loop})
    assert t["kernel"] == 2 and t["zc"] == min(zc, 70)
    assert info["code"] == 0, info
    g = O.Grid(*shape)
    assert O.rel_residual(g, c["K"], c["mask"], c["d"], c["q"], c["pD"], x) <= 1e-8 * 1.001


def test_tma_loop_modes_agree_bitwise(tp):
    shape = (48, 24, 20)
    c = _case(shape, 5, "wells")
    xa, ia, _ = _solve(tp, shape, c, 1e-8, 400000, {"sweep": 2, "loop": 0})
    xb, ib, _ = _solve(tp, shape, c, 1e-8, 400000, {"sweep": 2, "loop": 1})
    xc, ic, _ = _solve(tp, shape, c, 1e-8, 400000, {"sweep": 2, "loop": 0})
    assert np.array_equal(xa, xb) and np.array_equal(xa, xc)
    assert ia["iters"] == ib["iters"] == ic["iters"]


def _solve_var(tp, shape, c, tol, maxit, opts, b16):
    with tp.Context(*shape) as ctx:
        for k, v in opts.items():
            ctx.set_option(k, v)
        K, mask = _dev(c["K"]), _dev(c["mask"])
        coef, coef64 = ctx.build_trans(K, mask, None, c["d"])
        inner = ctx.build_trans_bf16(K, mask, None, c["d"]) if b16 else coef
        b = ctx.build_rhs(K, mask, _dev(c["q"]), _dev(c["pD"]))
        x, info = ctx.cg_solve(inner, coef64, b, tol=tol, maxit=maxit, check=False)
        torch.cuda.synchronize()
        return x.cpu().numpy(), info, ctx.tiling(1 if b16 else 0)


VARIANTS = [(False, 1), (True, 0), (True, 1)]  # (BF16 records, Jacobi)


@pytest.mark.parametrize("b16,jac", VARIANTS, ids=["f32-jacobi", "bf16", "bf16-jacobi"])
@pytest.mark.parametrize("shape,kind", [((32, 32, 32), "dirx"), ((36, 17, 9), "wells"),
                                        ((100, 30, 41), "wells"), ((64, 1, 7), "wells"),
                                        ((8, 50, 130), "dirx"), ((4, 1, 1), "wells")])
def test_tma_variants_match_cpasync_and_oracle(tp, oracle_mod, b16, jac, shape, kind):
    """The Jacobi and BF16-record TMA variants: the first iterates agree with
    the cp.async sweep's (same per-cell arithmetic; dot products summed in
    another order), and the refined solve meets the tolerance by the
    oracle's FP64 residual."""
    O = oracle_mod
    c = _case(shape, 6, kind)
    n = shape[0] * shape[1] * shape[2]
    for k in [k for k in (1, 3, 8) if k < n]:  # CG ends exactly within n iterations
        xs = {}
        for sweep in (1, 2):
            x, info, t = _solve_var(tp, shape, c, 1e-30, k,
                                    {"sweep": sweep, "precond": jac, "max_outer": 1}, b16)
            assert t["kernel"] == sweep and info["iters"] == k, (t, info)
            xs[sweep] = x
        assert np.linalg.norm(xs[1] - xs[2]) <= 1e-5 * np.linalg.norm(xs[1]), k
    tol = 1e-10 if b16 else 1e-8
    x, info, t = _solve_var(tp, shape, c, tol, 400000, {"sweep": 2, "precond": jac}, b16)
    assert t["kernel"] == 2 and info["code"] == 0, info
    g = O.Grid(*shape)
    assert O.rel_residual(g, c["K"], c["mask"], c["d"], c["q"], c["pD"], x) <= tol * 1.01
