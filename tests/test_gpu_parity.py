"""GPU path (through the C ABI) against the CPU FP64 oracle.

Inputs come from the seeded generator; every expected value comes from the
oracle.  Tolerances:
  * coefficients: FP64 bit-identical, FP32 within 1 ulp of RN(oracle FP64)
    (both compute the same IEEE operations in the same order);
  * operator: ||Ap_gpu - Ap_ref|| / ||Ap_ref|| <= 1e-6 for random p, and
    element-wise |Ap_gpu - Ap_ref| <= 10 u (|A| |p|), u = 2^-24, which covers
    the rounding of the coefficients to FP32 and seven FP32 fused
    multiply-adds;
  * FP64 residual: element-wise within 1e-13 (|b| + |A| |x|);
  * solve: the oracle's own FP64 residual of the GPU solution <= tol.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2408_03452_gb300 import synth

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def tp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03452_gb300 import build, tpfa
    build.build()
    return tpfa


def _case(shape, seed=0, sigma=1.0, dirichlet="x", d=0.0, wells=False, geom=None, layer=1,
          random_mask=0.0):
    nx, ny, nz = shape
    n = nx * ny * nz
    K = synth.lognormal_field(nx, ny, nz, sigma, seed, layer=layer)
    mask = pD = None
    if dirichlet is not None:
        mask, pD = synth.dirichlet_faces(nx, ny, nz, dirichlet, 1.0, 0.0)
    if random_mask > 0:
        extra = (synth.uniform(seed, 11, np.arange(n)) < random_mask).astype(np.uint8)
        mask = extra if mask is None else np.maximum(mask, extra)
        pD = synth.uniform(seed, 12, np.arange(n)) if pD is None else pD
    q = None
    if wells:
        idx, val = synth.well_pair(nx, ny, nz)
        q = synth.dense_sources(n, idx, val)
    geom = geom or {}
    return dict(shape=shape, n=n, K=K, mask=mask, pD=pD, d=d, q=q, geom=geom)


def _dev(a, dtype=None):
    if a is None:
        return None
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _ctx(tp, c):
    nx, ny, nz = c["shape"]
    return tp.Context(nx, ny, nz, **c["geom"])


def _ogrid(O, c):
    return O.Grid(*c["shape"], **c["geom"])


def _dargs(c):
    d = c["d"]
    if np.isscalar(d):
        return None, float(d)
    return _dev(d), 0.0


def _build(tp, ctx, c):
    d_arr, d0 = _dargs(c)
    return ctx.build_trans(_dev(c["K"]), _dev(c["mask"]), d_arr, d0)


SHAPES = [(32, 32, 32), (7, 5, 3), (33, 17, 9), (1, 1, 1), (1, 1, 40), (61, 1, 1), (31, 2, 3),
          (64, 9, 17), (95, 33, 20)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("variant", ["dirx", "wells_d", "mask_darr"])
def test_build_trans_matches_oracle(tp, oracle_mod, shape, variant):
    O = oracle_mod
    n = shape[0] * shape[1] * shape[2]
    if variant == "dirx":
        c = _case(shape, seed=1, geom=dict(dx=0.5, dy=2.0, dz=1.5, mu=1.3))
    elif variant == "wells_d":
        c = _case(shape, seed=2, sigma=1.5, dirichlet=None, d=1e-3, wells=True, layer=8)
    else:
        c = _case(shape, seed=3, sigma=2.0, dirichlet=None, random_mask=0.2,
                  d=0.01 * synth.uniform(3, 13, np.arange(n)))
    with _ctx(tp, c) as ctx:
        coef, coef64 = _build(tp, ctx, c)
        g32 = coef.cpu().numpy()
        g64 = coef64.cpu().numpy()
    ref = np.stack(O.coefficients(_ogrid(O, c), c["K"], c["mask"], c["d"]), axis=1)
    np.testing.assert_array_equal(g64, ref)
    r32 = ref.astype(np.float32)
    ulp = np.abs(g32.view(np.int32).astype(np.int64) - r32.view(np.int32).astype(np.int64))
    assert ulp.max() <= 1
    assert (ulp == 0).mean() >= 0.999


@pytest.mark.parametrize("shape", SHAPES)
def test_build_rhs_matches_oracle(tp, oracle_mod, shape):
    O = oracle_mod
    n = shape[0] * shape[1] * shape[2]
    c = _case(shape, seed=4, sigma=1.5, random_mask=0.1, geom=dict(dx=1.1, dy=0.9, dz=1.0, mu=2.0))
    q = 0.1 * synth.uniform(4, 14, np.arange(n))
    idx = np.array([0, n - 1, n // 2, n // 2], dtype=np.int64)
    val = np.array([1.0, -1.0, 0.25, 0.5])
    with _ctx(tp, c) as ctx:
        b = ctx.build_rhs(_dev(c["K"]), _dev(c["mask"]), _dev(q), _dev(c["pD"]),
                          _dev(idx), _dev(val)).cpu().numpy()
    qd = q.copy()
    keep = c["mask"][idx] == 0
    np.add.at(qd, idx[keep], val[keep])
    ref = O.rhs(_ogrid(O, c), c["K"], c["mask"], qd, c["pD"])
    np.testing.assert_allclose(b, ref, rtol=1e-14, atol=1e-15)


def _abs_apply(A, x):
    y = np.zeros(A.n)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    np.add.at(y, rows, np.abs(A.vals) * np.abs(x[A.cols]))
    return y


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("tile", [(4, 0, 3), (4, 0, 4), (8, 0, 3), (4, 1, 3), (4, 2, 4), (8, 5, 3)])
def test_apply_matches_oracle(tp, oracle_mod, shape, tile):
    O = oracle_mod
    c = _case(shape, seed=5, sigma=1.5, random_mask=0.05, d=1e-3,
              geom=dict(dx=0.7, dy=1.0, dz=1.3, mu=0.9))
    n = c["n"]
    p = synth.uniform_field(n, 7).astype(np.float32)
    with _ctx(tp, c) as ctx:
        ctx.set_option("tile_vy", tile[0])
        ctx.set_option("stages", tile[2])
        ctx.set_option("tile_zc", tile[1])
        coef, _ = _build(tp, ctx, c)
        pt = _dev(p)
        pAp = torch.zeros(1, dtype=torch.float64, device="cuda")
        Ap = ctx.apply(coef, pt, pAp=pAp)
        Ap2 = ctx.apply(coef, pt, pAp=(pAp2 := torch.zeros_like(pAp)))
        g = Ap.cpu().numpy().astype(np.float64)
        assert torch.equal(Ap, Ap2) and torch.equal(pAp, pAp2)  # bit-reproducible
        gp = pAp.item()
    A = O.assemble(_ogrid(O, c), c["K"], c["mask"], c["d"])
    p64 = p.astype(np.float64)
    ref = A.matvec(p64)
    assert np.linalg.norm(g - ref) <= 1e-6 * np.linalg.norm(ref)
    bound = 10 * U32 * _abs_apply(A, p64) + 1e-30
    assert np.all(np.abs(g - ref) <= bound)
    assert gp == pytest.approx(p64 @ ref, rel=1e-6)


@pytest.mark.parametrize("shape", [(32, 32, 32), (33, 17, 9), (1, 1, 1), (95, 33, 20)])
def test_apply_smooth_field_elementwise(tp, oracle_mod, shape):
    """Smooth p makes A p small against |A||p| (cancellation); the element-wise
    bound still holds."""
    O = oracle_mod
    c = _case(shape, seed=6, sigma=1.0, dirichlet=None, d=0.0)
    p = synth.smooth_field(*shape, seed=3).astype(np.float32)
    with _ctx(tp, c) as ctx:
        coef, _ = _build(tp, ctx, c)
        g = ctx.apply(coef, _dev(p)).cpu().numpy().astype(np.float64)
    A = O.assemble(_ogrid(O, c), c["K"], None, 0.0)
    p64 = p.astype(np.float64)
    ref = A.matvec(p64)
    assert np.all(np.abs(g - ref) <= 10 * U32 * _abs_apply(A, p64) + 1e-30)


@pytest.mark.parametrize("shape", [(32, 32, 32), (7, 5, 3), (95, 33, 20), (1, 1, 1)])
def test_residual64_matches_oracle(tp, oracle_mod, shape):
    O = oracle_mod
    c = _case(shape, seed=8, sigma=2.0, random_mask=0.1, d=1e-2)
    n = c["n"]
    x = synth.uniform_field(n, 9)
    b = synth.uniform_field(n, 10)
    with _ctx(tp, c) as ctx:
        _, coef64 = _build(tp, ctx, c)
        norms = torch.zeros(2, dtype=torch.float64, device="cuda")
        r = ctx.residual64(coef64, _dev(b), _dev(x), norms=norms).cpu().numpy()
        nr = norms.cpu().numpy()
    A = O.assemble(_ogrid(O, c), c["K"], c["mask"], c["d"])
    ref = b - A.matvec(x)
    assert np.all(np.abs(r - ref) <= 1e-13 * (np.abs(b) + _abs_apply(A, x)))
    assert nr[0] == pytest.approx(ref @ ref, rel=1e-12)
    assert nr[1] == pytest.approx(b @ b, rel=1e-12)


def _solve(tp, c, tol, loop=0, maxit=200000, x0=None, tile=None):
    with _ctx(tp, c) as ctx:
        ctx.set_option("loop", loop)
        if tile:
            ctx.set_option("tile_vy", tile[0])
            ctx.set_option("stages", tile[2])
            ctx.set_option("tile_zc", tile[1])
        coef, coef64 = _build(tp, ctx, c)
        b = ctx.build_rhs(_dev(c["K"]), _dev(c["mask"]), _dev(c["q"]), _dev(c["pD"]))
        x = None if x0 is None else _dev(x0)
        x, info = ctx.cg_solve(coef, coef64, b, x=x, tol=tol, maxit=maxit)
        torch.cuda.synchronize()
        return x.cpu().numpy(), info


def _oracle_rel(O, c, x):
    return O.rel_residual(_ogrid(O, c), c["K"], c["mask"], c["d"], c["q"], c["pD"], x)


@pytest.mark.parametrize("loop", [1, 0])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cg_small_config(tp, oracle_mod, loop, seed):
    """32^3, ln K ~ N(0,1), Dirichlet x end layers: FP32 CG to 1e-6, then the
    refined solve to FP64 relative residual 1e-8; the oracle re-evaluates the
    residual of the GPU solution and compares with its own solution."""
    O = oracle_mod
    c = _case((32, 32, 32), seed=seed, sigma=1.0)
    x6, info6 = _solve(tp, c, 1e-6, loop=loop)
    assert info6["code"] == 0, info6
    assert _oracle_rel(O, c, x6) <= 1e-6 * 1.001
    assert info6["rel_res_fp64"] <= 1e-6
    x8, info8 = _solve(tp, c, 1e-8, loop=loop)
    assert info8["code"] == 0, info8
    rel = _oracle_rel(O, c, x8)
    assert rel <= 1e-8 * 1.001
    assert info8["rel_res_fp64"] == pytest.approx(rel, rel=1e-3, abs=1e-12)
    xr, _ = O.solve(_ogrid(O, c), c["K"], c["mask"], c["d"], c["q"], c["pD"], tol=1e-13)
    assert np.linalg.norm(x8 - xr) <= 1e-6 * np.linalg.norm(xr)
    assert info8["iters"] > 0 and info8["outer"] >= 1


def test_cg_loop_modes_and_tiles_agree_bitwise(tp):
    c = _case((33, 17, 9), seed=3, sigma=1.5, dirichlet=None, d=1e-3, wells=True)
    xa, ia = _solve(tp, c, 1e-8, loop=0)
    xb, ib = _solve(tp, c, 1e-8, loop=1)
    xc, ic = _solve(tp, c, 1e-8, loop=0)
    assert np.array_equal(xa, xb) and np.array_equal(xa, xc)
    assert ia["iters"] == ib["iters"] == ic["iters"]
    # the stage count changes neither the arithmetic nor any summation
    # order: bit-identical; the block size regroups the FP64 partial sums
    # a different warp tiling changes only the order of the dot-product
    # partial sums: same solution to the tolerance
    xd, idd = _solve(tp, c, 1e-8, loop=0, tile=(8, 3, 3))
    xe, ie = _solve(tp, c, 1e-8, loop=1, tile=(4, 2, 4))
    assert ie["code"] == 0 and ie["rel_res_fp64"] <= 1e-8
    assert idd["code"] == 0 and idd["rel_res_fp64"] <= 1e-8


@pytest.mark.parametrize("shape", [(7, 5, 3), (61, 1, 1), (1, 1, 40), (95, 33, 20), (64, 9, 17),
                                   (2, 2, 2), (57, 6, 130)])
def test_cg_odd_shapes(tp, oracle_mod, shape):
    O = oracle_mod
    c = _case(shape, seed=4, sigma=1.5, dirichlet=None, d=1e-3, wells=True, layer=2)
    x, info = _solve(tp, c, 1e-8)
    assert info["code"] == 0, info
    assert _oracle_rel(O, c, x) <= 1e-8 * 1.001


def test_cg_edge_cases(tp, oracle_mod):
    O = oracle_mod
    # zero right-hand side: x = 0 without iterating
    c = _case((9, 8, 7), seed=5, dirichlet=None, d=1e-3)
    x, info = _solve(tp, c, 1e-8, x0=np.full(c["n"], 3.0))
    assert info["code"] == 0 and info["iters"] == 0 and np.all(x == 0)
    # single interior cell with accumulation: x = q / d
    c = _case((1, 1, 1), seed=0, dirichlet=None, d=0.25)
    c["q"] = np.array([2.0])
    x, info = _solve(tp, c, 1e-12)
    assert info["code"] == 0 and x[0] == pytest.approx(8.0, rel=1e-12)
    # every cell Dirichlet: the solution is p^D
    n = 6 * 5 * 4
    c = _case((6, 5, 4), seed=1, dirichlet=None)
    c["mask"] = np.ones(n, np.uint8)
    c["pD"] = synth.uniform_field(n, 4)
    x, info = _solve(tp, c, 1e-10)
    assert info["code"] == 0
    np.testing.assert_allclose(x, c["pD"], rtol=0, atol=1e-12)
    # initial guess already converged
    c = _case((12, 11, 10), seed=2, sigma=1.0)
    xr, _ = O.solve(_ogrid(O, c), c["K"], c["mask"], c["d"], c["q"], c["pD"], tol=1e-14)
    x, info = _solve(tp, c, 1e-8, x0=xr)
    assert info["code"] == 0 and info["iters"] == 0
    # iteration limit
    c = _case((32, 32, 32), seed=0)
    x, info = _solve(tp, c, 1e-10, maxit=5)
    assert info["code"] == 1 and info["iters"] == 5
    assert _oracle_rel(O, c, x) == pytest.approx(info["rel_res_fp64"], rel=1e-6)


def test_argument_checks(tp):
    L = tp.lib()
    g = tp._Grid(0, 4, 4, 1.0, 1.0, 1.0, 1.0)
    h = C.c_void_p()
    assert L.tpfa_create(C.byref(g), C.byref(h)) == tp.EINVAL
    g = tp._Grid(70000, 70000, 1, 1.0, 1.0, 1.0, 1.0)
    assert L.tpfa_create(C.byref(g), C.byref(h)) == tp.EINVAL
    g = tp._Grid(4, 4, 4, 1.0, -1.0, 1.0, 1.0)
    assert L.tpfa_create(C.byref(g), C.byref(h)) == tp.EINVAL
    c = _case((16, 8, 8), seed=0)
    with _ctx(tp, c) as ctx:
        coef, coef64 = _build(tp, ctx, c)
        n = c["n"]
        host = np.zeros(4 * n, np.float32)
        p = torch.zeros(n, dtype=torch.float32, device="cuda")
        Ap = torch.zeros(n, dtype=torch.float32, device="cuda")
        s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        # host pointer where a device pointer is required
        assert L.tpfa_apply(ctx._h, C.c_void_p(host.ctypes.data), C.c_void_p(p.data_ptr()),
                            C.c_void_p(Ap.data_ptr()), None, s) == tp.EINVAL
        # misaligned coefficient records
        assert L.tpfa_apply(ctx._h, C.c_void_p(coef.data_ptr() + 4), C.c_void_p(p.data_ptr()),
                            C.c_void_p(Ap.data_ptr()), None, s) == tp.EINVAL
        # aliasing input and output
        assert L.tpfa_apply(ctx._h, C.c_void_p(coef.data_ptr()), C.c_void_p(p.data_ptr()),
                            C.c_void_p(p.data_ptr()), None, s) == tp.EINVAL
        b = torch.zeros(n, dtype=torch.float64, device="cuda")
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        info = tp._Info()
        args = (ctx._h, C.c_void_p(coef.data_ptr()), C.c_void_p(coef64.data_ptr()),
                C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()))
        assert L.cg_solve(*args, 0.0, 10, C.byref(info), s) == tp.EINVAL
        assert L.cg_solve(*args, 1e-8, 0, C.byref(info), s) == tp.EINVAL
        with pytest.raises(tp.TpfaError):
            ctx.set_option("tile_vy", 5)
        with pytest.raises(tp.TpfaError):
            ctx.set_option("stages", 2)
    # a buffer far too small for the grid is refused, not read past its end
    big = _case((256, 256, 64), seed=0, dirichlet=None)
    with _ctx(tp, big) as ctx:
        small = torch.zeros(1024, dtype=torch.float64, device="cuda")
        out = torch.zeros(4 * big["n"], dtype=torch.float32, device="cuda")
        s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        assert L.tpfa_build_trans(ctx._h, C.c_void_p(small.data_ptr()), None, None, 0.0,
                                  C.c_void_p(out.data_ptr()), None, s) == tp.EINVAL
    torch.cuda.synchronize()
