"""Mixed precision: BF16 coefficient records, FP32 inner CG, FP64 refinement.

Expected values come from the CPU FP64 oracle:
  * records: the oracle's eliminated face transmissibilities T' and extra
    diagonal E, rounded to nearest-even BF16 here (exact emulation of the
    rounding), must equal the GPU's bit patterns;
  * operator: the face form sum_f T'(x_K - x_L) + E x_K with those rounded
    values, evaluated in FP64, bounds the GPU product element-wise by
    16 u (|A| |p|), u = 2^-24 (six FP32 additions forming D, seven fused
    multiply-adds);
  * solve: the oracle's FP64 residual of the GPU solution meets the tolerance,
    and the error against the oracle's own solution falls at every
    refinement step.
"""
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


def round_bf16(x):
    """Round float64 values to the nearest BF16 value, ties to even (8
    significant bits), returned as float64."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)  # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def bf16_bits_to_f64(a):
    u = np.asarray(a).astype(np.uint16).astype(np.uint32) << 16
    return u.view(np.float32).astype(np.float64)


def face_apply(shape, Tx, Ty, Tz, E, x):
    nx, ny, nz = shape
    x = x.reshape(nz, ny, nx)
    y = E.reshape(nz, ny, nx) * x
    for axis, Tf in zip((2, 1, 0), (Tx, Ty, Tz)):
        Tf = Tf.reshape(nz, ny, nx)
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[axis], hi[axis] = slice(0, -1), slice(1, None)
        f = Tf[tuple(lo)] * (x[tuple(lo)] - x[tuple(hi)])
        y[tuple(lo)] += f
        y[tuple(hi)] -= f
    return y.reshape(-1)


def face_abs(shape, Tx, Ty, Tz, E, x):
    """|A| |x| for the face form (diagonal sum_f T' + E)."""
    nx, ny, nz = shape
    ax = np.abs(x.reshape(nz, ny, nx))
    D = E.reshape(nz, ny, nx).copy()
    y = np.zeros_like(ax)
    for axis, Tf in zip((2, 1, 0), (Tx, Ty, Tz)):
        Tf = Tf.reshape(nz, ny, nx)
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[axis], hi[axis] = slice(0, -1), slice(1, None)
        t = Tf[tuple(lo)]
        D[tuple(lo)] += t
        D[tuple(hi)] += t
        y[tuple(lo)] += t * ax[tuple(hi)]
        y[tuple(hi)] += t * ax[tuple(lo)]
    return (D * ax + y).reshape(-1)


def _case(shape, seed, kind):
    nx, ny, nz = shape
    n = nx * ny * nz
    if kind == "channels":
        # moderate version of the channelized recipe (sigma 1, contrast 100):
        # the full sigma 2 / 1e4 version needs far more plain-CG iterations
        # than a test can spend
        K = synth.channelized_field(nx, ny, nz, 1.0, seed, n_channels=3, width=3, thickness=3,
                                    amplitude=3.0, wavelength=16.0, contrast=1e2)
        mask, pD = synth.dirichlet_faces(nx, ny, nz, "x", 1.0, 0.0)
        return dict(K=K, mask=mask, pD=pD, d=0.0, q=None)
    if kind == "wells":
        K = synth.lognormal_field(nx, ny, nz, 1.5, seed, layer=2)
        idx, val = synth.well_pair(nx, ny, nz)
        return dict(K=K, mask=None, pD=None, d=1e-3, q=synth.dense_sources(n, idx, val))
    K = synth.lognormal_field(nx, ny, nz, 2.0, seed)
    mask = (synth.uniform(seed, 11, np.arange(n)) < 0.15).astype(np.uint8)
    return dict(K=K, mask=mask, pD=synth.uniform(seed, 12, np.arange(n)),
                d=0.01 * synth.uniform(seed, 13, np.arange(n)), q=None)


def _dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _dargs(c):
    return (None, float(c["d"])) if np.isscalar(c["d"]) else (_dev(c["d"]), 0.0)


SHAPES = [(32, 32, 32), (7, 5, 3), (33, 17, 9), (1, 1, 1), (95, 33, 20), (2, 40, 3)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("kind", ["channels", "wells", "mask_darr"])
def test_bf16_records_match_oracle(tp, oracle_mod, shape, kind):
    O = oracle_mod
    c = _case(shape, 1, kind)
    d_arr, d0 = _dargs(c)
    with tp.Context(*shape) as ctx:
        r16 = ctx.build_trans_bf16(_dev(c["K"]), _dev(c["mask"]), d_arr, d0).cpu().numpy()
    g = O.Grid(*shape)
    Tx, Ty, Tz, _ = O.coefficients(g, c["K"], c["mask"], c["d"])
    E = O.extra_diagonal(g, c["K"], c["mask"], c["d"])
    ref = np.stack([round_bf16(v) for v in (Tx, Ty, Tz, E)], axis=1)
    np.testing.assert_array_equal(bf16_bits_to_f64(r16), ref)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("kind", ["channels", "wells", "mask_darr"])
def test_bf16_apply_matches_oracle(tp, oracle_mod, shape, kind):
    O = oracle_mod
    c = _case(shape, 2, kind)
    n = int(np.prod(shape))
    d_arr, d0 = _dargs(c)
    p = synth.uniform_field(n, 5).astype(np.float32)
    with tp.Context(*shape) as ctx:
        r16 = ctx.build_trans_bf16(_dev(c["K"]), _dev(c["mask"]), d_arr, d0)
        pAp = torch.zeros(1, dtype=torch.float64, device="cuda")
        g_ap = ctx.apply_bf16(r16, _dev(p), pAp=pAp).cpu().numpy().astype(np.float64)
        gp = pAp.item()
    g = O.Grid(*shape)
    Tx, Ty, Tz, _ = O.coefficients(g, c["K"], c["mask"], c["d"])
    E = O.extra_diagonal(g, c["K"], c["mask"], c["d"])
    R = [round_bf16(v) for v in (Tx, Ty, Tz, E)]
    p64 = p.astype(np.float64)
    ref = face_apply(shape, *R, p64)
    bound = 16 * U32 * face_abs(shape, *R, p64) + 1e-30
    assert np.all(np.abs(g_ap - ref) <= bound)
    assert gp == pytest.approx(p64 @ ref, rel=1e-6)
    # against the exact FP64 operator: BF16 rounding of each coefficient (2^-9)
    exact = O.assemble(g, c["K"], c["mask"], c["d"]).matvec(p64)
    assert np.linalg.norm(g_ap - exact) <= 2.0 ** -8 * np.linalg.norm(exact)


def _solve(tp, shape, c, tol, bf16=True, max_outer=None, maxit=200000):
    d_arr, d0 = _dargs(c)
    with tp.Context(*shape) as ctx:
        if max_outer is not None:
            ctx.set_option("max_outer", max_outer)
        K, mask = _dev(c["K"]), _dev(c["mask"])
        coef, coef64 = ctx.build_trans(K, mask, d_arr, d0)
        inner = ctx.build_trans_bf16(K, mask, d_arr, d0) if bf16 else coef
        b = ctx.build_rhs(K, mask, _dev(c["q"]), _dev(c["pD"]))
        x, info = ctx.cg_solve(inner, coef64, b, tol=tol, maxit=maxit)
        torch.cuda.synchronize()
        return x.cpu().numpy(), info


@pytest.mark.parametrize("kind", ["channels", "wells"])
def test_bf16_refined_solve_to_1e10(tp, oracle_mod, kind):
    O = oracle_mod
    shape = (32, 32, 32)
    c = _case(shape, 3, kind)
    g = O.Grid(*shape)
    x, info = _solve(tp, shape, c, 1e-10)
    assert info["code"] == 0, info
    rel = O.rel_residual(g, c["K"], c["mask"], c["d"], c["q"], c["pD"], x)
    # FP64 evaluation noise of a residual this small: |b| + |A||x| times a few ulps
    A = O.assemble(g, c["K"], c["mask"], c["d"])
    b = O.rhs(g, c["K"], c["mask"], c["q"], c["pD"])
    absAx = np.zeros(A.n)
    np.add.at(absAx, np.repeat(np.arange(A.n), np.diff(A.rowptr)), np.abs(A.vals) * np.abs(x[A.cols]))
    noise = 16 * 2.0 ** -53 * np.linalg.norm(np.abs(b) + absAx) / np.linalg.norm(b)
    assert rel <= 1e-10 + noise
    assert abs(info["rel_res_fp64"] - rel) <= 2 * noise + 1e-3 * rel
    assert info["outer"] >= 2  # BF16 alone cannot reach 1e-10: refinement did the rest
    xr, _ = O.solve(g, c["K"], c["mask"], c["d"], c["q"], c["pD"], tol=1e-14)
    assert np.linalg.norm(x - xr) <= 1e-7 * np.linalg.norm(xr)


def test_bf16_error_falls_at_every_refinement_step(tp, oracle_mod):
    """Error of the GPU iterate against the oracle's FP64 solution after
    1, 2, ... refinement steps (the solve stopped by the step limit)."""
    O = oracle_mod
    shape = (24, 20, 16)
    c = _case(shape, 4, "channels")
    g = O.Grid(*shape)
    xr, _ = O.solve(g, c["K"], c["mask"], c["d"], c["q"], c["pD"], tol=1e-14)
    errs = []
    for k in range(1, 6):
        x, info = _solve(tp, shape, c, 1e-12, max_outer=k)
        errs.append(np.linalg.norm(x - xr) / np.linalg.norm(xr))
        if info["code"] == 0:
            break
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[0] > 1e-6 > errs[-1], errs


def test_bf16_and_fp32_inner_reach_the_same_solution(tp, oracle_mod):
    shape = (33, 17, 9)
    c = _case(shape, 5, "wells")
    x16, i16 = _solve(tp, shape, c, 1e-10, bf16=True)
    x32, i32 = _solve(tp, shape, c, 1e-10, bf16=False)
    assert i16["code"] == 0 and i32["code"] == 0
    assert np.linalg.norm(x16 - x32) <= 1e-5 * np.linalg.norm(x32)


def _solve_opts(tp, shape, c, tol, opts, maxit=400000):
    d_arr, d0 = _dargs(c)
    with tp.Context(*shape) as ctx:
        for k, v in opts.items():
            ctx.set_option(k, v)
        K, mask = _dev(c["K"]), _dev(c["mask"])
        coef, coef64 = ctx.build_trans(K, mask, d_arr, d0)
        b = ctx.build_rhs(K, mask, _dev(c["q"]), _dev(c["pD"]))
        x, info = ctx.cg_solve(coef, coef64, b, tol=tol, maxit=maxit)
        torch.cuda.synchronize()
        return x.cpu().numpy(), info


@pytest.mark.parametrize("shape,kind", [((32, 32, 32), "channels"), ((33, 17, 9), "wells"),
                                        ((7, 5, 3), "mask_darr"), ((95, 33, 20), "channels"),
                                        ((1, 1, 1), "wells")])
@pytest.mark.parametrize("loop", [0, 1])
def test_jacobi_pcg_matches_oracle(tp, oracle_mod, shape, kind, loop):
    """Jacobi-preconditioned inner CG (M = diag(D)): the oracle's FP64 residual
    of the GPU solution meets the tolerance."""
    O = oracle_mod
    c = _case(shape, 6, kind)
    if kind == "wells" and shape == (1, 1, 1):
        c["q"] = np.array([0.5])
    x, info = _solve_opts(tp, shape, c, 1e-8, {"precond": 1, "loop": loop})
    assert info["code"] == 0, info
    g = O.Grid(*shape)
    assert O.rel_residual(g, c["K"], c["mask"], c["d"], c["q"], c["pD"], x) <= 1e-8 * 1.001


def test_jacobi_needs_fewer_iterations_on_high_contrast(tp, oracle_mod):
    shape = (48, 48, 48)
    nx, ny, nz = shape
    K = synth.channelized_field(nx, ny, nz, 2.0, 7, n_channels=4, width=4, thickness=4,
                                amplitude=6.0, wavelength=24.0, contrast=1e4)
    mask, pD = synth.dirichlet_faces(nx, ny, nz, "x", 1.0, 0.0)
    c = dict(K=K, mask=mask, pD=pD, d=0.0, q=None)
    xj, ij = _solve_opts(tp, shape, c, 1e-8, {"precond": 1})
    xp, ip = _solve_opts(tp, shape, c, 1e-8, {"precond": 0})
    assert ij["code"] == 0, ij
    assert ij["iters"] < ip["iters"], (ij["iters"], ip["iters"])
    g = O = oracle_mod
    assert O.rel_residual(O.Grid(*shape), K, mask, 0.0, None, pD, xj) <= 1e-8 * 1.001


def _solve_bf16_opts(tp, shape, c, tol, opts, x0=None, maxit=400000):
    d_arr, d0 = _dargs(c)
    with tp.Context(*shape) as ctx:
        for k, v in opts.items():
            ctx.set_option(k, v)
        K, mask = _dev(c["K"]), _dev(c["mask"])
        _, coef64 = ctx.build_trans(K, mask, d_arr, d0)
        c16 = ctx.build_trans_bf16(K, mask, d_arr, d0)
        b = ctx.build_rhs(K, mask, _dev(c["q"]), _dev(c["pD"]))
        x, info = ctx.cg_solve(c16, coef64, b, x=None if x0 is None else _dev(x0), tol=tol,
                               maxit=maxit)
        torch.cuda.synchronize()
        return x.cpu().numpy(), info


@pytest.mark.parametrize("shape,kind", [((32, 32, 32), "channels"), ((33, 17, 9), "wells"),
                                        ((7, 5, 3), "mask_darr"), ((95, 33, 20), "channels"),
                                        ((1, 1, 1), "wells"), ((61, 1, 1), "mask_darr")])
@pytest.mark.parametrize("loop", [0, 1])
def test_bf16_jacobi_pcg_matches_oracle(tp, oracle_mod, shape, kind, loop):
    """BF16 records with the Jacobi-preconditioned inner CG (M = the diagonal
    the BF16 sweep forms) and FP64 refinement: the oracle's FP64 residual of
    the GPU solution meets 1e-10."""
    O = oracle_mod
    c = _case(shape, 6, kind)
    if kind == "wells" and shape == (1, 1, 1):
        c["q"] = np.array([0.5])
    x, info = _solve_bf16_opts(tp, shape, c, 1e-10, {"precond": 1, "loop": loop})
    assert info["code"] == 0, info
    g = O.Grid(*shape)
    rel = O.rel_residual(g, c["K"], c["mask"], c["d"], c["q"], c["pD"], x)
    assert rel <= 1e-10 * 1.01, rel


def test_bf16_jacobi_matches_fp32_jacobi_solution(tp):
    shape = (40, 24, 16)
    c = _case(shape, 8, "channels")
    x16, i16 = _solve_bf16_opts(tp, shape, c, 1e-10, {"precond": 1})
    x32, i32 = _solve_opts(tp, shape, c, 1e-10, {"precond": 1})
    assert i16["code"] == 0 and i32["code"] == 0
    assert np.linalg.norm(x16 - x32) <= 1e-6 * np.linalg.norm(x32)


def test_bf16_jacobi_channelized_error_falls_at_every_refinement_step(tp, oracle_mod):
    """The mixed-precision configuration at 48^3: channelized field (sigma 2
    background, eight sinusoidal channels 1e4 times more permeable), Dirichlet
    x end layers, BF16 records, Jacobi-preconditioned FP32 inner CG, FP64
    refinement to 1e-10.  One refinement step per call (each call continues
    from the previous iterate, which is what the refinement loop does); after
    every step the error against the oracle's FP64 solution (Jacobi PCG to
    1e-13) must fall, and the last iterate must meet 1e-10 by the oracle's
    FP64 residual."""
    O = oracle_mod
    n = 48
    w = synth.channelized(seed=1, n=n)
    c = dict(K=w["K"], mask=w["mask"], pD=w["pD"], d=0.0, q=None)
    shape = (n, n, n)
    g = O.Grid(*shape)
    xr, _ = O.solve(g, c["K"], c["mask"], 0.0, None, c["pD"], tol=1e-13, jacobi=True)
    x = np.zeros(n ** 3)
    errs, rels = [], []
    for step in range(20):
        x, info = _solve_bf16_opts(tp, shape, c, 1e-10, {"precond": 1, "max_outer": 1}, x0=x)
        errs.append(np.linalg.norm(x - xr) / np.linalg.norm(xr))
        rels.append(info["rel_res_fp64"])
        assert info["code"] in (0, 1), info
        if info["code"] == 0:
            break
    assert info["code"] == 0, (errs, rels)
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert len(errs) >= 2  # BF16 records alone do not reach 1e-10: refinement did the rest
    assert O.rel_residual(g, c["K"], c["mask"], 0.0, None, c["pD"], x) <= 1e-10 * 1.01
    assert errs[-1] <= 1e-7, errs
