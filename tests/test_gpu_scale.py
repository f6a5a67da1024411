"""Parity at the benchmark's scale and tiling.

The small-grid parity tests never reach the tilings the paper-scale solve
uses: 128-plane z-runs, thousands of blocks in one reduction, inputs far
larger than L2.  Here the paper-scale recipe (layered lognormal K with
sigma 1.5, d = 1e-3, corner well pair) is built at 512 x 256 x 256 and at the
benchmark's own 1024 x 1024 x 256, with the default planner, and the GPU is
compared with the CPU FP64 oracle on sampled cells (evaluated row by row from
K, so no full matrix is needed) and, at 512 x 256 x 256, on whole vectors:
  * operator: |Ap_gpu - Ap_ref| <= 10 u (|A| |p|) per sampled row (u = 2^-24:
    FP32 rounding of the coefficients plus seven fused multiply-adds), and
    ||Ap_gpu - Ap_ref|| / ||Ap_ref|| <= 1e-6 over the sample;
  * FP64 residual of a capped solve: |r_gpu - (b - A x)| <= 1e-13 (|b| + |A| |x|)
    per sampled row;
  * fused CG iterations (512 x 256 x 256, both sweeps): x_k after k = 3 and 8
    iterations against the oracle's FP64 CG iterate, relative 2-norm <= 1e-4.
"""
import numpy as np
import pytest
import torch

from paper_2408_03452_gb300 import synth

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
N_SAMPLE = 100_000


@pytest.fixture(scope="module")
def tp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03452_gb300 import build, tpfa
    build.build()
    return tpfa


def sample_rows(nx, ny, nz, zc, seed=17):
    """N_SAMPLE seeded cells plus the cells on tile and run boundaries: the
    grid's faces, edges and corners, x next to multiples of 30 and 32 (warp
    and block columns), y next to multiples of 4 and 16 (warp and block rows)
    and z next to multiples of zc (z-runs)."""
    n = nx * ny * nz
    u = synth.uniform(seed, 3, np.arange(N_SAMPLE, dtype=np.uint64))
    rows = [np.minimum((u * n).astype(np.int64), n - 1)]
    xs = sorted({0, 1, nx - 2, nx - 1} | {v for m in range(30, nx, 30) for v in (m - 1, m)}
                | {v for m in range(32, nx, 32) for v in (m - 1, m)})
    ys = sorted({0, 1, ny - 2, ny - 1} | {v for m in range(16, ny, 16) for v in (m - 1, m)}
                | {v for m in range(4, ny, 4) for v in (m - 1, m)})
    zs = sorted({0, 1, nz - 2, nz - 1} | {v for m in range(zc, nz, zc) for v in (m - 1, m)})
    r = np.random.default_rng(seed)
    for _ in range(4):  # a few lines through the boundary sets in every direction
        x0, y0, z0 = r.integers(nx), r.integers(ny), r.integers(nz)
        rows.append(np.array([x + nx * (y0 + ny * z0) for x in xs], dtype=np.int64))
        rows.append(np.array([x0 + nx * (y + ny * z0) for y in ys], dtype=np.int64))
        rows.append(np.array([x0 + nx * (y0 + ny * z) for z in zs], dtype=np.int64))
    corners = [x + nx * (y + ny * z) for x in (0, nx - 1) for y in (0, ny - 1) for z in (0, nz - 1)]
    rows.append(np.array(corners, dtype=np.int64))
    return np.unique(np.concatenate(rows))


def _workload(nx, ny, nz):
    return synth.paper_scale(seed=3, nx=nx, ny=ny, nz=nz)


def _check_apply_and_residual(tp, O, w, nx, ny, nz):
    n = nx * ny * nz
    dev = torch.device("cuda", 0)
    g = O.Grid(nx, ny, nz)
    with tp.Context(nx, ny, nz, device=dev) as ctx:
        t_apply = ctx.tiling(2)
        t_cg = ctx.tiling(0)
        assert t_apply["zc"] == 128 and t_cg["zc"] == 128, (t_apply, t_cg)
        K = torch.from_numpy(w["K"]).to(dev)
        coef, coef64 = ctx.build_trans(K, None, None, w["d"])
        p_h = synth.uniform_field(n, 23).astype(np.float32)
        p = torch.from_numpy(p_h).to(dev)
        pAp = torch.zeros(1, dtype=torch.float64, device=dev)
        Ap = ctx.apply(coef, p, pAp=pAp).cpu().numpy().astype(np.float64)
        rows = sample_rows(nx, ny, nz, t_apply["zc"])
        p64 = p_h.astype(np.float64)
        ref = O.apply_rows(g, w["K"], None, w["d"], rows, p64)
        scale = O.abs_apply_rows(g, w["K"], None, w["d"], rows, p64)
        err = np.abs(Ap[rows] - ref)
        assert np.all(err <= 10 * U32 * scale + 1e-30), int(np.argmax(err / (scale + 1e-300)))
        assert np.linalg.norm(Ap[rows] - ref) <= 1e-6 * np.linalg.norm(ref)
        # p'Ap: FP64 sum of the GPU's own products
        assert pAp.item() == pytest.approx(float(p64 @ Ap), rel=1e-6)
        del p, Ap
        # FP64 residual of a capped solve (a few CG iterations, one refinement)
        si = torch.from_numpy(w["src_idx"]).to(dev)
        sv = torch.from_numpy(w["src_val"]).to(dev)
        b = ctx.build_rhs(K, None, None, None, si, sv)
        x, info = ctx.cg_solve(coef, coef64, b, tol=1e-30, maxit=5, check=False)
        assert info["iters"] == 5
        r = torch.empty(n, dtype=torch.float64, device=dev)
        norms = torch.zeros(2, dtype=torch.float64, device=dev)
        ctx.residual64(coef64, b, x, r=r, norms=norms)
        torch.cuda.synchronize()
        x_h, r_h, b_h = x.cpu().numpy(), r.cpu().numpy(), b.cpu().numpy()
        nr = norms.cpu().numpy()
    q = synth.dense_sources(n, w["src_idx"], w["src_val"])
    ref_r = q[rows] - O.apply_rows(g, w["K"], None, w["d"], rows, x_h)
    scale_r = np.abs(q[rows]) + O.abs_apply_rows(g, w["K"], None, w["d"], rows, x_h)
    np.testing.assert_array_equal(b_h[rows], q[rows])  # no Dirichlet cells: b = q
    assert np.all(np.abs(r_h[rows] - ref_r) <= 1e-13 * scale_r)
    assert nr[0] == pytest.approx(float(r_h @ r_h), rel=1e-12)
    assert nr[1] == pytest.approx(float(b_h @ b_h), rel=1e-12)
    return x_h


def test_apply_and_residual_at_512x256x256(tp, oracle_mod):
    nx, ny, nz = 512, 256, 256
    _check_apply_and_residual(tp, oracle_mod, _workload(nx, ny, nz), nx, ny, nz)


def test_cg_iterates_at_512x256x256(tp, oracle_mod):
    """The fused CG iteration (a1-a5) at scale: the TMA-staged sweep (default
    here) and the cp.async sweep, each capped at k iterations, against the
    oracle's FP64 CG on the assembled 33.5M-cell matrix."""
    O = oracle_mod
    nx, ny, nz = 512, 256, 256
    n = nx * ny * nz
    w = _workload(nx, ny, nz)
    g = O.Grid(nx, ny, nz)
    A = O.assemble(g, w["K"], None, w["d"])
    q = synth.dense_sources(n, w["src_idx"], w["src_val"])
    H = 8
    _, _, _, _, hist = O.cg(A, q, tol=0.0, maxit=H, history=H)
    del A
    dev = torch.device("cuda", 0)
    K = torch.from_numpy(w["K"]).to(dev)
    si = torch.from_numpy(w["src_idx"]).to(dev)
    sv = torch.from_numpy(w["src_val"]).to(dev)
    for sweep in (2, 1):
        with tp.Context(nx, ny, nz, device=dev) as ctx:
            ctx.set_option("sweep", sweep)
            ctx.set_option("max_outer", 1)
            assert ctx.tiling(0)["kernel"] == sweep and ctx.tiling(0)["zc"] == 128
            coef, coef64 = ctx.build_trans(K, None, None, w["d"])
            b = ctx.build_rhs(K, None, None, None, si, sv)
            for k in (3, 8):
                x, info = ctx.cg_solve(coef, coef64, b, tol=1e-30, maxit=k, check=False)
                assert info["iters"] == k
                xh = x.cpu().numpy()
                ref = hist[k - 1]
                assert np.linalg.norm(xh - ref) <= 1e-4 * np.linalg.norm(ref), (sweep, k)


def test_apply_and_residual_at_bench_size(tp, oracle_mod):
    """The benchmark grid itself, 1024 x 1024 x 256 (268M cells), sampled."""
    if torch.cuda.get_device_properties(0).total_memory < 40e9:
        pytest.skip("needs a large GPU")
    nx, ny, nz = 1024, 1024, 256
    _check_apply_and_residual(tp, oracle_mod, _workload(nx, ny, nz), nx, ny, nz)
