"""The TMA-staged operator application (tpfa_apply, tpfa_apply_bf16) against
the cp.async-staged one and against the oracle.

Both kernels evaluate Eq. 6 / Alg. 2 with the same operands and the same
fused multiply-adds in the same order, so q = A p must agree bit for bit;
p'q is summed in another grouping (other tiles) and agrees to FP32
compensated-sum accuracy.  Cases span several tiles with ragged tails in y
and z (nx must be a multiple of 4 for the TMA kernel), several z-runs, BF16
records, instances of a batch (the batched flexible-CG operator) and the
cases that must take the cp.async kernel (misaligned p, nx % 4 != 0,
the cp.async sweep selected).
"""
import numpy as np
import pytest
import torch

from paper_2408_03452_gb300 import synth
from test_gpu_parity import U32, _abs_apply, _build, _case, _ctx, _dev, _ogrid

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03452_gb300 import build, tpfa
    build.build()
    return tpfa


SHAPES = [(64, 20, 9), (96, 33, 20), (4, 1, 1), (32, 1, 1), (36, 7, 131), (128, 16, 3),
          (8, 50, 2)]


def _close_dots(a, b, p, Ap):
    """Two p'Ap of the same products summed in other groupings: compensated
    FP32 warp sums within 2u of exact each, so within 4u sum |p_i (Ap)_i|."""
    absdot = float((p.double() * Ap.double()).abs().sum())
    return abs(a - b) <= 4 * 2.0 ** -24 * absdot


def _apply_both(tp, ctx, coef, p, b16=False):
    """(Ap, p'Ap) from the default (TMA) kernel and from the cp.async kernel."""
    fn = ctx.apply_bf16 if b16 else ctx.apply
    out = []
    for sweep in (0, 1):
        ctx.set_option("sweep", sweep)
        pAp = torch.zeros(1, dtype=torch.float64, device="cuda")
        Ap = fn(coef, p, pAp=pAp)
        torch.cuda.synchronize()
        out.append((Ap, pAp.item()))
    ctx.set_option("sweep", 0)
    return out


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("zc", [0, 3])
def test_tma_apply_bitwise_equal_to_cp_async(tp, shape, zc):
    c = _case(shape, seed=11, sigma=1.5, random_mask=0.05, d=1e-3,
              geom=dict(dx=0.7, dy=1.0, dz=1.3, mu=0.9))
    n = c["n"]
    p = _dev(synth.uniform_field(n, 12).astype(np.float32))
    with _ctx(tp, c) as ctx:
        ctx.set_option("tile_zc", zc)
        t = ctx.tiling(2)
        assert t["kernel"] == 2 and (zc == 0 or t["zc"] == min(zc, shape[2])), t
        coef, _ = _build(tp, ctx, c)
        (a_tma, d_tma), (a_cp, d_cp) = _apply_both(tp, ctx, coef, p)
    assert torch.equal(a_tma, a_cp)
    assert _close_dots(d_tma, d_cp, p, a_cp)


@pytest.mark.parametrize("shape", SHAPES)
def test_tma_apply_bf16_bitwise_equal_to_cp_async(tp, shape):
    c = _case(shape, seed=13, sigma=2.0, random_mask=0.05, d=1e-2)
    n = c["n"]
    p = _dev(synth.uniform_field(n, 14).astype(np.float32))
    with _ctx(tp, c) as ctx:
        assert ctx.tiling(3)["kernel"] == 2
        r16 = ctx.build_trans_bf16(_dev(c["K"]), _dev(c["mask"]), None, 1e-2)
        (a_tma, d_tma), (a_cp, d_cp) = _apply_both(tp, ctx, r16, p, b16=True)
    assert torch.equal(a_tma, a_cp)
    assert _close_dots(d_tma, d_cp, p, a_cp)


@pytest.mark.parametrize("shape", [(64, 20, 9), (96, 33, 20), (36, 7, 131)])
def test_tma_apply_matches_oracle(tp, oracle_mod, shape):
    O = oracle_mod
    c = _case(shape, seed=15, sigma=1.5, random_mask=0.05, d=1e-3, wells=True)
    n = c["n"]
    p_h = synth.uniform_field(n, 16).astype(np.float32)
    with _ctx(tp, c) as ctx:
        assert ctx.tiling(2)["kernel"] == 2
        coef, _ = _build(tp, ctx, c)
        pAp = torch.zeros(1, dtype=torch.float64, device="cuda")
        g = ctx.apply(coef, _dev(p_h), pAp=pAp).cpu().numpy().astype(np.float64)
        gp = pAp.item()
    A = O.assemble(_ogrid(O, c), c["K"], c["mask"], c["d"])
    p64 = p_h.astype(np.float64)
    ref = A.matvec(p64)
    assert np.all(np.abs(g - ref) <= 10 * U32 * _abs_apply(A, p64) + 1e-30)
    assert np.linalg.norm(g - ref) <= 1e-6 * np.linalg.norm(ref)
    assert gp == pytest.approx(p64 @ ref, rel=1e-6)


def test_cases_that_take_the_cp_async_kernel(tp):
    """A p that starts 4 bytes past a 16-byte boundary, and a grid with
    nx % 4 != 0, are applied by the cp.async kernel: same values."""
    shape = (64, 20, 9)
    c = _case(shape, seed=17, sigma=1.0, d=1e-3)
    n = c["n"]
    p_h = synth.uniform_field(n, 18).astype(np.float32)
    with _ctx(tp, c) as ctx:
        coef, _ = _build(tp, ctx, c)
        ref = ctx.apply(coef, _dev(p_h))
        buf = torch.zeros(n + 4, dtype=torch.float32, device="cuda")
        buf[1:n + 1] = _dev(p_h)
        shifted = buf[1:n + 1]
        assert shifted.data_ptr() % 16 == 4
        got = ctx.apply(coef, shifted)
        torch.cuda.synchronize()
    assert torch.equal(got, ref)
    with tp.Context(66, 20, 9) as ctx:
        assert ctx.tiling(2)["kernel"] == 1 and ctx.tiling(3)["kernel"] == 1
    with tp.Context(64, 20, 9) as ctx:
        ctx.set_option("sweep", 1)
        assert ctx.tiling(2)["kernel"] == 1
        ctx.set_option("tile_vy", 8)
        ctx.set_option("sweep", 0)
        assert ctx.tiling(2)["kernel"] == 1  # another VY than the TMA tile's


def test_tma_apply_repeatable_and_stream_ordered(tp):
    """Two calls give identical Ap and p'Ap; calls on a side stream see the
    inputs written on it."""
    shape = (96, 33, 20)
    c = _case(shape, seed=19, sigma=1.5, d=1e-3)
    n = c["n"]
    with _ctx(tp, c) as ctx:
        coef, _ = _build(tp, ctx, c)
        s = torch.cuda.Stream()
        outs = []
        for _ in range(2):
            with torch.cuda.stream(s):
                p = torch.from_numpy(synth.uniform_field(n, 20).astype(np.float32)).to(
                    "cuda", non_blocking=False)
                pAp = torch.zeros(1, dtype=torch.float64, device="cuda")
                Ap = ctx.apply(coef, p, pAp=pAp)
            s.synchronize()
            outs.append((Ap.clone(), pAp.item()))
    assert torch.equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]


def test_batched_fcg_with_tma_and_cp_async_operators(tp, oracle_mod):
    """The batched flexible CG runs its operator through the TMA kernel when
    every instance has nx % 4 == 0 and 16-byte aligned offsets, else (or with
    the cp.async sweep selected) through the cp.async kernel: both reach the
    oracle's FP64 tolerance with iteration counts within a few percent."""
    from test_gpu_fcg_batch import _inst, _oracle_rel, _parts, _setup
    O = oracle_mod
    insts = [_inst((16, 16, 16), 71, 1.5), _inst((32, 16, 8), 72, 1.0, "y"),
             _inst((24, 20, 12), 73, 2.0, "z")]
    res = {}
    for sweep in (0, 1):
        bc, coef, coef64, b, _ = _setup(tp, insts)
        bc.set_option("sweep", sweep)
        bc.set_option("fcg_m", 2)
        x, per, total = bc.fcg_solve(coef, coef64, b, tol=1e-10, maxit=20000)
        assert total["code"] == tp.OK, (sweep, total, per)
        for i, xi in enumerate(_parts(bc, x)):
            assert _oracle_rel(O, insts[i], xi) <= 1e-10 * 1.01, (sweep, i, per[i])
        res[sweep] = [p["iters"] for p in per]
        bc.close()
    for a, b_ in zip(res[0], res[1]):
        assert abs(a - b_) <= 0.05 * b_ + 3, res


def test_batched_fcg_fused_dots_with_networks(tp, oracle_mod):
    """With networks the TMA-staged operator A u also forms the step's dot
    products (A u not stored); the cp.async sweep option takes the separate
    operator and dots passes.  Both reach the oracle's FP64 tolerance, with
    iteration counts within the spread that rounding gives a nonlinear
    preconditioner."""
    from test_gpu_fcg_batch import _mixed, _nets, _oracle_rel, _parts, _setup
    O = oracle_mod
    insts, net_of = _mixed()
    res = {}
    for sweep in (0, 1):
        bc, coef, coef64, b, lnk = _setup(tp, insts)
        bc.set_option("sweep", sweep)
        bc.set_option("fcg_m", 2)
        nets = _nets(tp, [((4, 4, 4), 2), ((16, 8, 8), 1)])
        x, per, total = bc.fcg_solve(coef, coef64, b, nets=nets, net_of=net_of, lnk=lnk,
                                     tol=1e-8, maxit=20000)
        assert total["code"] == tp.OK, (sweep, total, per)
        for i, xi in enumerate(_parts(bc, x)):
            assert _oracle_rel(O, insts[i], xi) <= 1e-8 * 1.01, (sweep, i, per[i])
        res[sweep] = [p["iters"] for p in per]
        bc.close()
    for a, b_ in zip(res[0], res[1]):
        assert abs(a - b_) <= 0.3 * b_ + 5, res


@pytest.mark.parametrize("m", [3, 4, 5])
def test_batched_fcg_fused_dots_retained_directions(tp, oracle_mod, m):
    """The fused operator carries up to four retained directions (one kernel
    variant per count); with five the separate dots pass takes over.  Every
    instance reaches the oracle's FP64 tolerance either way."""
    from test_gpu_fcg_batch import _mixed, _nets, _oracle_rel, _parts, _setup
    O = oracle_mod
    insts, net_of = _mixed()
    bc, coef, coef64, b, lnk = _setup(tp, insts)
    bc.set_option("fcg_m", m)
    nets = _nets(tp, [((4, 4, 4), 2), ((16, 8, 8), 1)])
    x, per, total = bc.fcg_solve(coef, coef64, b, nets=nets, net_of=net_of, lnk=lnk, tol=1e-8,
                                 maxit=20000)
    assert total["code"] == tp.OK, (total, per)
    for i, xi in enumerate(_parts(bc, x)):
        assert _oracle_rel(O, insts[i], xi) <= 1e-8 * 1.01, (i, per[i])
    bc.close()
