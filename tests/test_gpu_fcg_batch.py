"""Flexible CG over a batch of uneven instances (fcg_solve_batch): the
learned-preconditioned, mixed-precision, batched form.

Every instance's solution is judged by the oracle's FP64 residual.  With the
same sweep tiling, an instance solved inside a batch (next to instances of
other sizes, other networks and none) is bit-identical to the same instance
solved alone: its chunk partials, finish kernels, network sample and
operator blocks are its own."""
import numpy as np
import pytest
import torch

from paper_2408_03452_gb300 import synth
from test_gpu_unet import params_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03452_gb300 import build, tpfa
    build.build()
    return tpfa


def _inst(shape, seed, sigma=1.0, axis="x", p_hi=1.0):
    nx, ny, nz = shape
    K = synth.lognormal_field(nx, ny, nz, sigma, seed)
    mask, pD = synth.dirichlet_faces(nx, ny, nz, axis, p_hi, 0.0)
    return dict(shape=shape, K=K, mask=mask, pD=pD)


def _cat(insts, key):
    return torch.from_numpy(np.concatenate([w[key] for w in insts])).cuda()


def _setup(tp, insts, zc=None):
    bc = tp.BatchContext([w["shape"] for w in insts], zc=zc)
    K, mask, pD = _cat(insts, "K"), _cat(insts, "mask"), _cat(insts, "pD")
    coef, coef64 = bc.build_trans(K, mask, None, 0.0)
    b = bc.build_rhs(K, mask, None, pD)
    lnk = torch.log(K).float()
    return bc, coef, coef64, b, lnk


def _parts(bc, x):
    return [x[bc.offsets[i]:bc.offsets[i + 1]].cpu().numpy() for i in range(bc.ninst)]


def _oracle_rel(O, w, x):
    return O.rel_residual(O.Grid(*w["shape"]), w["K"], w["mask"], 0.0, None, w["pD"], x)


def _nets(tp, specs, seed=9):
    """specs: (coarse grid, samples) per network, all with the same weights."""
    _, flat = params_case(seed)
    P = torch.from_numpy(flat).cuda()
    out = []
    for (cx, cy, cz), ns in specs:
        u = tp.UNet(cx, cy, cz, ns=ns)
        u.set_params(P)
        out.append(u)
    return out


RAGGED = [(13, 11, 7), (9, 5, 3), (24, 20, 12), (1, 1, 1), (16, 16, 16)]
ALIGNED = [(16, 16, 16), (32, 16, 16), (8, 8, 8), (24, 20, 12)]


@pytest.mark.parametrize("shapes", [RAGGED, ALIGNED])
def test_fcg_batch_without_network_matches_oracle(tp, oracle_mod, shapes):
    """No network: FCG is plain CG per instance; ragged cell counts (scalar
    vector passes) and 16-byte aligned ones (float4 passes), a zero
    right-hand side, two retained-direction settings; iteration counts close
    to fcg_solve on each instance alone."""
    O = oracle_mod
    insts = [_inst(s, 30 + i, 0.5 + 0.4 * i, "xyz"[i % 3]) for i, s in enumerate(shapes)]
    insts.append(_inst((9, 8, 7), 7, 1.0, "y", 0.0))  # p^D = 0: b = 0
    bc, coef, coef64, b, _ = _setup(tp, insts)
    for m in (1, 3):
        bc.set_option("fcg_m", m)
        x, per, total = bc.fcg_solve(coef, coef64, b, tol=1e-10, maxit=20000)
        assert total["code"] == tp.OK, (total, per)
        xs = _parts(bc, x)
        for i, w in enumerate(insts):
            assert _oracle_rel(O, w, xs[i]) <= 1e-10 * 1.01, (i, per[i])
            assert not per[i]["fell_back"]
        assert per[-1]["iters"] == 0 and float(np.abs(xs[-1]).max()) == 0.0
    for i, w in enumerate(insts[:-1]):
        with tp.Context(*w["shape"]) as ctx:
            Kd, md = torch.from_numpy(w["K"]).cuda(), torch.from_numpy(w["mask"]).cuda()
            c1, c64 = ctx.build_trans(Kd, md)
            b1 = ctx.build_rhs(Kd, md, pD=torch.from_numpy(w["pD"]).cuda())
            ctx.set_option("fcg_m", 3)
            _, info = ctx.fcg_solve(c1, c64, b1, tol=1e-10, maxit=20000)
        assert abs(per[i]["iters"] - info["iters"]) <= 0.1 * info["iters"] + 5, (per[i], info)
    bc.close()


def _mixed():
    # two 16^3 instances share a network on the 4x coarser grid, a 32x16x16
    # instance has one on the 2x coarser grid, a 24x20x12 instance has none
    insts = [_inst((16, 16, 16), 41, 1.5), _inst((32, 16, 16), 42, 1.5, "y"),
             _inst((24, 20, 12), 43, 1.0, "z"), _inst((16, 16, 16), 44, 1.5, "x", 2.0)]
    return insts, [0, 1, -1, 0]


def test_fcg_batch_with_networks_matches_oracle(tp, oracle_mod):
    O = oracle_mod
    insts, net_of = _mixed()
    bc, coef, coef64, b, lnk = _setup(tp, insts)
    nets = _nets(tp, [((4, 4, 4), 2), ((16, 8, 8), 1)])
    for m in (1, 2):
        bc.set_option("fcg_m", m)
        x, per, total = bc.fcg_solve(coef, coef64, b, nets=nets, net_of=net_of, lnk=lnk,
                                     tol=1e-8, maxit=20000)
        assert total["code"] == tp.OK, (total, per)
        for i, xi in enumerate(_parts(bc, x)):
            assert _oracle_rel(O, insts[i], xi) <= 1e-8 * 1.01, (i, per[i])
    bc.close()


def test_fcg_batch_with_padded_network_grids(tp, oracle_mod):
    """Networks on the 4x coarser grid padded to multiples of 4 (16x16x8 ->
    4x4x2 stored 4x4x4; 24x16x24 -> 6x4x6 stored 8x4x8), next to an unpadded
    one: every instance reaches the FP64 tolerance."""
    O = oracle_mod
    insts = [_inst((16, 16, 8), 51, 1.5), _inst((24, 16, 24), 52, 1.5, "z"),
             _inst((16, 16, 8), 53, 1.0, "y"), _inst((16, 16, 16), 54, 1.5)]
    bc, coef, coef64, b, lnk = _setup(tp, insts)
    nets = _nets(tp, [((4, 4, 4), 2), ((8, 4, 8), 1), ((4, 4, 4), 1)])
    bc.set_option("fcg_m", 2)
    x, per, total = bc.fcg_solve(coef, coef64, b, nets=nets, net_of=[0, 1, 0, 2], lnk=lnk,
                                 tol=1e-8, maxit=20000)
    assert total["code"] == tp.OK, (total, per)
    for i, xi in enumerate(_parts(bc, x)):
        assert _oracle_rel(O, insts[i], xi) <= 1e-8 * 1.01, (i, per[i])
    bc.close()


def test_fcg_batch_networks_with_ragged_offsets(tp, oracle_mod):
    """An 18-cell instance first: every later instance starts at an even
    offset that is not a multiple of 4, so the vector passes take their
    scalar path while networks run on the 4x coarser grids (padded); a
    ragged instance without a network at the end."""
    O = oracle_mod
    insts = [_inst((3, 3, 2), 60, 1.0), _inst((16, 16, 16), 61, 1.5),
             _inst((16, 16, 8), 62, 1.5, "z"), _inst((16, 16, 16), 63, 1.0, "y"),
             _inst((13, 11, 7), 64, 1.0)]
    bc, coef, coef64, b, lnk = _setup(tp, insts)
    assert all(o % 2 == 0 and o % 4 != 0 for o in bc.offsets[1:4])
    nets = _nets(tp, [((4, 4, 4), 2), ((4, 4, 4), 1)])
    bc.set_option("fcg_m", 2)
    x, per, total = bc.fcg_solve(coef, coef64, b, nets=nets, net_of=[-1, 0, 1, 0, -1], lnk=lnk,
                                 tol=1e-8, maxit=20000)
    assert total["code"] == tp.OK, (total, per)
    for i, xi in enumerate(_parts(bc, x)):
        assert _oracle_rel(O, insts[i], xi) <= 1e-8 * 1.01, (i, per[i])
    bc.close()


def test_fcg_batch_instance_independent_of_the_batch(tp):
    """The last instance of the mixed batch, solved alone with its own
    one-sample network and the same tiling: bit-identical solution, same
    iteration count and outer steps."""
    insts, net_of = _mixed()
    bc, coef, coef64, b, lnk = _setup(tp, insts)
    nets = _nets(tp, [((4, 4, 4), 2), ((16, 8, 8), 1)])
    bc.set_option("fcg_m", 2)
    x, per, total = bc.fcg_solve(coef, coef64, b, nets=nets, net_of=net_of, lnk=lnk, tol=1e-8)
    assert total["code"] == tp.OK
    x_all = _parts(bc, x)
    zc = bc.zc
    bc.close()
    for i in (3, 1, 2):
        one = [insts[i]]
        b1c, c1, c64, b1, l1 = _setup(tp, one, zc=[zc[i]])
        b1c.set_option("fcg_m", 2)
        if net_of[i] >= 0:
            spec = [((4, 4, 4), 1)] if insts[i]["shape"] == (16, 16, 16) else [((16, 8, 8), 1)]
            x1, p1, t1 = b1c.fcg_solve(c1, c64, b1, nets=_nets(tp, spec), net_of=[0], lnk=l1,
                                       tol=1e-8)
        else:
            x1, p1, t1 = b1c.fcg_solve(c1, c64, b1, tol=1e-8)
        assert t1["code"] == tp.OK
        assert np.array_equal(_parts(b1c, x1)[0], x_all[i]), i
        assert p1[0]["iters"] == per[i]["iters"] and p1[0]["outer"] == per[i]["outer"], i
        assert p1[0]["fell_back"] == per[i]["fell_back"], i
        b1c.close()


def test_fcg_batch_iteration_cap(tp):
    """Each instance stops at exactly maxit inner iterations (TPFA_NOTCONV),
    with and without networks; x stays finite."""
    insts, net_of = _mixed()
    bc, coef, coef64, b, lnk = _setup(tp, insts)
    nets = _nets(tp, [((4, 4, 4), 2), ((16, 8, 8), 1)])
    for cap in (1, 6, 9):
        x, per, total = bc.fcg_solve(coef, coef64, b, nets=nets, net_of=net_of, lnk=lnk,
                                     tol=1e-14, maxit=cap, check=False)
        assert total["code"] == tp.NOTCONV
        assert all(p["status"] == tp.NOTCONV for p in per)
        assert all(p["iters"] == cap for p in per), [p["iters"] for p in per]
        assert torch.isfinite(x).all()
    bc.close()


def test_fcg_batch_rejects_bad_arguments(tp):
    insts, net_of = _mixed()
    bc, coef, coef64, b, lnk = _setup(tp, insts)
    good = _nets(tp, [((4, 4, 4), 2), ((16, 8, 8), 1)])

    def code(**kw):
        args = dict(nets=good, net_of=net_of, lnk=lnk)
        args.update(kw)
        return bc.fcg_solve(coef, coef64, args.pop("b", b), x=args.pop("x", None), check=False,
                            **args)[2]["code"]

    assert code(nets=_nets(tp, [((4, 4, 4), 1), ((16, 8, 8), 1)])) == tp.EINVAL  # ns != members
    assert code(nets=_nets(tp, [((8, 4, 4), 2), ((16, 8, 8), 1)])) == tp.EINVAL  # wrong grid
    assert code(net_of=[0, 0, -1, 1]) == tp.EINVAL  # one network, two grids
    assert code(net_of=[0, 2, -1, 0]) == tp.EINVAL  # no such network
    buf = torch.zeros(bc.n + 1, dtype=torch.float32, device="cuda")
    assert code(lnk=buf[1:]) == tp.EINVAL  # coarse-grid networks read ln K in pairs
    assert code(x=b) == tp.EINVAL
    bc.close()
