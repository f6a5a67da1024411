"""The U-Net preconditioner, its gradients, Adam, the A-norm loss and flexible
CG through the C ABI, against the FP64 oracle (oracle/unet_oracle.py).

Tolerances.  The network stores every activation and activation gradient in
BF16 (unit roundoff 2^-8) and uses BF16 weights.  Two comparisons:
  * against the exact FP64 oracle on the same BF16-rounded weights: about
    ten roundings of relative size <= 2^-8 lie on the longest forward path,
    so the output agrees in relative 2-norm to 3e-2;
  * against the oracle with its storage hook rounding each kept tensor to
    BF16 at the same points as the kernels: what remains is FP32
    accumulation order and the BF16 rounding (or ReLU) decisions it flips.
    The output agrees to 1e-2.  A parameter gradient passes through up to
    22 stored BF16 tensors (11 forward, 11 backward); the first-order bound
    of 22 roundings of relative size 2^-8 is 8.6e-2, the tolerance used.
    (It is not slack: perturbing the oracle's weights by 1e-6 relative moves
    its own BF16-emulated gradients by up to 3-7% per layer on these sizes.)
A wrong tap, layer, skip or mask produces O(1) relative errors.  Adam runs in FP32 against FP64:
relative 1e-5.  The loss gradient uses A e and A Mr in FP32 (FP32
coefficients, relative 1e-6 each) and a difference of two terms: 1e-4.  Solves are judged by the oracle's FP64 residual.
"""
import numpy as np
import pytest
import torch

from oracle import unet_oracle as U
from paper_2408_03452_gb300 import synth

pytestmark = pytest.mark.gpu

GRAD_TOL = 22 * 2.0 ** -8  # first-order bound: 22 BF16 roundings on a gradient's path


@pytest.fixture(scope="module")
def tp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03452_gb300 import build, tpfa
    build.build()
    return tpfa


def bf16_round(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(torch.bfloat16).to(torch.float64).numpy()


def params_case(seed):
    """Oracle parameter dict with BF16-representable weights, non-zero biases,
    and the flat FP32 vector in the library's layout."""
    p = U.init_params(seed)
    rng = np.random.default_rng(seed)
    flat = []
    for i, (name, cin, cout) in enumerate(U.LAYERS):
        p[name] = bf16_round(p[name])
        p["b%d" % i] = (0.05 * rng.standard_normal(cout)).astype(np.float32).astype(np.float64)
        flat += [p[name].ravel(), p["b%d" % i]]
    return p, np.concatenate(flat).astype(np.float32)


def flat_grads(g):
    return np.concatenate([np.concatenate([g[name].ravel(), g["b%d" % i]])
                           for i, (name, _, _) in enumerate(U.LAYERS)])


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def field_case(shape, ns, seed):
    nx, ny, nz = shape
    n = nx * ny * nz
    r = np.stack([synth.uniform_field(n, seed + s) for s in range(ns)])
    lnk = np.stack([np.log(synth.lognormal_field(nx, ny, nz, 1.0, seed + 10 + s))
                    for s in range(ns)])
    return r, lnk


def to_vol(a, shape, ns):
    nx, ny, nz = shape
    return a.reshape(ns, nz, ny, nx)


@pytest.mark.parametrize("shape,ns", [((8, 8, 8), 2), ((16, 12, 8), 1), ((12, 8, 20), 3)])
def test_unet_forward_backward_match_oracle(tp, shape, ns):
    p, flat = params_case(3)
    r, lnk = field_case(shape, ns, 100)
    dev = torch.device("cuda")
    net = tp.UNet(*shape, ns=ns, train=True)
    net.set_params(torch.from_numpy(flat).to(dev))
    R = torch.from_numpy(r.ravel().astype(np.float32)).to(dev)
    LK = torch.from_numpy(lnk.ravel().astype(np.float32)).to(dev)
    z = net.forward(R, LK)
    gz = np.stack([synth.uniform_field(r.shape[1], 500 + s) for s in range(ns)])
    grad = net.backward(torch.from_numpy(gz.ravel().astype(np.float32)).to(dev))
    tp.net_status()
    # oracle on the same FP32 inputs
    r32 = r.astype(np.float32).astype(np.float64)
    lnk32 = lnk.astype(np.float32).astype(np.float64)
    inp, rms = U.net_input(to_vol(r32, shape, ns), to_vol(lnk32, shape, ns))
    zo, cache = U.unet_forward(p, inp)
    mr = zo * rms[:, None, None, None]
    assert rel(z.cpu().double().numpy(), mr.ravel()) < 3e-2
    zb, cache = U.unet_forward(p, inp, store=bf16_round)
    assert rel(z.cpu().double().numpy(), (zb * rms[:, None, None, None]).ravel()) < 1e-2
    go = U.unet_backward(p, cache, to_vol(gz, shape, ns) * rms[:, None, None, None],
                         store=bf16_round)
    gg = grad.cpu().double().numpy()
    ref = flat_grads(go)
    off = 0
    for i, (name, cin, cout) in enumerate(U.LAYERS):
        nw = 27 * cin * cout
        assert rel(gg[off:off + nw], ref[off:off + nw]) < GRAD_TOL, name
        assert rel(gg[off + nw:off + nw + cout], ref[off + nw:off + nw + cout]) < GRAD_TOL, "b%d" % i
        off += nw + cout
    assert off == tp.unet_param_count() == gg.size


def test_unet_homogeneous_and_samples_independent(tp):
    """M(c r) = c M(r) up to BF16 rounding of r/rms (exact for c a power of
    two), and each sample of a batch equals the same sample run alone."""
    shape, ns = (8, 8, 12), 3
    _, flat = params_case(5)
    r, lnk = field_case(shape, ns, 7)
    dev = torch.device("cuda")
    P = torch.from_numpy(flat).to(dev)
    net = tp.UNet(*shape, ns=ns, train=True)
    net.set_params(P)
    R = torch.from_numpy(r.ravel().astype(np.float32)).to(dev)
    LK = torch.from_numpy(lnk.ravel().astype(np.float32)).to(dev)
    z1 = net.forward(R, LK).clone()
    z2 = net.forward(4.0 * R, LK)
    assert torch.equal(z2, 4.0 * z1)
    one = tp.UNet(*shape, ns=1)
    one.set_params(P)
    n = r.shape[1]
    for s in range(ns):
        zs = one.forward(R[s * n:(s + 1) * n].contiguous(), LK[s * n:(s + 1) * n].contiguous())
        assert torch.equal(zs, z1[s * n:(s + 1) * n])
    # a forward pass over the first k samples gives those samples' outputs,
    # and leaves the network without activations for a backward pass
    for k in (1, 2):
        zk = net.forward(R[:k * n].contiguous(), LK[:k * n].contiguous(), samples=k)
        assert torch.equal(zk, z1[:k * n])
    with pytest.raises(tp.TpfaError):
        net.backward(torch.ones_like(R))
    net.forward(R, LK)
    net.backward(torch.ones_like(R))  # a full pass restores it


def test_adam_matches_oracle(tp):
    n = 10007
    rng = np.random.default_rng(1)
    w, g = rng.standard_normal(n), rng.standard_normal(n)
    m, v = 0.1 * rng.standard_normal(n), rng.uniform(0, 1, n)
    dev = torch.device("cuda")
    W, G, M, V = (torch.from_numpy(a.astype(np.float32)).to(dev) for a in (w, g, m, v))
    tp.adam_step(W, G, M, V, 7, 1e-3)
    w32, g32, m32, v32 = (a.astype(np.float32).astype(np.float64) for a in (w, g, m, v))
    wr, mr, vr = U.adam_step(w32, g32, m32, v32, 7, 1e-3)
    np.testing.assert_allclose(M.cpu().double().numpy(), mr, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(V.cpu().double().numpy(), vr, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(W.cpu().double().numpy(), wr, rtol=1e-5, atol=1e-6)


def _problem(shape, seed=2, sigma=1.0):
    nx, ny, nz = shape
    K = synth.lognormal_field(nx, ny, nz, sigma, seed)
    mask, pD = synth.dirichlet_faces(nx, ny, nz, "x", 1.0, 0.0)
    return K, mask, pD


def _gpu_problem(tp, shape, K, mask, pD):
    dev = torch.device("cuda")
    ctx = tp.Context(*shape)
    Kd = torch.from_numpy(K).to(dev)
    md = torch.from_numpy(mask).to(dev)
    coef, coef64 = ctx.build_trans(Kd, md)
    b = ctx.build_rhs(Kd, md, pD=torch.from_numpy(pD).to(dev))
    return ctx, coef, coef64, b


def test_anorm_loss_grad_matches_oracle(tp, oracle_mod):
    O = oracle_mod
    shape = (12, 10, 8)
    K, mask, pD = _problem(shape)
    ctx, coef, coef64, _ = _gpu_problem(tp, shape, K, mask, pD)
    A = O.assemble(O.Grid(*shape), K, mask)
    n = A.n
    e = synth.uniform_field(n, 3).astype(np.float32)
    mr = (e + 0.3 * synth.uniform_field(n, 4)).astype(np.float32)
    dev = torch.device("cuda")
    E, MR = torch.from_numpy(e).to(dev), torch.from_numpy(mr).to(dev)
    eae = torch.zeros(1, dtype=torch.float64, device=dev)
    R = ctx.apply(coef, E, pAp=eae)
    q, g = (torch.empty(n, dtype=torch.float32, device=dev) for _ in range(2))
    stats = torch.zeros(2, dtype=torch.float64, device=dev)
    ctx.anorm_loss_grad(coef, MR, R, eae, q, g, stats)
    a, b = stats.cpu().numpy()
    L = 1.0 - a * a / (b * eae.item())
    # the oracle sees the FP32 r the kernel used (A e evaluated by the library)
    L_ref, g_ref = U.anorm_loss_scaled(mr.astype(np.float64), R.cpu().double().numpy(),
                                       e.astype(np.float64), A.matvec)
    assert abs(L - L_ref) <= 1e-4 * abs(L_ref)
    assert rel(g.cpu().double().numpy(), g_ref) < 1e-4


def test_jacobi_split_and_blend_loss_match_oracle(tp, oracle_mod):
    """s = r - A D^-1 r, w'Aw, and the gradient of the blended loss (the loss
    kernel fed with s) against the oracle's anorm_loss_blend."""
    O = oracle_mod
    shape = (12, 10, 8)
    K, mask, pD = _problem(shape)
    ctx, coef, coef64, _ = _gpu_problem(tp, shape, K, mask, pD)
    A = O.assemble(O.Grid(*shape), K, mask)
    n = A.n
    dev = torch.device("cuda")
    e = synth.uniform_field(n, 8).astype(np.float32)
    u = synth.uniform_field(n, 9).astype(np.float32)
    E, Ud = torch.from_numpy(e).to(dev), torch.from_numpy(u).to(dev)
    eae = torch.zeros(1, dtype=torch.float64, device=dev)
    R = ctx.apply(coef, E, pAp=eae)
    wAw = torch.zeros(1, dtype=torch.float64, device=dev)
    S = ctx.jacobi_split(coef, R, e=E, wAw=wAw)
    q, g = (torch.empty(n, dtype=torch.float32, device=dev) for _ in range(2))
    stats = torch.zeros(2, dtype=torch.float64, device=dev)
    ctx.anorm_loss_grad(coef, Ud, S, eae, q, g, stats)
    a, b = stats.cpu().numpy()
    L = (wAw.item() - a * a / b) / eae.item()
    r = R.cpu().double().numpy()
    dinv = 1.0 / coef[:, 3].cpu().double().numpy()
    s_ref = r - A.matvec(dinv * r)
    assert rel(S.cpu().double().numpy(), s_ref) < 1e-5
    L_ref, g_ref = U.anorm_loss_blend(u.astype(np.float64), r, e.astype(np.float64), dinv, A.matvec)
    assert abs(L - L_ref) <= 1e-4 * abs(L_ref)
    assert rel(g.cpu().double().numpy(), g_ref) < 1e-4


def _oracle_rel_residual(O, shape, K, mask, pD, x):
    return O.rel_residual(O.Grid(*shape), K, mask, 0.0, None, pD, x)


def test_fcg_identity_is_plain_cg(tp, oracle_mod):
    """Without a network FCG is plain CG: it reaches the FP64 tolerance with
    close to the iteration count of the library's own refined CG solve."""
    O = oracle_mod
    shape = (24, 20, 16)
    K, mask, pD = _problem(shape)
    ctx, coef, coef64, b = _gpu_problem(tp, shape, K, mask, pD)
    x, info = ctx.fcg_solve(coef, coef64, b, tol=1e-10, maxit=20000)
    assert info["code"] == tp.OK and not info["fell_back"]
    assert _oracle_rel_residual(O, shape, K, mask, pD, x.cpu().numpy()) <= 1e-10 * 1.01
    _, info_cg = ctx.cg_solve(coef, coef64, b, tol=1e-10, maxit=20000)
    assert abs(info["iters"] - info_cg["iters"]) <= 0.1 * info_cg["iters"] + 5, (info, info_cg)


@pytest.mark.parametrize("shape", [(32, 32, 32), (16, 24, 40)])
def test_fcg_with_unet_converges(tp, oracle_mod, shape):
    """With an untrained network (random weights) FCG still reaches the FP64
    tolerance (falling back to plain CG if the network is useless)."""
    O = oracle_mod
    K, mask, pD = _problem(shape, seed=4, sigma=1.5)
    ctx, coef, coef64, b = _gpu_problem(tp, shape, K, mask, pD)
    _, flat = params_case(9)
    dev = torch.device("cuda")
    net = tp.UNet(*shape)
    net.set_params(torch.from_numpy(flat).to(dev))
    lnk = torch.from_numpy(np.log(K).astype(np.float32)).to(dev)
    x, info = ctx.fcg_solve(coef, coef64, b, net=net, lnk=lnk, tol=1e-8, maxit=20000)
    assert info["code"] == tp.OK
    assert _oracle_rel_residual(O, shape, K, mask, pD, x.cpu().numpy()) <= 1e-8 * 1.01


def test_restrict_prolong_match_oracle(tp):
    rng = np.random.default_rng(21)
    nx, ny, nz, ns = 8, 6, 4, 2
    f = rng.standard_normal((ns, nz, ny, nx)).astype(np.float32)
    dev = torch.device("cuda")
    F = torch.from_numpy(f.ravel()).to(dev)
    rc = tp.restrict2(F, (nx, ny, nz, ns)).cpu().double().numpy()
    ref = U.restrict2(f.astype(np.float64)).ravel()
    np.testing.assert_allclose(rc, ref, rtol=1e-6, atol=1e-7)
    rs = tp.restrict2(F, (nx, ny, nz, ns), scale=1.0).cpu().double().numpy()
    np.testing.assert_allclose(rs, 8.0 * ref, rtol=1e-6, atol=1e-6)
    c = rng.standard_normal(ref.size).astype(np.float32)
    pf = tp.prolong2(torch.from_numpy(c).to(dev), (nx, ny, nz, ns)).cpu().numpy()
    assert np.array_equal(pf, U.prolong2(c.reshape(ns, nz // 2, ny // 2, nx // 2)).ravel()
                          .astype(np.float32))


@pytest.mark.parametrize("levels,shape", [(1, (8, 6, 4, 2)), (1, (6, 4, 2, 3)),
                                          (2, (16, 8, 12, 2)), (3, (16, 16, 8, 1))])
def test_restrict_prolong_levels_equal_repeated_single_level(tp, levels, shape):
    """The one-pass restriction to the 2^levels coarser grid (what the solvers
    use) is bit-identical to `levels` tpfa_restrict2 passes, the one-pass
    prolongation to `levels` tpfa_prolong2 passes; and both agree with the
    oracle's restrict2 / prolong2 applied `levels` times."""
    nx, ny, nz, ns = shape
    rng = np.random.default_rng(31 + levels)
    f = rng.standard_normal(nx * ny * nz * ns).astype(np.float32)
    F = torch.from_numpy(f).cuda()
    c = F
    for l in range(levels):
        c = tp.restrict2(c, (nx >> l, ny >> l, nz >> l, ns))
    fused = tp.restrict_levels(F, shape, levels)
    assert torch.equal(fused, c)
    ref = f.astype(np.float64).reshape(ns, nz, ny, nx)
    for _ in range(levels):
        ref = U.restrict2(ref)
    np.testing.assert_allclose(fused.cpu().double().numpy(), ref.ravel(), rtol=1e-5, atol=1e-6)
    cc = rng.standard_normal(c.numel()).astype(np.float32)
    CC = torch.from_numpy(cc).cuda()
    p = CC
    for l in reversed(range(levels)):
        p = tp.prolong2(p, (nx >> l, ny >> l, nz >> l, ns))
    fused_p = tp.prolong_levels(CC, shape, levels)
    assert torch.equal(fused_p, p)
    up = cc.astype(np.float64).reshape(ns, nz >> levels, ny >> levels, nx >> levels)
    for _ in range(levels):
        up = U.prolong2(up)
    assert np.array_equal(fused_p.cpu().double().numpy(), up.ravel())
    # a fine vector on an 8- but not 16-byte boundary takes the two-cell stores: same values
    buf2 = torch.zeros(nx * ny * nz * ns + 2, dtype=torch.float32, device="cuda")
    assert buf2[2:].data_ptr() % 16 == 8
    assert torch.equal(tp.prolong_levels(CC, shape, levels, fine=buf2[2:]), fused_p)
    # the prolongations write pairs of cells: a fine vector off an 8-byte boundary is refused
    buf = torch.zeros(nx * ny * nz * ns + 1, dtype=torch.float32, device="cuda")
    with pytest.raises(tp.TpfaError):
        tp.prolong2(c if levels == 1 else tp.restrict2(F, shape), shape, fine=buf[1:])


@pytest.mark.parametrize("shape", [(13, 11, 7), (9, 5, 3)])
def test_fcg_ragged_sizes(tp, oracle_mod, shape):
    """Cell counts that are not a multiple of 4 (vector kernels' scalar tail,
    padded direction slots), with and without Jacobi fallback settings."""
    O = oracle_mod
    K, mask, pD = _problem(shape, seed=7)
    ctx, coef, coef64, b = _gpu_problem(tp, shape, K, mask, pD)
    for m in (1, 3):
        ctx.set_option("fcg_m", m)
        x, info = ctx.fcg_solve(coef, coef64, b, tol=1e-10, maxit=5000)
        assert info["code"] == tp.OK
        assert _oracle_rel_residual(O, shape, K, mask, pD, x.cpu().numpy()) <= 1e-10 * 1.01


@pytest.mark.parametrize("shape,f", [((32, 32, 32), 2), ((16, 24, 40), 2), ((32, 16, 48), 4)])
def test_fcg_with_coarse_unet_converges(tp, oracle_mod, shape, f):
    """A network created for the f-times coarser grid is applied as
    P^l net(R^l r, R^l ln K) inside the blend; the solve reaches the FP64
    tolerance."""
    O = oracle_mod
    K, mask, pD = _problem(shape, seed=5, sigma=1.5)
    ctx, coef, coef64, b = _gpu_problem(tp, shape, K, mask, pD)
    _, flat = params_case(9)
    dev = torch.device("cuda")
    net = tp.UNet(*(d // f for d in shape))
    net.set_params(torch.from_numpy(flat).to(dev))
    lnk = torch.from_numpy(np.log(K).astype(np.float32)).to(dev)
    x, info = ctx.fcg_solve(coef, coef64, b, net=net, lnk=lnk, tol=1e-8, maxit=20000)
    assert info["code"] == tp.OK
    assert _oracle_rel_residual(O, shape, K, mask, pD, x.cpu().numpy()) <= 1e-8 * 1.01


def test_fcg_iteration_cap_zero_rhs_and_status(tp):
    """The inner iteration stops exactly at maxit (TPFA_NOTCONV, checked
    between the host's looks as well); a zero right-hand side converges with
    no iteration; the returned x is always finite."""
    shape = (24, 16, 16)
    K, mask, pD = _problem(shape, seed=8)
    ctx, coef, coef64, b = _gpu_problem(tp, shape, K, mask, pD)
    for cap in (1, 6, 9):
        x, info = ctx.fcg_solve(coef, coef64, b, tol=1e-12, maxit=cap, check=False)
        assert info["code"] == tp.NOTCONV and info["iters"] == cap
        assert torch.isfinite(x).all()
    z = torch.zeros_like(b)
    x, info = ctx.fcg_solve(coef, coef64, z, tol=1e-8)
    assert info["code"] == tp.OK and info["iters"] == 0 and float(x.abs().max()) == 0.0
    # with a network on the 2x coarser grid the cap holds too
    _, flat = params_case(2)
    net = tp.UNet(12, 8, 8)
    net.set_params(torch.from_numpy(flat).cuda())
    lnk = torch.from_numpy(np.log(K).astype(np.float32)).cuda()
    _, info = ctx.fcg_solve(coef, coef64, b, net=net, lnk=lnk, tol=1e-12, maxit=7, check=False)
    assert info["code"] == tp.NOTCONV and info["iters"] == 7


def test_fcg_rejects_mismatched_network(tp):
    shape = (16, 16, 16)
    K, mask, pD = _problem(shape)
    ctx, coef, coef64, b = _gpu_problem(tp, shape, K, mask, pD)
    net = tp.UNet(16, 16, 8)
    _, flat = params_case(1)
    net.set_params(torch.from_numpy(flat).cuda())
    lnk = torch.zeros(16 ** 3, dtype=torch.float32, device="cuda")
    _, info = ctx.fcg_solve(coef, coef64, b, net=net, lnk=lnk, check=False)
    assert info["code"] == tp.EINVAL


def test_log_perm_is_the_rounded_natural_log(tp):
    """The network's permeability input ln K: the FP64 natural logarithm
    rounded to FP32, within one FP32 ulp of numpy's (CUDA's log is accurate to
    a couple of FP64 ulps, so the rounding to FP32 agrees except where the
    FP64 value sits within those ulps of a rounding boundary)."""
    from paper_2408_03452_gb300 import synth
    K = synth.lognormal_field(37, 19, 11, 2.5, 4)
    K[:3] = [1.0, 1e-30, 7e30]
    got = tp.log_perm(torch.from_numpy(K).cuda()).cpu().numpy()
    ref = np.log(K).astype(np.float32)
    ulp = np.abs(got.view(np.int32).astype(np.int64) - ref.view(np.int32).astype(np.int64))
    assert ulp.max() <= 1 and (ulp == 0).mean() >= 0.999
    assert got[0] == 0.0
