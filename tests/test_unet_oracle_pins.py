"""Pins for the learned-preconditioner oracle (oracle/unet_oracle.py).

Each check comes from outside the function it tests: seven nested loops, a
scipy library correlation, hand-written expectations for a shift kernel,
adjoint identities (which determine a linear map's adjoint uniquely), central
finite differences for every gradient, closed forms of Adam, and for flexible
CG: equality with the C oracle's plain CG, with scipy's preconditioned CG for
a fixed SPD preconditioner, and one-step termination with the exact inverse.
A dropped tap, a flipped offset, a transposed weight, a missing skip term or
a wrong ReLU mask fails at least one of them.
"""
import numpy as np
import pytest
import scipy.ndimage
import scipy.sparse
import scipy.sparse.linalg

from oracle import unet_oracle as U
from paper_2408_03452_gb300 import synth


def _rand(rng, *shape):
    return rng.standard_normal(shape)


def test_tap_order():
    assert U.TAPS[0] == (-1, -1, -1) and U.TAPS[13] == (0, 0, 0) and U.TAPS[26] == (1, 1, 1)
    for t, (dz, dy, dx) in enumerate(U.TAPS):
        assert U.tap_index(dz, dy, dx) == t


def test_conv3d_bruteforce():
    rng = np.random.default_rng(1)
    x = _rand(rng, 2, 3, 4, 5, 3)
    w = _rand(rng, 27, 2, 3)
    b = _rand(rng, 2)
    np.testing.assert_allclose(U.conv3d(x, w, b), U.conv3d_bruteforce(x, w, b), rtol=1e-12,
                               atol=1e-12)


def test_conv3d_scipy_correlate():
    """One input and one output channel: scipy.ndimage.correlate with a
    3x3x3 kernel and zero boundary computes the same cross-correlation."""
    rng = np.random.default_rng(2)
    x = _rand(rng, 1, 5, 6, 7, 1)
    w = _rand(rng, 27, 1, 1)
    k = w[:, 0, 0].reshape(3, 3, 3)  # k[dz+1, dy+1, dx+1]
    ref = scipy.ndimage.correlate(x[0, ..., 0], k, mode="constant", cval=0.0)
    np.testing.assert_allclose(U.conv3d(x, w)[0, ..., 0], ref, rtol=1e-12, atol=1e-12)


def test_conv3d_shift_kernel():
    """A weight of one at tap (0, 0, +1) reads the right-hand neighbour:
    y[x] = x[x+1] and zero in the last column."""
    x = np.arange(1.0, 1.0 + 2 * 3 * 4).reshape(1, 2, 3, 4, 1)
    w = np.zeros((27, 1, 1))
    w[U.tap_index(0, 0, 1)] = 1.0
    y = U.conv3d(x, w)[0, ..., 0]
    assert y[0, 0].tolist() == [2.0, 3.0, 4.0, 0.0]
    assert y[1, 2].tolist() == [22.0, 23.0, 24.0, 0.0]
    w[:] = 0.0
    w[U.tap_index(-1, 0, 0)] = 1.0  # the plane below
    y = U.conv3d(x, w)[0, ..., 0]
    assert np.all(y[0] == 0.0) and y[1, 0, 0] == 1.0


def test_conv3d_samples_independent():
    """Samples never see each other's values through the zero boundary."""
    rng = np.random.default_rng(3)
    x = _rand(rng, 3, 4, 4, 4, 2)
    w = _rand(rng, 27, 3, 2)
    y = U.conv3d(x, w)
    for s in range(3):
        np.testing.assert_allclose(y[s:s + 1], U.conv3d(x[s:s + 1], w), rtol=1e-13, atol=1e-13)


def test_conv3d_adjoint_and_wgrad_identities():
    """<conv(x, w), y> = <x, conv^T(y, w)> = sum(w * wgrad(x, y))."""
    rng = np.random.default_rng(4)
    x = _rand(rng, 2, 4, 3, 5, 3)
    y = _rand(rng, 2, 4, 3, 5, 4)
    w = _rand(rng, 27, 4, 3)
    lhs = float(np.sum(U.conv3d(x, w) * y))
    assert abs(lhs - float(np.sum(x * U.conv3d_adjoint(y, w)))) < 1e-10 * abs(lhs) + 1e-10
    assert abs(lhs - float(np.sum(w * U.conv3d_wgrad(x, y)))) < 1e-10 * abs(lhs) + 1e-10


def test_pool_and_upsample_bruteforce_and_adjoints():
    rng = np.random.default_rng(5)
    x = _rand(rng, 2, 4, 6, 2, 3)
    p = U.avgpool2(x)
    for s, k, j, i, c in [(0, 0, 0, 0, 0), (1, 1, 2, 0, 2), (0, 1, 1, 0, 1)]:
        ref = np.mean([x[s, 2 * k + a, 2 * j + b, 2 * i + d, c]
                       for a in (0, 1) for b in (0, 1) for d in (0, 1)])
        assert abs(p[s, k, j, i, c] - ref) < 1e-14
    u = U.upsample2(p)
    assert u.shape == x.shape and u[1, 3, 5, 1, 2] == p[1, 1, 2, 0, 2]
    y = _rand(rng, *p.shape)
    assert abs(np.sum(p * y) - np.sum(x * U.avgpool2_adjoint(y))) < 1e-10
    z = _rand(rng, *x.shape)
    assert abs(np.sum(U.upsample2(y) * z) - np.sum(y * U.upsample2_adjoint(z))) < 1e-10


def _tiny_net(seed=7):
    p = U.init_params(seed)
    rng = np.random.default_rng(seed + 1)
    for i in range(7):  # non-zero biases so that every bias gradient is exercised
        p["b%d" % i] = 0.1 * rng.standard_normal(p["b%d" % i].shape)
    inp = rng.standard_normal((2, 4, 4, 8, 2))
    g = rng.standard_normal((2, 4, 4, 8))
    return p, inp, g


def test_unet_backward_finite_differences():
    """Directional derivative of <z, g> along a random parameter direction and
    single-entry derivatives, by central differences."""
    p, inp, g = _tiny_net()
    z, cache = U.unet_forward(p, inp)
    grads = U.unet_backward(p, cache, g)

    def f(q):
        return float(np.sum(U.unet_forward(q, inp)[0] * g))

    rng = np.random.default_rng(11)
    dirn = {k: rng.standard_normal(v.shape) for k, v in p.items()}
    h = 1e-6
    fp = f({k: p[k] + h * dirn[k] for k in p})
    fm = f({k: p[k] - h * dirn[k] for k in p})
    fd = (fp - fm) / (2 * h)
    an = sum(float(np.sum(grads[k] * dirn[k])) for k in p)
    assert abs(fd - an) < 1e-5 * max(1.0, abs(an)), (fd, an)
    for k in p:
        idx = tuple(int(rng.integers(0, n)) for n in p[k].shape)
        q = {kk: vv.copy() for kk, vv in p.items()}
        q[k][idx] += h
        fp = f(q)
        q[k][idx] -= 2 * h
        fm = f(q)
        fd = (fp - fm) / (2 * h)
        assert abs(fd - grads[k][idx]) < 1e-5 * max(1.0, abs(fd)), (k, idx, fd, grads[k][idx])


def test_unet_shapes_and_skip_paths():
    """With W1 and the coarse biases zero the coarse branch carries nothing,
    so z sees the input only through W0, W5 and W6: three 3x3x3 layers, a
    point perturbation reaches at most 3 cells away."""
    p, inp, _ = _tiny_net()
    q = {k: v.copy() for k, v in p.items()}
    q["W1"][:] = 0.0
    q["b1"][:] = 0.0
    q["b3"][:] = 0.0
    q["b2"][:] = 0.0
    q["b4"][:] = 0.0
    base = np.zeros_like(inp)
    pert = base.copy()
    pert[0, 0, 0, 0, 0] = 1.0
    z0 = U.unet_forward(q, base)[0]
    z1 = U.unet_forward(q, pert)[0]
    diff = np.abs(z1 - z0)[0]
    far = np.zeros_like(diff, dtype=bool)
    far[:, :, 4:] = True  # x >= 4 is beyond radius 3 of the source at x = 0
    assert np.all(diff[far] == 0.0)
    assert np.any(diff[:, :, :4] != 0.0)
    assert np.all(U.unet_forward(q, pert)[0][1] == z0[1])  # other sample untouched


def test_precondition_homogeneous():
    p, inp, _ = _tiny_net()
    rng = np.random.default_rng(3)
    r = rng.standard_normal((2, 4, 4, 8))
    lnk = rng.standard_normal((2, 4, 4, 8))
    m1 = U.precondition(p, r, lnk)
    m2 = U.precondition(p, 3.5 * r, lnk)
    np.testing.assert_allclose(m2, 3.5 * m1, rtol=1e-12, atol=1e-14)


def test_restrict_prolong_pins():
    """R is the block mean (loops), P copies the parent, R P = identity, and
    P is 8 times the adjoint of R."""
    rng = np.random.default_rng(12)
    v = rng.standard_normal((2, 4, 6, 8))
    rv = U.restrict2(v)
    for s_, k, j, i in [(0, 0, 0, 0), (1, 1, 2, 3), (0, 1, 1, 2)]:
        ref = np.mean([v[s_, 2 * k + a, 2 * j + b, 2 * i + c] for a in (0, 1) for b in (0, 1)
                       for c in (0, 1)])
        assert abs(rv[s_, k, j, i] - ref) < 1e-14
    w = rng.standard_normal(rv.shape)
    pw = U.prolong2(w)
    assert pw[1, 3, 5, 7] == w[1, 1, 2, 3]
    np.testing.assert_allclose(U.restrict2(pw), w, rtol=0, atol=1e-15)
    assert abs(np.sum(pw * v) - 8.0 * np.sum(w * rv)) < 1e-10


def test_precondition_coarse_homogeneous_and_smooth():
    p, _, _ = _tiny_net()
    rng = np.random.default_rng(13)
    r = rng.standard_normal((1, 8, 8, 16))
    lnk = rng.standard_normal((1, 8, 8, 16))
    m1 = U.precondition_coarse(p, r, lnk)
    np.testing.assert_allclose(U.precondition_coarse(p, 2.5 * r, lnk), 2.5 * m1, rtol=1e-12,
                               atol=1e-14)
    # constant on every 2x2x2 block
    assert np.all(m1[:, 0::2, 0::2, 0::2] == m1[:, 1::2, 1::2, 1::2])
    # two levels: constant on 4x4x4 blocks, equal to one level applied to R r
    r2 = rng.standard_normal((1, 16, 16, 16))
    l2 = rng.standard_normal((1, 16, 16, 16))
    m2 = U.precondition_coarse(p, r2, l2, levels=2)
    assert np.all(m2[:, 0::4, 0::4, 0::4] == m2[:, 3::4, 3::4, 3::4])
    np.testing.assert_allclose(
        m2, U.prolong2(U.precondition_coarse(p, U.restrict2(r2), U.restrict2(l2), levels=1)),
        rtol=1e-13, atol=1e-15)


def _tpfa_problem(oracle_mod, nx=6, ny=5, nz=4, seed=3):
    O = oracle_mod
    g = O.Grid(nx, ny, nz)
    K = synth.lognormal_field(nx, ny, nz, 1.0, seed)
    mask, pD = synth.dirichlet_faces(nx, ny, nz, "x", 1.0, 0.0)
    A = O.assemble(g, K, mask)
    b = O.rhs(g, K, mask, None, pD)
    return O, A, b


def test_anorm_loss(oracle_mod):
    O, A, b = _tpfa_problem(oracle_mod)
    e = O.cholesky_solve(A.dense(), b)
    L, grad = U.anorm_loss(e, e, A.matvec)
    assert L == 0.0 and np.all(grad == 0.0)
    L, _ = U.anorm_loss(np.zeros_like(e), e, A.matvec)
    assert abs(L - 1.0) < 1e-14
    rng = np.random.default_rng(0)
    mr = e + 0.1 * rng.standard_normal(e.shape)
    L, grad = U.anorm_loss(mr, e, A.matvec)
    d = rng.standard_normal(e.shape)
    h = 1e-6
    fd = (U.anorm_loss(mr + h * d, e, A.matvec)[0] - U.anorm_loss(mr - h * d, e, A.matvec)[0]) / (2 * h)
    assert abs(fd - grad @ d) < 1e-7 * max(1.0, abs(fd))


def test_anorm_loss_scaled(oracle_mod):
    """Equals the plain A-norm loss at the scale found by a library 1-D
    minimiser; invariant to the scale of Mr; zero when Mr is a multiple of
    e; gradient by central differences."""
    import scipy.optimize
    O, A, b = _tpfa_problem(oracle_mod)
    e = O.cholesky_solve(A.dense(), b)
    rng = np.random.default_rng(4)
    mr = e + 0.3 * np.abs(e).max() * rng.standard_normal(e.shape)
    L, grad = U.anorm_loss_scaled(mr, b, e, A.matvec)
    res = scipy.optimize.minimize_scalar(lambda c: U.anorm_loss(c * mr, e, A.matvec)[0],
                                         bracket=(0.1, 10.0), tol=1e-12)
    assert abs(L - res.fun) < 1e-9
    L2, _ = U.anorm_loss_scaled(-3.0 * mr, b, e, A.matvec)
    assert abs(L2 - L) < 1e-12
    L0, g0 = U.anorm_loss_scaled(2.5 * e, b, e, A.matvec)
    assert abs(L0) < 1e-12 and np.abs(g0).max() < 1e-9 * np.abs(b).max() / np.abs(e).max()
    d = rng.standard_normal(e.shape)
    h = 1e-6 * np.abs(mr).max()
    fd = (U.anorm_loss_scaled(mr + h * d, b, e, A.matvec)[0] -
          U.anorm_loss_scaled(mr - h * d, b, e, A.matvec)[0]) / (2 * h)
    assert abs(fd - grad @ d) < 1e-6 * max(abs(fd), 1e-12)


def test_jacobi_blend_and_its_loss(oracle_mod):
    """The blend weight minimises the A-norm error (library 1-D minimiser);
    u = w (the exact Jacobi error) makes the blend exact; u = 0 gives Jacobi;
    the loss equals the minimised error and its gradient matches central
    differences."""
    import scipy.optimize
    O, A, b = _tpfa_problem(oracle_mod)
    Ad = A.dense()
    e = O.cholesky_solve(Ad, b)
    dinv = 1.0 / np.diag(Ad)
    rng = np.random.default_rng(6)
    u = rng.standard_normal(e.shape)

    def err(z):
        d = z - e
        return float(d @ A.matvec(d))

    z, c = U.jacobi_blend(u, b, dinv, A.matvec)
    res = scipy.optimize.minimize_scalar(lambda cc: err(dinv * b + cc * u), bracket=(-1, 1), tol=1e-14)
    assert abs(c - res.x) < 1e-6 * max(1.0, abs(res.x)) and abs(err(z) - res.fun) < 1e-9 * err(e * 0)
    w = e - dinv * b
    zw, cw = U.jacobi_blend(3.0 * w, b, dinv, A.matvec)
    np.testing.assert_allclose(zw, e, rtol=0, atol=1e-10 * np.abs(e).max())
    z0, c0 = U.jacobi_blend(np.zeros_like(u), b, dinv, A.matvec)
    assert c0 == 0.0 and np.array_equal(z0, dinv * b)
    L, grad = U.anorm_loss_blend(u, b, e, dinv, A.matvec)
    assert abs(L - err(z) / err(0 * e)) < 1e-10
    d = rng.standard_normal(e.shape)
    h = 1e-6
    fd = (U.anorm_loss_blend(u + h * d, b, e, dinv, A.matvec)[0] -
          U.anorm_loss_blend(u - h * d, b, e, dinv, A.matvec)[0]) / (2 * h)
    assert abs(fd - grad @ d) < 1e-6 * max(abs(fd), 1e-12)


def test_adam_closed_forms():
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    w0 = np.array([1.0, 1.0, 1.0, 1.0])
    lr, eps = 1e-2, 1e-8
    # first step: m_hat = g and v_hat = g^2 exactly, so the step is lr * g / (|g| + eps)
    w, m, v = U.adam_step(w0, g, np.zeros(4), np.zeros(4), 1, lr, eps=eps)
    np.testing.assert_allclose(w, w0 - lr * g / (np.abs(g) + eps), rtol=1e-14, atol=1e-16)
    # a constant gradient keeps m_hat = g and v_hat = g^2 at every step
    w, m, v = w0.copy(), np.zeros(4), np.zeros(4)
    for t in range(1, 26):
        w, m, v = U.adam_step(w, g, m, v, t, lr, eps=eps)
    np.testing.assert_allclose(w, w0 - 25 * lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-13)
    # the update is invariant to a positive rescaling of the gradient (eps aside)
    wa, _, _ = U.adam_step(w0[:2], g[:2], np.zeros(2), np.zeros(2), 1, lr, eps=0.0)
    wb, _, _ = U.adam_step(w0[:2], 7.0 * g[:2], np.zeros(2), np.zeros(2), 1, lr, eps=0.0)
    np.testing.assert_allclose(wa, wb, rtol=1e-15)


def test_fcg_identity_is_plain_cg(oracle_mod):
    O, A, b = _tpfa_problem(oracle_mod)
    x, it, hist = U.fcg(A.matvec, b, lambda r: r.copy(), 1e-10, 500)
    xc, st, itc, _, hc = O.cg(A, b, tol=1e-10, history=500)
    assert it == itc
    np.testing.assert_allclose(x, xc, rtol=1e-9, atol=1e-12)


def test_fcg_fixed_spd_preconditioner_matches_scipy_pcg(oracle_mod):
    """For a fixed SPD preconditioner FCG generates the PCG iterates; scipy's
    cg with the same preconditioner is the reference."""
    O, A, b = _tpfa_problem(oracle_mod)
    S = scipy.sparse.csr_matrix((A.vals, A.cols, A.rowptr), shape=(A.n, A.n))
    dinv = 1.0 / S.diagonal()
    M = scipy.sparse.linalg.LinearOperator(S.shape, matvec=lambda r: dinv * r)
    for k in (1, 3, 8):
        xs, _ = scipy.sparse.linalg.cg(S, b, rtol=1e-300, atol=0.0, maxiter=k, M=M)
        xf, itf, _ = U.fcg(A.matvec, b, lambda r: dinv * r, 1e-300, k)
        assert itf == k
        np.testing.assert_allclose(xf, xs, rtol=1e-9, atol=1e-12)


def test_fcg_exact_inverse_one_step(oracle_mod):
    O, A, b = _tpfa_problem(oracle_mod)
    Ad = A.dense()
    x, it, hist = U.fcg(A.matvec, b, lambda r: np.linalg.solve(Ad, r), 1e-10, 10)
    assert it == 1 and hist[-1] < 1e-12


def test_fcg_variable_preconditioner_converges(oracle_mod):
    """A preconditioner that changes every call (a random positive diagonal
    scaling) still drives FCG to the solution."""
    O, A, b = _tpfa_problem(oracle_mod)
    rng = np.random.default_rng(9)
    x, it, hist = U.fcg(A.matvec, b, lambda r: r * rng.uniform(0.5, 2.0, r.shape), 1e-10, 2000)
    assert hist[-1] <= 1e-10
    xe = O.cholesky_solve(A.dense(), b)
    np.testing.assert_allclose(x, xe, rtol=0, atol=1e-8 * np.abs(xe).max())


# --- planted mistakes: each must make at least one pin above fail ----------

def _expect_fail(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_mutants_fail_pins(monkeypatch, oracle_mod):
    shift0 = U.shift
    # an offset applied with the wrong sign in the forward convolution
    monkeypatch.setattr(U, "shift", lambda x, dz, dy, dx: shift0(x, -dz, dy, dx))
    _expect_fail(test_conv3d_bruteforce)
    monkeypatch.setattr(U, "shift", shift0)
    # adjoint without the flipped offsets
    adj0 = U.conv3d_adjoint
    monkeypatch.setattr(U, "conv3d_adjoint",
                        lambda dy, w: sum(shift0(dy, dz, a, b) @ w[t]
                                          for t, (dz, a, b) in enumerate(U.TAPS)))
    _expect_fail(test_conv3d_adjoint_and_wgrad_identities)
    monkeypatch.setattr(U, "conv3d_adjoint", adj0)
    # a weight gradient with the weight transposed per tap
    wg0 = U.conv3d_wgrad
    monkeypatch.setattr(U, "conv3d_wgrad", lambda x, dy: wg0(x, dy)[:, ::-1, :])
    _expect_fail(test_conv3d_adjoint_and_wgrad_identities)
    monkeypatch.setattr(U, "conv3d_wgrad", wg0)
    # the skip path dropped from the backward pass
    ua0 = U.upsample2_adjoint
    monkeypatch.setattr(U, "upsample2_adjoint", lambda dy: ua0(dy) * 0.5)
    _expect_fail(test_unet_backward_finite_differences)
    monkeypatch.setattr(U, "upsample2_adjoint", ua0)
    # FCG with the wrong sign of beta
    f0 = U.fcg

    def fcg_bad(apply_a, b, precond, tol, maxit, x0=None):
        x = np.zeros_like(b)
        r = b.copy()
        p = q = None
        it = 0
        while it < maxit:
            z = precond(r)
            p = z.copy() if p is None else z + (float(z @ q) / float(p @ q)) * p
            q = apply_a(p)
            a = float(p @ r) / float(p @ q)
            x, r = x + a * p, r - a * q
            it += 1
        return x, it, [0.0]

    monkeypatch.setattr(U, "fcg", fcg_bad)
    _expect_fail(test_fcg_fixed_spd_preconditioner_matches_scipy_pcg, oracle_mod)
    monkeypatch.setattr(U, "fcg", f0)
