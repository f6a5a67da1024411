"""FP64 oracle for the learned preconditioner: 3D convolutions, the 3-level
U-Net, its gradients, the A-norm training loss, Adam and flexible CG.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the CPU-baseline leg of the benchmark.  The CUDA library and its binding never
import anything here, and nothing here imports them.

None of this is from the finite-volume paper itself, which solves its systems
with unpreconditioned CG; it is the learned-preconditioner extension of that
solver.  Each function states the published definition it writes out:

* 3x3x3 convolution with zero padding (cross-correlation, as in deep-learning
  frameworks), its adjoint and its weight gradient;
* the U-Net of Ronneberger, Fischer and Brox (2015), here with three
  resolution levels (16, 32, 64 channels), 2x2x2 average pooling, nearest
  upsampling and additive skip connections;
* the A-norm error loss  (M r - e)^T A (M r - e) / (e^T A e)  with A e = r,
  the same loss minimised over a scalar multiple of M r, and the loss of the
  network output inside the Jacobi blend D^-1 r + c u;
* Adam (Kingma and Ba, 2015, Algorithm 1);
* flexible CG (Notay 2000, truncated to one previous direction), which for a
  fixed SPD preconditioner generates the PCG iterates.

Layout of a volume tensor: numpy array of shape (ns, nz, ny, nx, C) -- ns
independent samples, x fastest, channels last -- in float64.  Tap index of
the offset (dz, dy, dx), each in {-1, 0, 1}:  t = 9 (dz+1) + 3 (dy+1) + (dx+1).
A weight tensor has shape (27, cout, cin).
"""
from __future__ import annotations

import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def tap_index(dz: int, dy: int, dx: int) -> int:
    return 9 * (dz + 1) + 3 * (dy + 1) + (dx + 1)


def shift(x: np.ndarray, dz: int, dy: int, dx: int) -> np.ndarray:
    """out[s, z, y, x] = x[s, z+dz, y+dy, x+dx], zero where that lies outside
    the volume of the sample."""
    out = np.zeros_like(x)
    nz, ny, nx = x.shape[1:4]

    def rng(d, n):
        # destination range [lo, hi) for which the source index stays in [0, n)
        return max(0, -d), min(n, n - d)

    z0, z1 = rng(dz, nz)
    y0, y1 = rng(dy, ny)
    x0, x1 = rng(dx, nx)
    out[:, z0:z1, y0:y1, x0:x1] = x[:, z0 + dz:z1 + dz, y0 + dy:y1 + dy, x0 + dx:x1 + dx]
    return out


def conv3d(x: np.ndarray, w: np.ndarray, b: np.ndarray | None = None) -> np.ndarray:
    """y[s,v,co] = b[co] + sum_t sum_ci x[s, v + off_t, ci] w[t, co, ci]
    (zero outside the volume).  A library matrix product per tap."""
    cout = w.shape[1]
    y = np.zeros(x.shape[:4] + (cout,))
    for t, (dz, dy, dx) in enumerate(TAPS):
        y += shift(x, dz, dy, dx) @ w[t].T
    if b is not None:
        y += b
    return y


def conv3d_adjoint(dy: np.ndarray, w: np.ndarray) -> np.ndarray:
    """The adjoint of conv3d in x (input gradient):
    dx[s,u,ci] = sum_t sum_co dy[s, u - off_t, co] w[t, co, ci]."""
    cin = w.shape[2]
    dx = np.zeros(dy.shape[:4] + (cin,))
    for t, (dz, ddy, ddx) in enumerate(TAPS):
        dx += shift(dy, -dz, -ddy, -ddx) @ w[t]
    return dx


def conv3d_wgrad(x: np.ndarray, dy: np.ndarray) -> np.ndarray:
    """Weight gradient: dw[t,co,ci] = sum_{s,v} dy[s,v,co] x[s, v + off_t, ci]."""
    cin, cout = x.shape[4], dy.shape[4]
    dw = np.zeros((27, cout, cin))
    dyf = dy.reshape(-1, cout)
    for t, (dz, ddy, ddx) in enumerate(TAPS):
        dw[t] = dyf.T @ shift(x, dz, ddy, ddx).reshape(-1, cin)
    return dw


def conv3d_bruteforce(x: np.ndarray, w: np.ndarray, b: np.ndarray | None = None) -> np.ndarray:
    """The same convolution as seven nested loops (small inputs only)."""
    ns, nz, ny, nx, cin = x.shape
    cout = w.shape[1]
    y = np.zeros((ns, nz, ny, nx, cout))
    for s in range(ns):
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    for co in range(cout):
                        acc = 0.0 if b is None else float(b[co])
                        for t, (dz, dy, dx) in enumerate(TAPS):
                            kk, jj, ii = k + dz, j + dy, i + dx
                            if 0 <= kk < nz and 0 <= jj < ny and 0 <= ii < nx:
                                for ci in range(cin):
                                    acc += x[s, kk, jj, ii, ci] * w[t, co, ci]
                        y[s, k, j, i, co] = acc
    return y


def avgpool2(x: np.ndarray) -> np.ndarray:
    """Mean over each 2x2x2 block of children (all extents even)."""
    ns, nz, ny, nx, c = x.shape
    return x.reshape(ns, nz // 2, 2, ny // 2, 2, nx // 2, 2, c).mean(axis=(2, 4, 6))


def avgpool2_adjoint(dy: np.ndarray) -> np.ndarray:
    """Adjoint of avgpool2: each child receives 1/8 of its parent's value."""
    return upsample2(dy) / 8.0


def upsample2(x: np.ndarray) -> np.ndarray:
    """Nearest-neighbour 2x upsampling: child (z,y,x) copies parent (z/2,y/2,x/2)."""
    return x.repeat(2, axis=1).repeat(2, axis=2).repeat(2, axis=3)


def upsample2_adjoint(dy: np.ndarray) -> np.ndarray:
    """Adjoint of upsample2: each parent receives the sum of its 8 children."""
    return avgpool2(dy) * 8.0


def relu(x):
    return np.maximum(x, 0.0)


# ----------------------------------------------------------------------------
# The U-Net.  Levels L0 (full resolution), L1 (half), L2 (quarter):
#   e0 = relu(conv(in; W0 2->16))          L0
#   e1 = relu(conv(pool(e0); W1 16->32))   L1
#   e2 = relu(conv(pool(e1); W2 32->64))   L2
#   d2 = relu(conv(e2; W3 64->32))         L2
#   s1 = up(d2) + e1                       L1
#   d1 = relu(conv(s1; W4 32->16))         L1
#   s0 = up(d1) + e0                       L0
#   d0 = relu(conv(s0; W5 16->16))         L0
#   z  = conv(d0; W6 16->1)                L0   (no activation)
# ----------------------------------------------------------------------------
LAYERS = [("W0", 2, 16), ("W1", 16, 32), ("W2", 32, 64), ("W3", 64, 32),
          ("W4", 32, 16), ("W5", 16, 16), ("W6", 16, 1)]


def init_params(seed: int, scale: float = 1.0) -> dict:
    """He-style initial weights, N(0, 2/(27 cin)) * scale, zero biases."""
    rng = np.random.default_rng(seed)
    p = {}
    for i, (name, cin, cout) in enumerate(LAYERS):
        p[name] = rng.standard_normal((27, cout, cin)) * np.sqrt(2.0 / (27 * cin)) * scale
        p["b%d" % i] = np.zeros(cout)
    return p


def unet_forward(p: dict, inp: np.ndarray, store=None):
    """inp (ns, nz, ny, nx, 2) -> (z (ns, nz, ny, nx), cache).

    store, if given, is applied to every tensor the network keeps (the input,
    each activation, each pooled, summed or output tensor), e.g. a rounding
    to the storage precision of an implementation; by default every value
    stays exact (FP64)."""
    st = store or (lambda a: a)
    c = {"in": st(inp)}
    c["e0"] = st(relu(conv3d(c["in"], p["W0"], p["b0"])))
    c["p0"] = st(avgpool2(c["e0"]))
    c["e1"] = st(relu(conv3d(c["p0"], p["W1"], p["b1"])))
    c["p1"] = st(avgpool2(c["e1"]))
    c["e2"] = st(relu(conv3d(c["p1"], p["W2"], p["b2"])))
    c["d2"] = st(relu(conv3d(c["e2"], p["W3"], p["b3"])))
    c["s1"] = st(upsample2(c["d2"]) + c["e1"])
    c["d1"] = st(relu(conv3d(c["s1"], p["W4"], p["b4"])))
    c["s0"] = st(upsample2(c["d1"]) + c["e0"])
    c["d0"] = st(relu(conv3d(c["s0"], p["W5"], p["b5"])))
    z = st(conv3d(c["d0"], p["W6"], p["b6"]))[..., 0]
    return z, c


def unet_backward(p: dict, c: dict, dz: np.ndarray, store=None) -> dict:
    """Reverse-mode derivative of unet_forward: dz (ns, nz, ny, nx) -> grads
    of every weight and bias (same keys as the parameters).  store, if given,
    is applied to every activation gradient that is kept (see unet_forward)."""
    st = store or (lambda a: a)
    g = {}

    def layer_back(name, bname, xin, dpre):
        g[name] = conv3d_wgrad(xin, dpre)
        g[bname] = dpre.sum(axis=(0, 1, 2, 3))
        return st(conv3d_adjoint(dpre, p[name]))

    dpre6 = st(dz)[..., None]
    dd0 = layer_back("W6", "b6", c["d0"], dpre6)
    ds0 = layer_back("W5", "b5", c["s0"], dd0 * (c["d0"] > 0))
    dd1 = st(upsample2_adjoint(ds0))
    de0 = ds0.copy()
    ds1 = layer_back("W4", "b4", c["s1"], dd1 * (c["d1"] > 0))
    dd2 = st(upsample2_adjoint(ds1))
    de1 = ds1.copy()
    de2 = layer_back("W3", "b3", c["e2"], dd2 * (c["d2"] > 0))
    dp1 = layer_back("W2", "b2", c["p1"], de2 * (c["e2"] > 0))
    de1 = st(de1 + avgpool2_adjoint(dp1))
    dp0 = layer_back("W1", "b1", c["p0"], de1 * (c["e1"] > 0))
    de0 = st(de0 + avgpool2_adjoint(dp0))
    layer_back("W0", "b0", c["in"], de0 * (c["e0"] > 0))
    return g


def net_input(r: np.ndarray, lnk: np.ndarray):
    """Stack (r / rms(r), ln K) per sample; returns (inp, rms[ns]).  r and lnk
    have shape (ns, nz, ny, nx)."""
    rms = np.sqrt(np.mean(r.reshape(r.shape[0], -1) ** 2, axis=1))
    rn = r / rms[:, None, None, None]
    return np.stack([rn, lnk], axis=-1), rms


def precondition(p: dict, r: np.ndarray, lnk: np.ndarray) -> np.ndarray:
    """M(r) = rms(r) * net(r / rms(r), ln K): homogeneous of degree one in r."""
    inp, rms = net_input(r, lnk)
    z, _ = unet_forward(p, inp)
    return z * rms[:, None, None, None]


def restrict2(v: np.ndarray) -> np.ndarray:
    """Scalar field (ns, nz, ny, nx) -> the mean of each 2x2x2 block of cells."""
    return avgpool2(v[..., None])[..., 0]


def prolong2(v: np.ndarray) -> np.ndarray:
    """Scalar field on the 2x coarser grid -> each fine cell takes its parent's value."""
    return upsample2(v[..., None])[..., 0]


def precondition_coarse(p: dict, r: np.ndarray, lnk: np.ndarray, levels: int = 1) -> np.ndarray:
    """The network applied on the 2^levels coarser grid: P^l net(R^l r, R^l ln K),
    with R the 2x2x2 mean and P the nearest prolongation (homogeneous of
    degree one in r, like precondition)."""
    for _ in range(levels):
        r, lnk = restrict2(r), restrict2(lnk)
    u = precondition(p, r, lnk)
    for _ in range(levels):
        u = prolong2(u)
    return u


# ----------------------------------------------------------------------------
# Loss, optimiser, solver
# ----------------------------------------------------------------------------
def anorm_loss(mr: np.ndarray, e: np.ndarray, apply_a):
    """L = (Mr - e)^T A (Mr - e) / (e^T A e) and dL/dMr = 2 A (Mr - e) / (e^T A e)
    for one sample (flat vectors); apply_a(v) returns A v."""
    d = mr - e
    ad = apply_a(d)
    eae = float(e @ apply_a(e))
    return float(d @ ad) / eae, 2.0 * ad / eae


def anorm_loss_scaled(mr: np.ndarray, r: np.ndarray, e: np.ndarray, apply_a):
    """The A-norm loss of the best multiple of Mr:  min_c L(c Mr) with
    L(v) = (v - e)^T A (v - e) / (e^T A e) and A e = r.  The minimiser is
    c* = Mr^T r / Mr^T A Mr, giving
        L* = 1 - (Mr^T r)^2 / ((Mr^T A Mr)(e^T A e)),
    which is invariant to the scale of Mr (as CG is to the scale of its
    preconditioner).  Returns (L*, dL*/dMr) with
        dL*/dMr = (2 a / (b g)) ((a / b) A Mr - r),  a = Mr^T r, b = Mr^T A Mr,
    g = e^T A e."""
    amr = apply_a(mr)
    a = float(mr @ r)
    b = float(mr @ amr)
    g = float(e @ apply_a(e))
    return 1.0 - a * a / (b * g), (2.0 * a / (b * g)) * ((a / b) * amr - r)


def jacobi_blend(u: np.ndarray, r: np.ndarray, dinv: np.ndarray, apply_a):
    """The preconditioner z = D^-1 r + c u with the A-norm-optimal weight:
    c* minimises ||D^-1 r + c u - e||_A over c, where A e = r, which gives
        c* = (u^T r - (A u)^T D^-1 r) / (u^T A u)
    (c* = 0 when u^T A u is not positive).  Returns (z, c*)."""
    au = apply_a(u)
    den = float(u @ au)
    c = (float(u @ r) - float(au @ (dinv * r))) / den if den > 0 else 0.0
    return dinv * r + c * u, c


def anorm_loss_blend(u: np.ndarray, r: np.ndarray, e: np.ndarray, dinv: np.ndarray, apply_a):
    """Training loss of the network output u inside jacobi_blend: the A-norm
    error of the blended preconditioner relative to ||e||_A,
        L = min_c ||D^-1 r + c u - e||_A^2 / ||e||_A^2
          = (w^T A w - (u^T s)^2 / (u^T A u)) / (e^T A e),
    with w = e - D^-1 r (the error left by one Jacobi step) and
    s = A w = r - A D^-1 r.  Returns (L, dL/du)."""
    w = e - dinv * r
    sv = r - apply_a(dinv * r)
    au = apply_a(u)
    a = float(u @ sv)
    b = float(u @ au)
    g = float(e @ apply_a(e))
    L = (float(w @ apply_a(w)) - a * a / b) / g
    return L, (2.0 * a / (b * g)) * ((a / b) * au - sv)


def adam_step(w, g, m, v, t: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015, Algorithm 1); t counts from 1.
    Returns the new (w, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v


def fcg(apply_a, b: np.ndarray, precond, tol: float, maxit: int, x0=None):
    """Flexible CG with one retained direction (Notay 2000):
        r0 = b - A x0,  z_k = M(r_k),
        p_0 = z_0,  p_k = z_k - (z_k^T q_{k-1} / p_{k-1}^T q_{k-1}) p_{k-1},
        q_k = A p_k,  alpha_k = p_k^T r_k / p_k^T q_k,
        x_{k+1} = x_k + alpha_k p_k,  r_{k+1} = r_k - alpha_k q_k,
    stopping when ||r|| <= tol ||b||.  Returns (x, iterations, history of
    ||r_k|| / ||b||)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply_a(x)
    bn = float(np.linalg.norm(b))
    hist = [float(np.linalg.norm(r)) / bn]
    p = q = None
    it = 0
    while hist[-1] > tol and it < maxit:
        z = precond(r)
        if p is None:
            p = z.copy()
        else:
            p = z - (float(z @ q) / float(p @ q)) * p
        q = apply_a(p)
        alpha = float(p @ r) / float(p @ q)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        hist.append(float(np.linalg.norm(r)) / bn)
    return x, it, hist
