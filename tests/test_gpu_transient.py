"""Backward-Euler time steps through the library against the oracle's
time steps (same recipe: slightly compressible, wells, optional Dirichlet)."""
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


@pytest.mark.parametrize("shape,dirichlet,precond", [((24, 20, 16), False, 0),
                                                     ((24, 20, 16), True, 1),
                                                     ((33, 17, 9), False, 1)])
def test_transient_steps_match_oracle(tp, oracle_mod, shape, dirichlet, precond):
    from paper_2408_03452_gb300 import transient
    O = oracle_mod
    nx, ny, nz = shape
    n = nx * ny * nz
    K = synth.lognormal_field(nx, ny, nz, 1.5, 31, layer=2)
    d = 0.02 + 0.05 * synth.uniform(31, 5, np.arange(n))
    idx, val = synth.well_pair(nx, ny, nz)
    q = synth.dense_sources(n, idx, val)
    mask = pD = None
    if dirichlet:
        mask, pD = synth.dirichlet_faces(nx, ny, nz, "z", 1.0, 0.0)
    p0 = synth.uniform_field(n, 32)
    if mask is not None:
        p0 = np.where(mask == 1, pD, p0)
    steps = 4
    dev = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()
    with tp.Context(nx, ny, nz) as ctx:
        ctx.set_option("precond", precond)
        coef, coef64 = ctx.build_trans(dev(K), dev(mask), dev(d))
        ps, infos = transient.run(ctx, coef, coef64, dev(K), dev(p0), steps, d=dev(d),
                                  dirichlet=dev(mask), q=dev(q), pD=dev(pD), tol=1e-10)
        torch.cuda.synchronize()
        gp = [p.cpu().numpy() for p in ps]
    g = O.Grid(nx, ny, nz)
    ref = O.transient(g, K, mask, d, q, pD, p0, steps, tol=1e-13)
    A = O.assemble(g, K, mask, d)
    for k in range(steps):
        assert infos[k]["code"] == 0
        b = O.rhs_transient(g, K, mask, q, pD, d, gp[k - 1] if k else p0)
        # the GPU step solves its own system to 1e-10 ...
        assert np.linalg.norm(b - A.matvec(gp[k])) <= 1e-10 * np.linalg.norm(b) * 1.01
        # ... and follows the oracle's trajectory
        assert np.linalg.norm(gp[k] - ref[k]) <= 1e-7 * np.linalg.norm(ref[k])
    if mask is None:  # mass balance: sum d p^n = sum d p^0 + n sum q
        for k in range(steps):
            assert np.dot(d, gp[k]) == pytest.approx(np.dot(d, p0) + (k + 1) * q.sum(), abs=1e-7)
