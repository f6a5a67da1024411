"""Pins for the CPU FP64 oracle against facts fixed by physics and mathematics.

The paper prints no solution values, so each check here comes from outside
the oracle: the exact solution of the continuous problem, Darcy's law,
conservation, symmetry of the operator, a library dense solve, exact-
arithmetic termination of CG, and the equivalence of the printed Eq. 6
operator with its symmetric elimination.  Together they fail on a dropped
term, a wrong sign, a wrong mean, a transposed index or a wrong geometric
factor anywhere in assembly, right-hand side or CG.
"""
import numpy as np
import pytest

from paper_2408_03452_gb300 import synth


def _grid(O, nx, ny, nz, **kw):
    return O.Grid(nx, ny, nz, **kw)


# --- closed forms ----------------------------------------------------------

@pytest.mark.parametrize("shape", [(9, 1, 1), (9, 5, 4), (2, 3, 3)])
@pytest.mark.parametrize("geom", [dict(), dict(dx=0.5, dy=2.0, dz=3.0, mu=2.5)])
def test_linear_pressure_homogeneous(oracle_mod, shape, geom):
    """Homogeneous K, p=1 on the x=0 layer, p=0 on the last x layer: the
    pressure is linear in x and independent of y, z (Section II.A, Eq. 1)."""
    O = oracle_mod
    nx, ny, nz = shape
    g = _grid(O, nx, ny, nz, **geom)
    K = np.full(g.n, 3.7)
    mask, pD = synth.dirichlet_faces(nx, ny, nz, "x", 1.0, 0.0)
    p, _ = O.solve(g, K, mask, 0.0, None, pD, tol=1e-14)
    i = np.arange(g.n) % nx
    np.testing.assert_allclose(p, 1.0 - i / (nx - 1), rtol=0, atol=1e-12)


def _continuous_layered_solution(k, dx):
    """Exact solution of -(k(x) p')' = 0 on piecewise-constant k, sampled at
    cell centres, with p = 1 / 0 at the first / last centre.  Integrates
    1/k(x) along x: p(x) = 1 - int_{x0}^{x} dx'/k / int_{x0}^{xN} dx'/k."""
    n = len(k)
    centres = (np.arange(n) + 0.5) * dx
    edges = np.arange(n + 1) * dx

    def integral(a, b):  # int_a^b 1/k(x) dx for a <= b
        lo = np.clip(edges[:-1], a, b)
        hi = np.clip(edges[1:], a, b)
        return np.sum((hi - lo) / k)

    R = np.array([integral(centres[0], c) for c in centres])
    return 1.0 - R / R[-1]


@pytest.mark.parametrize("seed", [0, 1])
def test_series_resistance_layered(oracle_mod, seed):
    """x-layered heterogeneous K: the cell-centred solution equals the exact
    solution of the continuous 1D problem (TPFA with the harmonic face
    average is exact for layered media; an arithmetic or geometric mean
    is not)."""
    O = oracle_mod
    nx, ny, nz = 12, 3, 2
    dx = 0.7
    kx = np.exp(2.0 * synth.normal(seed, 9, np.arange(nx)))
    g = _grid(O, nx, ny, nz, dx=dx, dy=1.3, dz=0.4, mu=1.7)
    K = np.tile(kx, ny * nz)
    mask, pD = synth.dirichlet_faces(nx, ny, nz, "x", 1.0, 0.0)
    p, _ = O.solve(g, K, mask, 0.0, None, pD, tol=1e-14)
    expect = _continuous_layered_solution(kx, dx)
    np.testing.assert_allclose(p.reshape(nz, ny, nx), np.broadcast_to(expect, (nz, ny, nx)),
                               rtol=0, atol=1e-11)


@pytest.mark.parametrize("axis", ["x", "y", "z"])
def test_darcy_flux(oracle_mod, axis):
    """Total flow through a homogeneous box equals Darcy's law
    Q = k * A * dp / (mu * L) with L the distance between the Dirichlet cell
    centres (Eq. 1a); pins areas, spacings and the 1/mu mobility."""
    O = oracle_mod
    nx, ny, nz = 6, 5, 4
    dx, dy, dz, mu, k = 0.5, 2.0, 1.5, 3.0, 2.2
    g = _grid(O, nx, ny, nz, dx=dx, dy=dy, dz=dz, mu=mu)
    K = np.full(g.n, k)
    mask, pD = synth.dirichlet_faces(nx, ny, nz, axis, 1.0, 0.0)
    p, _ = O.solve(g, K, mask, 0.0, None, pD, tol=1e-14)
    flux = O.net_flux(g, K, p)
    hi = (pD == 1.0) & (mask == 1)
    Q = flux[hi].sum()
    area, L = {"x": (ny * dy * nz * dz, (nx - 1) * dx),
               "y": (nx * dx * nz * dz, (ny - 1) * dy),
               "z": (nx * dx * ny * dy, (nz - 1) * dz)}[axis]
    assert Q == pytest.approx(k * area * 1.0 / (mu * L), rel=1e-12)
    # the flux into the low-pressure layer balances it
    lo = (pD == 0.0) & (mask == 1)
    assert flux[lo].sum() == pytest.approx(-Q, rel=1e-12)


# --- invariants ------------------------------------------------------------

def _hetero_case(nx=7, ny=6, nz=5, seed=3, sigma=2.0):
    K = synth.lognormal_field(nx, ny, nz, sigma, seed)
    u = synth.uniform(seed, 7, np.arange(nx * ny * nz))
    mask = (u < 0.15).astype(np.uint8)
    d = synth.uniform(seed, 8, np.arange(nx * ny * nz), ) * 0.1
    return K, mask, d


def test_symmetry(oracle_mod):
    """x^T A y = y^T A x for the eliminated operator with scattered Dirichlet
    cells, heterogeneous K and a per-cell diagonal."""
    O = oracle_mod
    nx, ny, nz = 7, 6, 5
    g = _grid(O, nx, ny, nz, dx=0.9, dy=1.1, dz=0.8, mu=1.3)
    K, mask, d = _hetero_case(nx, ny, nz)
    A = O.assemble(g, K, mask, d)
    rng = np.random.default_rng(0)
    for _ in range(5):
        x, y = rng.standard_normal(g.n), rng.standard_normal(g.n)
        a, b = x @ A.matvec(y), y @ A.matvec(x)
        assert abs(a - b) <= 1e-12 * max(abs(a), abs(b))
    Ad = A.dense()
    np.testing.assert_allclose(Ad, Ad.T, rtol=0, atol=1e-14 * np.abs(Ad).max())
    # the operator as printed in Eq. 6 is not symmetric once Dirichlet
    # cells have interior neighbours
    Al = O.assemble(g, K, mask, d, literal=True).dense()
    assert np.abs(Al - Al.T).max() > 1e-3


def test_zero_row_sums(oracle_mod):
    """With d = 0, rows of cells without Dirichlet neighbours sum to zero
    (the diagonal equals the sum of the face transmissibilities)."""
    O = oracle_mod
    nx, ny, nz = 6, 5, 4
    g = _grid(O, nx, ny, nz, dx=0.3, dy=1.7, dz=2.0, mu=0.8)
    K = synth.lognormal_field(nx, ny, nz, 1.5, 11)
    A = O.assemble(g, K, None, 0.0)
    rs = A.matvec(np.ones(g.n))
    diag = np.array([A.vals[A.rowptr[r]] for r in range(g.n)])
    assert np.all(np.abs(rs) <= 1e-15 * diag * 8)
    mask, _ = synth.dirichlet_faces(nx, ny, nz, "z")
    A = O.assemble(g, K, mask, 0.0)
    rs = A.matvec(np.ones(g.n)).reshape(nz, ny, nx)
    diag = np.array([A.vals[A.rowptr[r]] for r in range(g.n)]).reshape(nz, ny, nx)
    inner = rs[2:-2]
    assert np.all(np.abs(inner) <= 1e-15 * diag[2:-2] * 8)
    # rows next to a Dirichlet layer keep the lifted coupling on the diagonal
    assert np.all(rs[1] > 0) and np.all(rs[-2] > 0)


def test_global_conservation(oracle_mod):
    """d > 0, no Dirichlet cells, sources q: summing all rows of A p = b gives
    sum_i d_i p_i = sum_i q_i (fluxes cancel pairwise)."""
    O = oracle_mod
    nx, ny, nz = 8, 7, 6
    g = _grid(O, nx, ny, nz)
    K = synth.lognormal_field(nx, ny, nz, 1.5, 5, layer=2)
    n = g.n
    d = 1e-2 + 0.05 * synth.uniform(5, 8, np.arange(n))
    q = np.zeros(n)
    idx, val = synth.well_pair(nx, ny, nz)
    q[idx] = val
    q[17] += 0.3
    p, _ = O.solve(g, K, None, d, q, None, tol=1e-13)
    assert np.dot(d, p) == pytest.approx(q.sum(), abs=1e-10)
    assert np.dot(d, p) == pytest.approx(0.3, abs=1e-10)


def test_point_reflection_antisymmetry(oracle_mod):
    """Homogeneous K, accumulation d > 0, injector / producer at opposite
    corners: p(c) = -p(reflection of c through the box centre)."""
    O = oracle_mod
    nx, ny, nz = 7, 6, 5
    g = _grid(O, nx, ny, nz, dx=1.0, dy=0.5, dz=2.0)
    n = g.n
    idx, val = synth.well_pair(nx, ny, nz)
    q = synth.dense_sources(n, idx, val)
    p, _ = O.solve(g, np.full(n, 4.0), None, 1e-3, q, None, tol=1e-14)
    np.testing.assert_allclose(p, -p[::-1], rtol=0, atol=1e-10 * np.abs(p).max())
    assert p[0] > 0 > p[-1]


# --- solver against library / exact-arithmetic facts ------------------------

@pytest.mark.parametrize("shape,seed", [((5, 4, 3), 0), ((8, 6, 5), 1), ((3, 9, 7), 2)])
def test_cg_and_cholesky_match_library_dense_solve(oracle_mod, shape, seed):
    O = oracle_mod
    nx, ny, nz = shape
    g = _grid(O, nx, ny, nz, dx=1.2, dy=0.7, dz=1.0, mu=1.1)
    K = synth.lognormal_field(nx, ny, nz, 1.0, seed)
    mask, pD = synth.dirichlet_faces(nx, ny, nz, "x", 1.0, 0.0)
    q = 0.1 * synth.uniform(seed, 3, np.arange(g.n))
    A = O.assemble(g, K, mask, 1e-3)
    b = O.rhs(g, K, mask, q, pD)
    ref = np.linalg.solve(A.dense(), b)
    x, st, it, _ = O.cg(A, b, tol=1e-14)
    assert st == 0
    np.testing.assert_allclose(x, ref, rtol=0, atol=1e-11 * np.abs(ref).max())
    xc = O.cholesky_solve(A.dense(), b)
    np.testing.assert_allclose(xc, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_cg_terminates_within_n(oracle_mod):
    """For an SPD system of size N with moderate condition number, CG in FP64
    reaches 1e-12 relative residual in at most N iterations."""
    O = oracle_mod
    nx, ny, nz = 4, 4, 4
    g = _grid(O, nx, ny, nz)
    K = synth.lognormal_field(nx, ny, nz, 0.5, 4)
    A = O.assemble(g, K, None, 0.05)
    ev = np.linalg.eigvalsh(A.dense())
    assert ev[0] > 0 and ev[-1] / ev[0] <= 1e3
    b = synth.uniform(4, 5, np.arange(g.n))
    x, st, it, rel = O.cg(A, b, tol=1e-12)
    assert st == 0 and it <= g.n and rel <= 1e-12
    assert np.linalg.norm(b - A.matvec(x)) <= 1e-11 * np.linalg.norm(b)


def test_literal_eq6_gives_same_iterates(oracle_mod):
    """With x0 = p^D on the Dirichlet cells, CG on the operator printed in
    Eq. 6 (couplings to Dirichlet cells kept, b = q) produces the same iterates
    as CG on the symmetric eliminated operator."""
    O = oracle_mod
    nx, ny, nz = 6, 5, 4
    g = _grid(O, nx, ny, nz)
    K = synth.lognormal_field(nx, ny, nz, 1.0, 8)
    mask, pD = synth.dirichlet_faces(nx, ny, nz, "x", 1.0, 0.25)
    q = 0.01 * synth.uniform(8, 2, np.arange(g.n))
    x0 = np.where(mask == 1, pD, 0.0)
    A = O.assemble(g, K, mask, 0.0)
    b = O.rhs(g, K, mask, q, pD)
    Al = O.assemble(g, K, mask, 0.0, literal=True)
    bl = O.rhs(g, K, mask, q, pD, literal=True)
    H = 12
    _, _, _, _, h1 = O.cg(A, b, x0=x0, tol=0.0, maxit=H, history=H)
    _, _, _, _, h2 = O.cg(Al, bl, x0=x0, tol=0.0, maxit=H, history=H)
    np.testing.assert_allclose(h1, h2, rtol=0, atol=1e-12)
    # and both end at the same solution
    xs, _ = O.solve(g, K, mask, 0.0, q, pD, tol=1e-13, x0=x0)
    xl, st, _, _ = O.cg(Al, bl, x0=x0, tol=1e-13)
    np.testing.assert_allclose(xs, xl, rtol=0, atol=1e-10)


# --- Jacobi-preconditioned CG (the oracle's reference solver on high contrast)

@pytest.mark.parametrize("shape,seed", [((5, 4, 3), 0), ((8, 6, 5), 1)])
def test_pcg_jacobi_matches_library_dense_solve(oracle_mod, shape, seed):
    O = oracle_mod
    nx, ny, nz = shape
    g = _grid(O, nx, ny, nz, dx=0.8, dy=1.3, dz=1.0, mu=0.9)
    K = synth.channelized_field(nx, ny, nz, 2.0, seed, n_channels=1, width=2, thickness=2,
                                amplitude=1.0, wavelength=8.0, contrast=1e4)
    mask, pD = synth.dirichlet_faces(nx, ny, nz, "y", 1.5, 0.0)
    A = O.assemble(g, K, mask, 1e-3)
    b = O.rhs(g, K, mask, None, pD)
    ref = np.linalg.solve(A.dense(), b)
    x, st, it, rel = O.pcg_jacobi(A, b, tol=1e-14)
    assert st == 0 and rel <= 1e-14
    np.testing.assert_allclose(x, ref, rtol=0, atol=1e-10 * np.abs(ref).max())


def test_pcg_jacobi_iterates_are_cg_on_the_scaled_system(oracle_mod):
    """PCG with M = diag(A) produces x_k = S xh_k, where xh_k are the iterates
    of plain CG on the symmetrically scaled system (S A S) xh = S b with
    S = diag(A)^(-1/2) (the textbook equivalence of preconditioned CG).  The
    scaled system is assembled here by scaling the CSR values and solved by
    the oracle's plain CG, which the pins above tie to a library solve."""
    O = oracle_mod
    nx, ny, nz = 6, 5, 4
    g = _grid(O, nx, ny, nz)
    K = synth.lognormal_field(nx, ny, nz, 2.0, 9)
    mask, pD = synth.dirichlet_faces(nx, ny, nz, "z", 1.0, 0.5)
    A = O.assemble(g, K, mask, 0.02)
    b = O.rhs(g, K, mask, None, pD)
    diag = A.dense().diagonal()
    S = 1.0 / np.sqrt(diag)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    As = O.CSR(A.n, A.rowptr, A.cols, A.vals * S[rows] * S[A.cols])
    H = 10
    _, _, _, _, hp = O.pcg_jacobi(A, b, tol=0.0, maxit=H, history=H)
    _, _, _, _, hc = O.cg(As, S * b, tol=0.0, maxit=H, history=H)
    np.testing.assert_allclose(hp, hc * S[None, :], rtol=0, atol=1e-12 * np.abs(hp).max())


@pytest.mark.parametrize("solver", ["cg", "pcg_jacobi"])
def test_solvers_match_library_sparse_solve_beyond_one_dot_block(oracle_mod, solver):
    """A grid of 72,000 cells (many blocks of the blocked dot products and
    above the threshold of the parallel loops; two layers keep the library's
    sparse factorisation fast): CG and Jacobi PCG agree with scipy's sparse
    direct solve of the same CSR."""
    sla = pytest.importorskip("scipy.sparse.linalg")
    sp = pytest.importorskip("scipy.sparse")
    O = oracle_mod
    nx, ny, nz = 200, 180, 2
    g = _grid(O, nx, ny, nz)
    K = synth.lognormal_field(nx, ny, nz, 1.0, 12)
    mask, pD = synth.dirichlet_faces(nx, ny, nz, "x", 1.0, 0.0)
    A = O.assemble(g, K, mask, 1e-2)
    b = O.rhs(g, K, mask, None, pD)
    ref = sla.spsolve(sp.csr_matrix((A.vals, A.cols, A.rowptr), shape=(A.n, A.n)).tocsc(), b)
    x, st, it, rel = getattr(O, solver)(A, b, tol=1e-13)
    assert st == 0 and rel <= 1e-13
    np.testing.assert_allclose(x, ref, rtol=0, atol=1e-9 * np.abs(ref).max())
    # the recursive residual the solver reports is the true one (dot products intact)
    assert np.linalg.norm(b - A.matvec(x)) <= 2e-13 * np.linalg.norm(b)


@pytest.mark.parametrize("solver", ["cg", "pcg_jacobi"])
def test_iterates_are_galerkin_solutions_on_krylov_spaces(oracle_mod, solver):
    """The k-th CG iterate (x0 = 0) minimises the A-norm of the error over the
    Krylov space span{z0, B z0, ..., B^(k-1) z0}, with B = A, z0 = b for CG and
    B = M^-1 A, z0 = M^-1 b for Jacobi PCG: the defining property of the
    method, independent of its recurrences.  Here the projected system is
    solved with numpy on an orthonormal basis of the space, for k = 1..5, on a
    72,000-cell grid (so every dot product of the solver spans many blocks)."""
    O = oracle_mod
    nx, ny, nz = 200, 180, 2
    g = _grid(O, nx, ny, nz)
    K = synth.lognormal_field(nx, ny, nz, 1.0, 13)
    A = O.assemble(g, K, None, 0.05)
    b = synth.uniform(13, 4, np.arange(g.n)) - 0.5
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    dg = np.zeros(A.n)
    np.add.at(dg, rows[A.cols == rows], A.vals[A.cols == rows])
    minv = 1.0 / dg
    pre = (lambda v: minv * v) if solver == "pcg_jacobi" else (lambda v: v)
    H = 5
    _, _, _, _, hist = getattr(O, solver)(A, b, tol=0.0, maxit=H, history=H)
    V = [pre(b)]
    for k in range(1, H + 1):
        Q, _ = np.linalg.qr(np.stack(V, axis=1))
        AQ = np.stack([A.matvec(Q[:, i]) for i in range(k)], axis=1)
        y = np.linalg.solve(Q.T @ AQ, Q.T @ b)
        xk = Q @ y
        np.testing.assert_allclose(hist[k - 1], xk, rtol=0, atol=1e-9 * np.abs(xk).max())
        V.append(pre(A.matvec(V[-1])))


def test_pcg_jacobi_terminates_within_n(oracle_mod):
    O = oracle_mod
    g = _grid(O, 4, 4, 4)
    K = synth.lognormal_field(4, 4, 4, 3.0, 2)
    A = O.assemble(g, K, None, 0.05)
    b = synth.uniform(2, 5, np.arange(g.n))
    x, st, it, rel = O.pcg_jacobi(A, b, tol=1e-12)
    assert st == 0 and it <= g.n
    assert np.linalg.norm(b - A.matvec(x)) <= 1e-11 * np.linalg.norm(b)


def test_parallel_loops_do_not_depend_on_the_thread_count(oracle_mod, tmp_path):
    """Dot products sum fixed blocks in a fixed order and every row is
    computed by one thread: a solve gives bit-identical iterates with one
    thread and with all of them (a subprocess with OMP_NUM_THREADS=1)."""
    import os
    import subprocess
    import sys
    code = ("import numpy as np, sys; sys.path.insert(0, %r)\n"
            "from oracle import oracle as O\n"
            "from paper_2408_03452_gb300 import synth\n"
            "g = O.Grid(50, 40, 35); K = synth.lognormal_field(50, 40, 35, 1.5, 4)\n"
            "A = O.assemble(g, K, None, 1e-3); b = synth.uniform(1, 2, np.arange(g.n))\n"
            "x, _, it, _ = O.pcg_jacobi(A, b, tol=1e-10)\n"
            "y, _, it2, _ = O.cg(A, b, tol=1e-8)\n"
            "np.save(sys.argv[1], np.concatenate([x, y, [it, it2]]))\n"
            % os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    outs = []
    for nt in ("1", str(max(2, os.cpu_count() or 2))):
        f = str(tmp_path / f"out{nt}.npy")
        subprocess.run([sys.executable, "-c", code, f], check=True,
                       env=dict(os.environ, OMP_NUM_THREADS=nt))
        outs.append(np.load(f))
    assert np.array_equal(outs[0], outs[1])


# --- consistency of the oracle's own views of the operator ------------------

def test_coefficients_rows_and_apply_agree(oracle_mod):
    O = oracle_mod
    nx, ny, nz = 5, 4, 6
    g = _grid(O, nx, ny, nz, dx=0.6, dy=1.4, dz=1.0, mu=0.9)
    K, mask, d = _hetero_case(nx, ny, nz, seed=6)
    A = O.assemble(g, K, mask, d)
    Tx, Ty, Tz, D = O.coefficients(g, K, mask, d)
    Ad = A.dense()
    np.testing.assert_array_equal(np.diag(Ad), D)
    c = np.arange(g.n)
    i = c % nx
    j = (c // nx) % ny
    k = c // (nx * ny)
    for T, ok, step in ((Tx, i + 1 < nx, 1), (Ty, j + 1 < ny, nx), (Tz, k + 1 < nz, nx * ny)):
        cc = c[ok]
        np.testing.assert_array_equal(-Ad[cc, cc + step], T[cc])
        np.testing.assert_array_equal(-Ad[cc + step, cc], T[cc])
        assert np.all(T[~ok] == 0)
    x = synth.uniform_field(g.n, 1)
    rows = np.array([0, 7, 33, g.n - 1])
    np.testing.assert_allclose(O.apply_rows(g, K, mask, d, rows, x), A.matvec(x)[rows],
                               rtol=1e-15, atol=1e-15)
    # |A| |x| at the same rows: the dense matrix's absolute values
    np.testing.assert_allclose(O.abs_apply_rows(g, K, mask, d, rows, x),
                               (np.abs(Ad) @ np.abs(x))[rows], rtol=1e-14, atol=0)


def test_face_form_with_extra_diagonal_reproduces_csr(oracle_mod):
    """A x = sum_f T'_f (x_K - x_L) + E_K x_K with the eliminated face
    transmissibilities and the extra diagonal E reproduces the CSR product
    (the compact record of the mixed-precision path stores T' and E)."""
    O = oracle_mod
    nx, ny, nz = 6, 5, 7
    g = _grid(O, nx, ny, nz, dx=0.8, dy=1.2, dz=1.0, mu=1.4)
    K, mask, d = _hetero_case(nx, ny, nz, seed=9)
    A = O.assemble(g, K, mask, d)
    Tx, Ty, Tz, D = O.coefficients(g, K, mask, d)
    E = O.extra_diagonal(g, K, mask, d)
    x = synth.uniform_field(g.n, 2).reshape(nz, ny, nx)
    T = [a.reshape(nz, ny, nx) for a in (Tx, Ty, Tz)]
    y = E.reshape(nz, ny, nx) * x
    for axis, Tf in zip((2, 1, 0), T):
        sl_lo = [slice(None)] * 3
        sl_hi = [slice(None)] * 3
        sl_lo[axis] = slice(0, -1)
        sl_hi[axis] = slice(1, None)
        flux = Tf[tuple(sl_lo)] * (x[tuple(sl_lo)] - x[tuple(sl_hi)])
        y[tuple(sl_lo)] += flux
        y[tuple(sl_hi)] -= flux
    np.testing.assert_allclose(y.reshape(-1), A.matvec(x.reshape(-1)), rtol=1e-13, atol=1e-13)
    # D = sum of the six T' + E to rounding; E = 1 and T' = 0 around Dirichlet cells
    m = mask.astype(bool)
    assert np.all(E[m] == 1.0)


def test_transient_single_cell_closed_form(oracle_mod):
    """One cell, no faces: d (p^{n+1} - p^n) = q, so p^n = p^0 + n q / d."""
    O = oracle_mod
    g = _grid(O, 1, 1, 1)
    ps = O.transient(g, np.array([3.0]), None, 0.25, np.array([0.5]), None, np.array([1.0]), 4)
    np.testing.assert_allclose([p[0] for p in ps], [1.0 + 2.0 * k for k in range(1, 5)], rtol=1e-14)


def test_transient_mass_balance(oracle_mod):
    """No Dirichlet cells: summing the rows of each step gives
    sum d (p^{n+1} - p^n) = sum q, so sum d p^n = sum d p^0 + n sum q."""
    O = oracle_mod
    nx, ny, nz = 7, 6, 5
    g = _grid(O, nx, ny, nz, dx=0.8, dy=1.1, dz=1.3, mu=1.2)
    K = synth.lognormal_field(nx, ny, nz, 1.0, 21)
    n = g.n
    d = 0.05 + 0.1 * synth.uniform(21, 3, np.arange(n))
    q = np.zeros(n)
    q[3], q[n - 5] = 0.7, -0.2
    p0 = synth.uniform_field(n, 22)
    ps = O.transient(g, K, None, d, q, None, p0, 5, tol=1e-14)
    for k, p in enumerate(ps, start=1):
        assert np.dot(d, p) == pytest.approx(np.dot(d, p0) + k * q.sum(), rel=1e-11)


def test_transient_step_matches_dense_implicit_euler(oracle_mod):
    """Small grid with Dirichlet cells: each oracle step equals the dense
    implicit-Euler update (A_eliminated) p^{n+1} = b_lift + q + D_acc p^n
    solved with LAPACK."""
    O = oracle_mod
    nx, ny, nz = 5, 4, 3
    g = _grid(O, nx, ny, nz)
    K = synth.lognormal_field(nx, ny, nz, 1.0, 23)
    mask, pD = synth.dirichlet_faces(nx, ny, nz, "x", 2.0, 0.5)
    d = 0.3
    p0 = np.where(mask == 1, pD, 0.0)
    ps = O.transient(g, K, mask, d, None, pD, p0, 3, tol=1e-14)
    A = O.assemble(g, K, mask, d).dense()
    b0 = O.rhs(g, K, mask, None, pD)
    p = p0.copy()
    for k in range(3):
        p = np.linalg.solve(A, b0 + np.where(mask == 1, 0.0, d * p))
        np.testing.assert_allclose(ps[k], p, rtol=0, atol=1e-11)
