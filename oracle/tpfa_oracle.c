/*
 * CPU FP64 oracle for the matrix-free TPFA pressure solve.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this library.  The product path (the
 * CUDA library) shares no code with it and never calls it.
 *
 * What it computes, written as the plain definitions of the paper
 * ("Matrix-Free Finite Volume Kernels on a Dataflow Architecture",
 * arXiv 2408.03452), in double precision, with an explicit CSR matrix:
 *
 *   Section II.A, Eq. 4   two-point flux f_KL = Y_KL * lambda_KL * (p_L - p_K).
 *                         Y_KL (geometry + permeability) is not printed; the
 *                         standard TPFA half-transmissibility form is used:
 *                         Y = A_f / (h/(2 k_K) + h/(2 k_L)), the harmonic mean
 *                         of the two cell permeabilities for unit cells.
 *                         lambda_KL = arithmetic mean of the two (equal)
 *                         mobilities = 1/mu.
 *   Section II.A, Eq. 3   constrained residual: cells in the Dirichlet set
 *                         T^D carry the row p_K - p_K^D.
 *   Section II.A, Eq. 5-6 the operator J x.  Eq. 6 is printed with the sign
 *                         that makes interior rows negative semidefinite
 *                         while the text calls J SPD; the positive form
 *                         (A x)_K = sum_L T_KL (x_K - x_L) + d_K x_K is used.
 *                         Couplings from interior rows to Dirichlet cells are
 *                         moved to the right-hand side, which makes A
 *                         symmetric; orc_assemble_literal keeps them, as
 *                         Eq. 6 prints them, for the equivalence check.
 *   Section II.A, Alg. 1  conjugate gradient (Hestenes-Stiefel form).
 *
 * Readings where the paper is silent (no-flow outer boundary faces, the
 * accumulation diagonal d, sources q, the stopping rule) are the same ones
 * the CUDA path uses and are listed in the project's design notes.
 *
 * Layout: flat index c = i + nx*(j + ny*k), X innermost, Z outermost
 * (Section IV).  Face order for every sum: -x, +x, -y, +y, -z, +z.
 *
 * Compile with -ffp-contract=off so that no multiply-add is fused, and with
 * -fopenmp: the matrix-vector product, the vector updates and the CSR
 * assembly run their rows on all host threads (each row is computed by one
 * thread, so the values do not depend on the thread count); dot products add
 * fixed blocks of DOT_BLOCK terms each, then the block sums in order, so
 * they do not depend on the thread count either.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define DOT_BLOCK 4096
/* loops over fewer rows run on one thread (thread start-up would dominate) */
#define PAR_MIN 65536

/* threads the parallel loops use */
int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

typedef struct {
  int64_t nx, ny, nz;
  double dx, dy, dz, mu;
} orc_grid;

static int64_t ncells(const orc_grid* g) { return g->nx * g->ny * g->nz; }

/* Eq. 4: Y_KL * lambda_KL for the face between lower cell K and upper cell L
 * along one axis; a = face area / mu, h = cell size along the axis. */
static double face_trans(double kK, double kL, double a_over_mu, double h) {
  double half = 0.5 * h;
  return a_over_mu / (half / kK + half / kL);
}

/* neighbour of cell c through face f (0..5 = -x,+x,-y,+y,-z,+z); -1 if the
 * face is on the domain boundary (no-flow). */
static int64_t neighbour(const orc_grid* g, int64_t c, int f) {
  int64_t i = c % g->nx, j = (c / g->nx) % g->ny, k = c / (g->nx * g->ny);
  switch (f) {
    case 0: return i > 0 ? c - 1 : -1;
    case 1: return i + 1 < g->nx ? c + 1 : -1;
    case 2: return j > 0 ? c - g->nx : -1;
    case 3: return j + 1 < g->ny ? c + g->nx : -1;
    case 4: return k > 0 ? c - g->nx * g->ny : -1;
    default: return k + 1 < g->nz ? c + g->nx * g->ny : -1;
  }
}

/* transmissibility of face f of cell c (f must have a neighbour n) */
static double face_T(const orc_grid* g, const double* K, int64_t c, int f, int64_t n) {
  int axis = f / 2;
  double a = axis == 0 ? (g->dy * g->dz) / g->mu
           : axis == 1 ? (g->dx * g->dz) / g->mu
                       : (g->dx * g->dy) / g->mu;
  double h = axis == 0 ? g->dx : axis == 1 ? g->dy : g->dz;
  int64_t lo = (f % 2 == 0) ? n : c, hi = (f % 2 == 0) ? c : n;
  return face_trans(K[lo], K[hi], a, h);
}

static int is_dir(const uint8_t* mask, int64_t c) { return mask != NULL && mask[c] != 0; }
static double dval(const double* d, double d0, int64_t c) { return d != NULL ? d[c] : d0; }

/* Row c of the symmetric (eliminated) matrix A.  Returns the entry count
 * (<= 7); the diagonal comes first. */
int orc_row(const orc_grid* g, const double* K, const uint8_t* mask, const double* d, double d0,
            int64_t c, int64_t* cols, double* vals) {
  if (is_dir(mask, c)) { cols[0] = c; vals[0] = 1.0; return 1; }
  int m = 1;
  double diag = 0.0;
  for (int f = 0; f < 6; ++f) {
    int64_t n = neighbour(g, c, f);
    if (n < 0) continue;
    double T = face_T(g, K, c, f, n);
    diag += T;
    if (!is_dir(mask, n)) { cols[m] = n; vals[m] = -T; ++m; }
  }
  cols[0] = c;
  vals[0] = diag + dval(d, d0, c);
  return m;
}

/* Same row as printed by Eq. 6 (positive sign): interior rows keep their
 * couplings to Dirichlet neighbours. */
static int orc_row_literal(const orc_grid* g, const double* K, const uint8_t* mask, const double* d,
                           double d0, int64_t c, int64_t* cols, double* vals) {
  if (is_dir(mask, c)) { cols[0] = c; vals[0] = 1.0; return 1; }
  int m = 1;
  double diag = 0.0;
  for (int f = 0; f < 6; ++f) {
    int64_t n = neighbour(g, c, f);
    if (n < 0) continue;
    double T = face_T(g, K, c, f, n);
    diag += T;
    cols[m] = n; vals[m] = -T; ++m;
  }
  cols[0] = c;
  vals[0] = diag + dval(d, d0, c);
  return m;
}

/* CSR assembly.  rowptr has N+1 entries, cols/vals room for 7N. Returns nnz.
 * Rows are first built at a fixed stride of 7 (in parallel), then packed in
 * row order. */
int64_t orc_assemble(const orc_grid* g, const double* K, const uint8_t* mask, const double* d,
                     double d0, int literal, int64_t* rowptr, int64_t* cols, double* vals) {
  int64_t N = ncells(g);
#pragma omp parallel for schedule(static) if (N >= PAR_MIN)
  for (int64_t c = 0; c < N; ++c) {
    int m = literal ? orc_row_literal(g, K, mask, d, d0, c, cols + 7 * c, vals + 7 * c)
                    : orc_row(g, K, mask, d, d0, c, cols + 7 * c, vals + 7 * c);
    rowptr[c + 1] = m;
  }
  rowptr[0] = 0;
  for (int64_t c = 0; c < N; ++c) rowptr[c + 1] += rowptr[c];
  /* pack: row c moves from 7c down to rowptr[c] <= 7c, so rows are moved in
   * increasing order and never overwrite a row not yet moved */
  for (int64_t c = 0; c < N; ++c) {
    int64_t m = rowptr[c + 1] - rowptr[c];
    if (rowptr[c] == 7 * c) continue;
    for (int64_t e = 0; e < m; ++e) {
      cols[rowptr[c] + e] = cols[7 * c + e];
      vals[rowptr[c] + e] = vals[7 * c + e];
    }
  }
  return rowptr[N];
}

/* Right-hand side of A p = b: Dirichlet rows carry p^D (Eq. 3); interior rows
 * carry the source q plus the lifted couplings to Dirichlet neighbours.  With
 * literal != 0 the couplings stay in the operator, so b = q on interior rows. */
void orc_rhs(const orc_grid* g, const double* K, const uint8_t* mask, const double* q,
             const double* pD, int literal, double* b) {
  int64_t N = ncells(g);
  for (int64_t c = 0; c < N; ++c) {
    if (is_dir(mask, c)) { b[c] = pD != NULL ? pD[c] : 0.0; continue; }
    double s = q != NULL ? q[c] : 0.0;
    if (!literal && mask != NULL) {
      for (int f = 0; f < 6; ++f) {
        int64_t n = neighbour(g, c, f);
        if (n < 0 || !is_dir(mask, n)) continue;
        s += face_T(g, K, c, f, n) * (pD != NULL ? pD[n] : 0.0);
      }
    }
    b[c] = s;
  }
}

/* Right-hand side of one backward-Euler step of the slightly compressible
 * problem (Section II.A, implicit time discretisation): the accumulation
 * d_K (p_K^{n+1} - p_K^n) joins the flux balance, so the known part
 * d_K p_K^n adds to the interior rows of orc_rhs. */
void orc_rhs_transient(const orc_grid* g, const double* K, const uint8_t* mask, const double* q,
                       const double* pD, const double* d, double d0, const double* p_prev,
                       double* b) {
  orc_rhs(g, K, mask, q, pD, 0, b);
  int64_t N = ncells(g);
  for (int64_t c = 0; c < N; ++c)
    if (!is_dir(mask, c)) b[c] += dval(d, d0, c) * p_prev[c];
}

/* The eliminated operator as a coefficient set: for each cell the +x, +y, +z
 * face transmissibility (0 on the outer boundary and on faces that touch a
 * Dirichlet cell) and the diagonal (1 on Dirichlet cells). */
void orc_coefficients(const orc_grid* g, const double* K, const uint8_t* mask, const double* d,
                      double d0, double* Tx, double* Ty, double* Tz, double* D) {
  int64_t N = ncells(g);
  int64_t cols[7];
  double vals[7];
  for (int64_t c = 0; c < N; ++c) {
    double* out[3] = {Tx, Ty, Tz};
    for (int axis = 0; axis < 3; ++axis) {
      int f = 2 * axis + 1;
      int64_t n = neighbour(g, c, f);
      out[axis][c] = (n < 0 || is_dir(mask, c) || is_dir(mask, n)) ? 0.0 : face_T(g, K, c, f, n);
    }
    orc_row(g, K, mask, d, d0, c, cols, vals);
    D[c] = vals[0];
  }
}

/* The same operator written as face terms plus a diagonal remainder:
 *   (A x)_K = sum_f T'_f (x_K - x_L) + E_K x_K,
 * T' the eliminated face transmissibilities of orc_coefficients and
 * E_K = d_K + sum over faces to Dirichlet neighbours of T_KL (faces in the
 * order -x, +x, -y, +y, -z, +z), E = 1 on Dirichlet cells. */
void orc_extra_diagonal(const orc_grid* g, const double* K, const uint8_t* mask, const double* d,
                        double d0, double* E) {
  int64_t N = ncells(g);
  for (int64_t c = 0; c < N; ++c) {
    if (is_dir(mask, c)) { E[c] = 1.0; continue; }
    double s = dval(d, d0, c);
    for (int f = 0; f < 6; ++f) {
      int64_t n = neighbour(g, c, f);
      if (n < 0 || !is_dir(mask, n)) continue;
      s += face_T(g, K, c, f, n);
    }
    E[c] = s;
  }
}

/* Face transmissibilities of the +x/+y/+z face of every cell, without any
 * Dirichlet elimination (0 on the outer boundary). */
void orc_face_trans(const orc_grid* g, const double* K, double* Tx, double* Ty, double* Tz) {
  int64_t N = ncells(g);
  for (int64_t c = 0; c < N; ++c) {
    double* out[3] = {Tx, Ty, Tz};
    for (int axis = 0; axis < 3; ++axis) {
      int64_t n = neighbour(g, c, 2 * axis + 1);
      out[axis][c] = n < 0 ? 0.0 : face_T(g, K, c, 2 * axis + 1, n);
    }
  }
}

/* y = A x for the rows listed in idx (matrix-free evaluation of single rows,
 * for sampled checks on grids too large to assemble). */
void orc_apply_rows(const orc_grid* g, const double* K, const uint8_t* mask, const double* d,
                    double d0, const int64_t* idx, int64_t n, const double* x, double* y) {
  int64_t cols[7];
  double vals[7];
  for (int64_t t = 0; t < n; ++t) {
    int m = orc_row(g, K, mask, d, d0, idx[t], cols, vals);
    double s = 0.0;
    for (int e = 0; e < m; ++e) s += vals[e] * x[cols[e]];
    y[t] = s;
  }
}

/* |A| |x| for the rows listed in idx: the sum of |a_ij| |x_j| over row i, the
 * scale of the rounding error of any evaluation of (A x)_i. */
void orc_abs_apply_rows(const orc_grid* g, const double* K, const uint8_t* mask, const double* d,
                        double d0, const int64_t* idx, int64_t n, const double* x, double* y) {
  int64_t cols[7];
  double vals[7];
  for (int64_t t = 0; t < n; ++t) {
    int m = orc_row(g, K, mask, d, d0, idx[t], cols, vals);
    double s = 0.0;
    for (int e = 0; e < m; ++e) s += fabs(vals[e]) * fabs(x[cols[e]]);
    y[t] = s;
  }
}

/* Sum of T_KL (x_K - x_L) over all faces of each cell, ignoring the
 * Dirichlet set: the net flux leaving each cell for a pressure field x. */
void orc_net_flux(const orc_grid* g, const double* K, const double* x, double* y) {
  int64_t N = ncells(g);
  for (int64_t c = 0; c < N; ++c) {
    double s = 0.0;
    for (int f = 0; f < 6; ++f) {
      int64_t n = neighbour(g, c, f);
      if (n < 0) continue;
      s += face_T(g, K, c, f, n) * (x[c] - x[n]);
    }
    y[c] = s;
  }
}

void orc_spmv(int64_t N, const int64_t* rowptr, const int64_t* cols, const double* vals,
              const double* x, double* y) {
#pragma omp parallel for schedule(static) if (N >= PAR_MIN)
  for (int64_t r = 0; r < N; ++r) {
    double s = 0.0;
    for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) s += vals[e] * x[cols[e]];
    y[r] = s;
  }
}

/* sum of a[i] b[i]: each block of DOT_BLOCK terms is summed in index order,
 * then the block sums in block order */
static double dot(int64_t N, const double* a, const double* b) {
  int64_t nb = (N + DOT_BLOCK - 1) / DOT_BLOCK;
  if (nb <= 1) {
    double s = 0.0;
    for (int64_t i = 0; i < N; ++i) s += a[i] * b[i];
    return s;
  }
  double* part = (double*)malloc(sizeof(double) * (size_t)nb);
  if (part == NULL) {
    double s = 0.0;
    for (int64_t blk = 0; blk < nb; ++blk) {
      double t = 0.0;
      int64_t e = (blk + 1) * DOT_BLOCK < N ? (blk + 1) * DOT_BLOCK : N;
      for (int64_t i = blk * DOT_BLOCK; i < e; ++i) t += a[i] * b[i];
      s += t;
    }
    return s;
  }
#pragma omp parallel for schedule(static) if (nb >= PAR_MIN / DOT_BLOCK)
  for (int64_t blk = 0; blk < nb; ++blk) {
    double t = 0.0;
    int64_t e = (blk + 1) * DOT_BLOCK < N ? (blk + 1) * DOT_BLOCK : N;
    for (int64_t i = blk * DOT_BLOCK; i < e; ++i) t += a[i] * b[i];
    part[blk] = t;
  }
  double s = 0.0;
  for (int64_t blk = 0; blk < nb; ++blk) s += part[blk];
  free(part);
  return s;
}

/* Textbook conjugate gradient (Alg. 1; Hestenes-Stiefel):
 *   r0 = b - A x0, p0 = r0;  alpha = r'r / p'Ap;  x += alpha p;  r -= alpha Ap;
 *   beta = r+'r+ / r'r;  p = r+ + beta p.
 * Stops when ||r||_2 <= tol * ||b||_2 (recursive residual) or after maxit
 * iterations.  Returns 0 converged, 1 not converged, -4 breakdown (p'Ap <= 0).
 * If hist_x is not NULL, the iterate after iteration k is stored at
 * hist_x + k*N for k < hist_len. */
int orc_cg(int64_t N, const int64_t* rowptr, const int64_t* cols, const double* vals,
           const double* b, double* x, double tol, int64_t maxit, int64_t* iters, double* relres,
           double* hist_x, int64_t hist_len) {
  double* r = (double*)malloc(sizeof(double) * (size_t)N);
  double* p = (double*)malloc(sizeof(double) * (size_t)N);
  double* Ap = (double*)malloc(sizeof(double) * (size_t)N);
  if (!r || !p || !Ap) { free(r); free(p); free(Ap); return -2; }
  double bn = sqrt(dot(N, b, b));
  int status = 1;
  int64_t k = 0;
  if (bn == 0.0) {
    for (int64_t i = 0; i < N; ++i) x[i] = 0.0;
    *iters = 0; *relres = 0.0;
    free(r); free(p); free(Ap);
    return 0;
  }
  orc_spmv(N, rowptr, cols, vals, x, Ap);
#pragma omp parallel for schedule(static) if (N >= PAR_MIN)
  for (int64_t i = 0; i < N; ++i) { r[i] = b[i] - Ap[i]; p[i] = r[i]; }
  double rr = dot(N, r, r);
  for (k = 0; k < maxit; ++k) {
    if (sqrt(rr) <= tol * bn) { status = 0; break; }
    orc_spmv(N, rowptr, cols, vals, p, Ap);
    double pAp = dot(N, p, Ap);
    if (!(pAp > 0.0)) { status = -4; break; }
    double alpha = rr / pAp;
#pragma omp parallel for schedule(static) if (N >= PAR_MIN)
    for (int64_t i = 0; i < N; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * Ap[i]; }
    double rr_new = dot(N, r, r);
    double beta = rr_new / rr;
#pragma omp parallel for schedule(static) if (N >= PAR_MIN)
    for (int64_t i = 0; i < N; ++i) p[i] = r[i] + beta * p[i];
    rr = rr_new;
    if (hist_x != NULL && k < hist_len) memcpy(hist_x + k * N, x, sizeof(double) * (size_t)N);
  }
  if (status == 1 && sqrt(rr) <= tol * bn) status = 0;
  *iters = k;
  *relres = sqrt(rr) / bn;
  free(r); free(p); free(Ap);
  return status;
}

/* Conjugate gradient preconditioned with M = diag(A) (Jacobi), in the
 * textbook order:
 *   r0 = b - A x0, z0 = M^-1 r0, p0 = z0;
 *   alpha = r'z / p'Ap;  x += alpha p;  r -= alpha Ap;  z+ = M^-1 r+;
 *   beta = r+'z+ / r'z;  p = z+ + beta p.
 * Not part of the paper (Alg. 1 is unpreconditioned); the oracle uses it to
 * reach its FP64 reference solution on high-contrast fields, where plain CG
 * needs far more iterations.  M is read from the diagonal entries of the
 * CSR.  Stopping rule, return codes and history as orc_cg. */
int orc_pcg_jacobi(int64_t N, const int64_t* rowptr, const int64_t* cols, const double* vals,
                   const double* b, double* x, double tol, int64_t maxit, int64_t* iters,
                   double* relres, double* hist_x, int64_t hist_len) {
  double* r = (double*)malloc(sizeof(double) * (size_t)N);
  double* z = (double*)malloc(sizeof(double) * (size_t)N);
  double* p = (double*)malloc(sizeof(double) * (size_t)N);
  double* Ap = (double*)malloc(sizeof(double) * (size_t)N);
  double* minv = (double*)malloc(sizeof(double) * (size_t)N);
  if (!r || !z || !p || !Ap || !minv) {
    free(r); free(z); free(p); free(Ap); free(minv);
    return -2;
  }
  int status = 1;
  int64_t k = 0;
  for (int64_t i = 0; i < N; ++i) {
    double dg = 0.0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
      if (cols[e] == i) dg += vals[e];
    if (!(dg > 0.0)) status = -4;
    minv[i] = 1.0 / dg;
  }
  double bn = sqrt(dot(N, b, b));
  if (status == -4 || bn == 0.0) {
    if (bn == 0.0 && status != -4) {
      for (int64_t i = 0; i < N; ++i) x[i] = 0.0;
      status = 0;
    }
    *iters = 0; *relres = bn == 0.0 ? 0.0 : NAN;
    free(r); free(z); free(p); free(Ap); free(minv);
    return status;
  }
  orc_spmv(N, rowptr, cols, vals, x, Ap);
#pragma omp parallel for schedule(static) if (N >= PAR_MIN)
  for (int64_t i = 0; i < N; ++i) { r[i] = b[i] - Ap[i]; z[i] = minv[i] * r[i]; p[i] = z[i]; }
  double rz = dot(N, r, z);
  double rr = dot(N, r, r);
  for (k = 0; k < maxit; ++k) {
    if (sqrt(rr) <= tol * bn) { status = 0; break; }
    orc_spmv(N, rowptr, cols, vals, p, Ap);
    double pAp = dot(N, p, Ap);
    if (!(pAp > 0.0)) { status = -4; break; }
    double alpha = rz / pAp;
#pragma omp parallel for schedule(static) if (N >= PAR_MIN)
    for (int64_t i = 0; i < N; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * Ap[i];
      z[i] = minv[i] * r[i];
    }
    double rz_new = dot(N, r, z);
    rr = dot(N, r, r);
    double beta = rz_new / rz;
#pragma omp parallel for schedule(static) if (N >= PAR_MIN)
    for (int64_t i = 0; i < N; ++i) p[i] = z[i] + beta * p[i];
    rz = rz_new;
    if (hist_x != NULL && k < hist_len) memcpy(hist_x + k * N, x, sizeof(double) * (size_t)N);
  }
  if (status == 1 && sqrt(rr) <= tol * bn) status = 0;
  *iters = k;
  *relres = sqrt(rr) / bn;
  free(r); free(z); free(p); free(Ap); free(minv);
  return status;
}

/* Dense Cholesky factorisation and solve of an SPD n x n row-major matrix
 * (A = L L^T, Cholesky-Banachiewicz), for tiny grids.  A is overwritten by
 * L.  Returns 0, or -4 if a pivot is not positive. */
int orc_cholesky_solve(int64_t n, double* A, const double* b, double* x) {
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = 0; j <= i; ++j) {
      double s = A[i * n + j];
      for (int64_t k = 0; k < j; ++k) s -= A[i * n + k] * A[j * n + k];
      if (i == j) {
        if (!(s > 0.0)) return -4;
        A[i * n + i] = sqrt(s);
      } else {
        A[i * n + j] = s / A[j * n + j];
      }
    }
  }
  for (int64_t i = 0; i < n; ++i) {  /* L y = b */
    double s = b[i];
    for (int64_t k = 0; k < i; ++k) s -= A[i * n + k] * x[k];
    x[i] = s / A[i * n + i];
  }
  for (int64_t i = n - 1; i >= 0; --i) {  /* L^T x = y */
    double s = x[i];
    for (int64_t k = i + 1; k < n; ++k) s -= A[k * n + i] * x[k];
    x[i] = s / A[i * n + i];
  }
  return 0;
}
