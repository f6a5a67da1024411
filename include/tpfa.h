/*
 * tpfa.h -- C ABI of the GB300 (sm_103a) matrix-free TPFA pressure solver.
 *
 * Problem (arXiv 2408.03452, "Matrix-Free Finite Volume Kernels on a
 * Dataflow Architecture", Section II.A): single-phase incompressible Darcy
 * flow (Eq. 1a-1b) discretised with two-point flux approximation (Eq. 4) on a
 * structured nx x ny x nz Cartesian grid, giving the linear system
 *
 *     (A p)_K = sum_{L in adj(K)} T_KL (p_K - p_L) + d_K p_K = b_K   (K not in T^D)
 *     p_K = p^D_K                                                  (K in T^D)
 *
 * solved matrix-free (Eq. 6, Alg. 2) by conjugate gradient (Alg. 1).
 *
 * Layout of every per-cell array: flat index c = i + nx*(j + ny*k), X
 * innermost and Z outermost (Section IV).  N = nx*ny*nz.
 *
 * Coefficient record ("coef"): 4 values per cell, cell-interleaved,
 *     coef[4c+0] = Tx  transmissibility of the face between c and c+1 (x)
 *     coef[4c+1] = Ty  ... between c and c+nx (y)
 *     coef[4c+2] = Tz  ... between c and c+nx*ny (z)
 *     coef[4c+3] = D   diagonal: sum of the six face transmissibilities + d_c
 * A face on the outer boundary has T = 0 (no-flow).  A face touching a
 * Dirichlet cell has T = 0 (its coupling is moved to the right-hand side),
 * and a Dirichlet cell has D = 1, so the stored operator is the symmetric
 * positive definite elimination of Eq. 6's constrained rows.
 *
 * Conventions for every entry point:
 *  - Pointers marked "dev" are CUDA device pointers (or managed memory) on
 *    the current device; the caller allocates and owns them.  Pointers marked
 *    "host" are host memory.  A context owns only its internal workspace.
 *  - "stream" is a cudaStream_t (NULL = the legacy default stream).  Calls
 *    enqueue work on it and return without waiting, except cg_solve, which
 *    waits for its stream (it drives the refinement loop and fills *info).
 *  - Return value: TPFA_OK (0) on success, a negative TPFA_E* code on error,
 *    TPFA_NOTCONV (+1) when cg_solve stops at maxit.  On error nothing was
 *    enqueued unless the code is TPFA_ECUDA.
 *  - A context is not thread-safe: calls on one context must not overlap
 *    (same host thread or externally serialised, one stream at a time).
 */
#ifndef TPFA_H
#define TPFA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TPFA_ABI_VERSION 1

enum tpfa_status {
  TPFA_OK = 0,
  TPFA_NOTCONV = 1,        /* maxit reached; x holds the last iterate          */
  TPFA_EINVAL = -1,        /* bad size, NULL or misaligned pointer, bad option  */
  TPFA_ENOMEM = -2,        /* device allocation of the workspace failed         */
  TPFA_ECUDA = -3,         /* a CUDA runtime call failed                        */
  TPFA_EBREAKDOWN = -4,    /* CG breakdown: p'Ap <= 0 (operator not SPD)        */
  TPFA_ENONFINITE = -5,    /* NaN or Inf met in a reduction                     */
  TPFA_EINTERNAL = -6,     /* iteration guard tripped (should not happen)       */
  TPFA_ESTAGNATION = -7    /* refinement stopped reducing the FP64 residual     */
};

/* Grid: nx, ny, nz >= 1 cells of size dx, dy, dz > 0; viscosity mu > 0;
 * nx*ny + 2*nx < 2^31 (one z-plane is addressed with 32-bit offsets). */
typedef struct {
  int64_t nx, ny, nz;
  double dx, dy, dz, mu;
} tpfa_grid;

/* Result of cg_solve (host struct filled by the call). */
typedef struct {
  int64_t iters;          /* CG iterations (operator applications) in total       */
  int32_t outer;          /* FP64 refinement corrections applied                  */
  int32_t status;         /* same as the return code                              */
  double rel_res_inner;   /* last inner recursive residual, relative to its rhs   */
  double rel_res_fp64;    /* ||b - A x||_2 / ||b||_2 at exit, in FP64 with coef64 */
  double inner_ms;        /* GPU time inside the CG iteration loops (CUDA events) */
  double total_ms;        /* GPU time of the whole call (CUDA events)             */
  int64_t kernel_launches; /* kernels this call ran (sweeps counted on the device) */
} tpfa_cg_info;

typedef struct tpfa_ctx tpfa_ctx;

/* Options for tpfa_set_option. */
enum tpfa_option {
  TPFA_OPT_INNER_RTOL = 1,   /* lower bound on the inner FP32 CG relative tolerance (default 1e-6) */
  TPFA_OPT_MAX_OUTER = 2,    /* maximum FP64 refinement steps (default 20)                        */
  TPFA_OPT_LOOP = 3,         /* 0 = CUDA-graph while node (default), 1 = host-polled graph chunks */
  TPFA_OPT_TILE_VY = 4,      /* rows per warp in the stencil sweeps: 4 or 8 (default 4; 8 sets 3 stages) */
  TPFA_OPT_TILE_ZC = 5,      /* planes per warp in the stencil sweeps, 0 = automatic              */
  TPFA_OPT_CHUNK = 6,        /* CG iterations per graph launch when TPFA_OPT_LOOP = 1 (default 32) */
  TPFA_OPT_STAGES = 7,       /* shared-memory plane stages per warp: 3 or 4 (default 4; 4 needs VY = 4) */
  /* 8, 9, 10: retired (a CG sweep that recomputed q = A p at 40 B/cell was
     measured slower than the stored-q sweep); tpfa_set_option refuses them */
  TPFA_OPT_INNER_RTOL_BF16 = 11, /* lower bound on the inner relative tolerance of cg_solve_bf16 (1e-3) */
  TPFA_OPT_PRECOND = 12,     /* inner CG of cg_solve and cg_solve_bf16: 0 = unpreconditioned
                                (Alg. 1, default), 1 = Jacobi, M = diag(D) (with BF16 records D
                                is the diagonal the BF16 sweep forms; cg_solve_bf16 then
                                allocates one FP32 vector of M^-1 on its first call)            */
  TPFA_OPT_FCG_M = 13,       /* fcg_solve: previous directions each new one is A-orthogonalised
                                against, 1..16 (default 4)                                        */
  TPFA_OPT_FCG_FALLBACK = 14, /* fcg_solve with a network, after breakdown or stagnation:
                                0 = unpreconditioned CG (default); 1 = drop the network, keep
                                Jacobi                                                            */
  TPFA_OPT_SWEEP = 15,       /* CG sweep kernel of cg_solve: 0 = automatic (default: the TMA-staged
                                sweep for unpreconditioned CG on FP32 records, else the
                                cp.async-staged sweep), 1 = cp.async-staged sweep, 2 = TMA-staged
                                sweep (cg_solve returns TPFA_EINVAL where it cannot run: BF16
                                records, Jacobi, or a driver without the tensor-map encoder).
                                The TMA-staged sweep keeps r, q, p, x of a cell in one 16-byte
                                record (32 B/cell of context memory, allocated on first use).
                                tpfa_apply and tpfa_apply_bf16 follow it: TMA-staged unless 1,
                                when nx % 4 == 0 and coef and p are 16-byte aligned, else
                                cp.async-staged (same values either way)                         */
  TPFA_OPT_TMA_TILE = 16     /* tile of the TMA-staged sweep, 32 columns x rows per block:
                                0 = 4 warps x 4 rows, 4 stages (default); 1 = 4 x 4, 3 stages;
                                2 = 8 x 4, 3 stages; 3 = 4 x 2, 6 stages                         */
};

/* The stencil-sweep tiling a context uses, for inspection and tests.
 * which: 0 = the CG loop of cg_solve with FP32 records, 1 = the CG loop of
 * cg_solve_bf16, 2 = tpfa_apply, 3 = tpfa_apply_bf16 (for 16-byte aligned
 * arguments).  out: host array of 6 values:
 * kernel (1 = cp.async-staged sweep, 2 = TMA-staged sweep), rows per warp,
 * shared-memory stages, compute warps per block, z-planes per run (zc),
 * blocks per launch.  Returns TPFA_EINVAL for a NULL argument, a bad `which`
 * or a requested TMA sweep that cannot run for this grid. */
int tpfa_sweep_tiling(const tpfa_ctx* ctx, int which, int64_t* out);

/* Create a context for one grid on the current CUDA device.  Allocates the
 * small reduction workspace (partials, scalars); the CG vectors are
 * allocated by the first cg_solve.  *out receives the handle. */
int tpfa_create(const tpfa_grid* grid, tpfa_ctx** out);

/* Free the context and everything it allocated (synchronises the device). */
int tpfa_destroy(tpfa_ctx* ctx);

/* Human-readable text for a status code (static storage). */
const char* tpfa_strerror(int code);

/* TPFA_ABI_VERSION of the loaded library. */
int tpfa_abi_version(void);

/* Set a solver option (see enum tpfa_option); TPFA_EINVAL if out of range. */
int tpfa_set_option(tpfa_ctx* ctx, int option, double value);

/*
 * Transmissibilities and diagonal (Section II.A, Eq. 4 and Eq. 6).
 *   T_KL = (A_f / mu) / (h/(2 k_K) + h/(2 k_L)),  A_f the face area, h the
 *   cell size normal to the face; lambda_KL = 1/mu (arithmetic mean of the
 *   two equal mobilities).  Computed in FP64 and rounded to nearest FP32.
 *   D_K = T(-x)+T(+x)+T(-y)+T(+y)+T(-z)+T(+z) + d_K summed in that order
 *   in FP64 over the faces that exist (faces to Dirichlet cells included),
 *   then rounded; D = 1 on Dirichlet cells.
 * K         dev, N doubles, permeability > 0.
 * dirichlet dev, N bytes (nonzero = cell in T^D) or NULL (no Dirichlet cells).
 * d         dev, N doubles, accumulation diagonal d_K >= 0, or NULL: every
 *           cell uses d_uniform.
 * coef      dev, 4N floats, 16-byte aligned: output coefficient records.
 * coef64    dev, 4N doubles, 16-byte aligned: the same in FP64 (needed by
 *           cg_solve's FP64 residual), or NULL.
 */
int tpfa_build_trans(tpfa_ctx* ctx, const double* K, const uint8_t* dirichlet, const double* d,
                     double d_uniform, float* coef, double* coef64, void* stream);

/*
 * Right-hand side (Section II.A, Eq. 3 with sources).
 *   b_K = p^D_K                                    for K in T^D,
 *   b_K = q_K + sum_{L in adj(K), L in T^D} T_KL p^D_L   otherwise
 *   (lifted couplings summed in FP64 in the face order -x,+x,-y,+y,-z,+z).
 * q         dev, N doubles (dense source term) or NULL.
 * pD        dev, N doubles, Dirichlet values (read on T^D only), or NULL = 0.
 * src_idx   dev, n_src int64 cell indices, src_val dev, n_src doubles: point
 *           sources added to q (duplicates add up); both NULL when n_src = 0.
 *           Indices outside [0, N) are ignored.
 * b         dev, N doubles, output.
 */
int tpfa_build_rhs(tpfa_ctx* ctx, const double* K, const uint8_t* dirichlet, const double* q,
                   const double* pD, const int64_t* src_idx, const double* src_val, int64_t n_src,
                   double* b, void* stream);

/*
 * Right-hand side of one backward-Euler time step of the slightly
 * compressible problem (Section II.A: implicit time discretisation; the
 * accumulation diagonal d = c V / dt is the one given to tpfa_build_trans):
 *   b = (tpfa_build_rhs) + d_K p_prev_K   on interior cells,
 * so that solving A p = b gives p^{n+1} from p^n = p_prev.  d / d_uniform:
 * as for tpfa_build_trans.  p_prev: dev, N doubles (must not alias b).
 */
int tpfa_build_rhs_transient(tpfa_ctx* ctx, const double* K, const uint8_t* dirichlet,
                             const double* q, const double* pD, const int64_t* src_idx,
                             const double* src_val, int64_t n_src, const double* d,
                             double d_uniform, const double* p_prev, double* b, void* stream);

/*
 * Matrix-free operator application (Eq. 6, Alg. 2) in FP32:
 *   Ap_K = D_K p_K - Tx_K p_{K+x} - Tx_{K-x} p_{K-x} - Ty_K p_{K+y}
 *          - Ty_{K-y} p_{K-y} - Tz_K p_{K+z} - Tz_{K-z} p_{K-z}
 * evaluated with fused multiply-adds in that order.
 * coef dev 4N floats (16-byte aligned); p dev N floats; Ap dev N floats
 * (must not alias p).  pAp: dev pointer to one double receiving p.Ap
 * (FP32 products, compensated FP32 partial sums, FP64 across warps and
 * blocks in a fixed order: bit-reproducible run to run), or NULL.
 * Kernel: TMA-staged when nx % 4 == 0 and p is 16-byte aligned (unless
 * TPFA_OPT_SWEEP = 1 or TPFA_OPT_TILE_VY != 4), else cp.async-staged; both
 * give identical Ap (pAp may differ in the last bits: another grouping).  In
 * the TMA-staged kernel every wait for a copy is bounded; a copy that never
 * lands (not expected on working hardware) leaves NaN in the cells it held
 * up and in pAp instead of hanging the GPU.
 */
int tpfa_apply(tpfa_ctx* ctx, const float* coef, const float* p, float* Ap, double* pAp,
               void* stream);

/*
 * FP64 residual r = b - A x with the FP64 coefficient records (final check
 * of the solve).  coef64 dev 4N doubles (16-byte aligned); b, x dev N
 * doubles; r dev N doubles (may alias neither b nor x).  norms: dev pointer
 * to two doubles receiving ||r||_2^2 and ||b||_2^2 (fixed-order FP64
 * reductions), or NULL.
 */
int tpfa_residual64(tpfa_ctx* ctx, const double* coef64, const double* b, const double* x,
                    double* r, double* norms, void* stream);

/*
 * Solve A x = b (Alg. 1) to ||b - A x||_2 <= tol ||b||_2 measured in FP64.
 * Inner solver: unpreconditioned CG in FP32 on coef, one fused sweep per
 * iteration (operator, both vector updates and the single reduction), run
 * inside a CUDA graph whose while-loop condition is set on the device.
 * Outer loop: FP64 residual with coef64, FP32 correction solve, FP64 update
 * (iterative refinement) until tol is met.
 * coef    dev 4N floats; coef64 dev 4N doubles (both from tpfa_build_trans).
 * b       dev N doubles.
 * x       dev N doubles: initial guess on entry, solution on exit.
 * tol     > 0; maxit >= 1 bounds the total number of CG iterations.
 * info    host, filled on return (may be NULL).
 * Returns TPFA_OK, TPFA_NOTCONV, or an error.  Waits for the stream.
 */
int cg_solve(tpfa_ctx* ctx, const float* coef, const double* coef64, const double* b, double* x,
             double tol, int64_t maxit, tpfa_cg_info* info, void* stream);

/*
 * Mixed precision (BF16 coefficients, FP32 inner CG, FP64 refinement).
 *
 * BF16 record ("coef16"): 4 bf16 values per cell, cell-interleaved, 8 bytes:
 *     coef16[4c+0..2] = Tx', Ty', Tz'  eliminated face transmissibilities as in
 *                                      the FP32 record, rounded to nearest-even
 *     coef16[4c+3]    = E   d_K + sum of T_KL over faces to Dirichlet
 *                           neighbours (1 on Dirichlet cells)
 * The diagonal is not stored: the sweep forms D = T'(-x) + T'(+x) + T'(-y) +
 * T'(+y) + T'(-z) + T'(+z) + E in FP32 from the six face values it reads
 * anyway.  The BF16 operator is therefore the TPFA operator of the rounded
 * face values: symmetric positive definite like the FP64 one, with x'Ax
 * within a factor 1 +- 2^-9 of it, so iterative refinement against the
 * FP64 residual contracts the error by about 2^-9 per step.
 */

/* BF16 records (Eq. 4 as tpfa_build_trans, then rounded).  coef16: dev, 4N
 * uint16 (bf16 bit patterns), 8-byte aligned.  Other arguments as for
 * tpfa_build_trans. */
int tpfa_build_trans_bf16(tpfa_ctx* ctx, const double* K, const uint8_t* dirichlet,
                          const double* d, double d_uniform, uint16_t* coef16, void* stream);

/* tpfa_apply with BF16 records (Eq. 6 / Alg. 2, FP32 arithmetic on the
 * exactly widened BF16 values; D formed as stated above). */
int tpfa_apply_bf16(tpfa_ctx* ctx, const uint16_t* coef16, const float* p, float* Ap,
                    double* pAp, void* stream);

/* cg_solve with the BF16 operator inside the FP32 CG sweeps: each refinement
 * step solves A_bf16 e = r (relative tolerance max(tol/2 / current relative
 * residual, TPFA_OPT_INNER_RTOL_BF16)), then x += e and r = b - A x in FP64
 * with coef64.  Stops when the FP64 relative residual <= tol.  With
 * TPFA_OPT_PRECOND = 1 the inner CG is Jacobi-preconditioned: M^-1 = 1/D per
 * cell, D formed from the BF16 faces and E exactly as the sweep forms it,
 * computed into a context vector at the start of each call (the sweep then
 * reads 8 + 4 bytes of coefficients per cell instead of 16).  Arguments and
 * return codes as cg_solve. */
int cg_solve_bf16(tpfa_ctx* ctx, const uint16_t* coef16, const double* coef64, const double* b,
                  double* x, double tol, int64_t maxit, tpfa_cg_info* info, void* stream);

/*
 * Batched ensembles: n_inst independent problems (each its own grid, K,
 * boundary set and tolerance target) solved together.  Every per-cell array
 * of a batch is the concatenation of the instances' arrays: instance i
 * occupies cells offsets[i] .. offsets[i+1]-1 (tpfa_batch_offsets), X
 * innermost inside the instance.  The CG iterations of all instances run as
 * one sweep launch per iteration inside one CUDA-graph while loop; each
 * instance has its own scalars and convergence flag, and the blocks of a
 * converged instance return immediately.
 */
typedef struct tpfa_batch tpfa_batch;

/* grids: host array of n_inst grids (rules of tpfa_create each).  zc: host
 * array of n_inst z-run lengths for the sweep tiling (0 = automatic), or NULL
 * (all automatic); an autotuner may supply them. */
int tpfa_batch_create(const tpfa_grid* grids, int n_inst, const int* zc, tpfa_batch** out);
int tpfa_batch_destroy(tpfa_batch* batch);
/* offsets: host, n_inst + 1 entries (cell offsets, last = total cells). */
int tpfa_batch_offsets(const tpfa_batch* batch, int64_t* offsets);
/* zc: host, n_inst entries: the z-run length each instance uses. */
int tpfa_batch_zc(const tpfa_batch* batch, int* zc);
/* TPFA_OPT_INNER_RTOL, TPFA_OPT_MAX_OUTER, TPFA_OPT_PRECOND; for fcg_solve_batch
 * also TPFA_OPT_FCG_M and TPFA_OPT_FCG_FALLBACK. */
int tpfa_batch_set_option(tpfa_batch* batch, int option, double value);
/* As tpfa_build_trans / tpfa_build_rhs over the concatenated arrays. */
int tpfa_batch_build_trans(tpfa_batch* batch, const double* K, const uint8_t* dirichlet,
                           const double* d, double d_uniform, float* coef, double* coef64,
                           void* stream);
int tpfa_batch_build_rhs(tpfa_batch* batch, const double* K, const uint8_t* dirichlet,
                         const double* q, const double* pD, double* b, void* stream);
/* Solve every instance to ||b_i - A_i x_i|| <= tol ||b_i|| (FP64), refined
 * as cg_solve.  infos: host, n_inst entries (per-instance results; the
 * timing fields are the whole call's), or NULL.  total: host summary
 * (iterations summed over instances, largest relative residual), or NULL.
 * Returns TPFA_OK if every instance converged, else the most severe status
 * (errors before TPFA_NOTCONV).  Waits for the stream. */
int cg_solve_batch(tpfa_batch* batch, const float* coef, const double* coef64, const double* b,
                   double* x, double tol, int64_t maxit, tpfa_cg_info* infos,
                   tpfa_cg_info* total, void* stream);

/*
 * Tensor-core GEMM tile (tcgen05, BF16 inputs, FP32 accumulation in tensor
 * memory): C[M x N] = A[M x K] * B[K x N], with A row-major (K contiguous),
 * B passed as its transpose Bt[N x K] (K contiguous), C row-major FP32; all
 * dev, 16-byte aligned.  1 <= M, K a multiple of 16 up to 256, N in
 * {16, 32, 64, 128}.  The building block of the learned preconditioner's
 * implicit-GEMM convolutions, exposed so that it can be checked on its own.
 * Waits for the stream; TPFA_EINTERNAL if the tensor core did not complete.
 */
int tpfa_tc_gemm_bf16(const uint16_t* A, const uint16_t* Bt, float* C, int M, int N, int K,
                      void* stream);

/*
 * Learned preconditioner: 3x3x3 convolutions (the layers of a 3D U-Net,
 * Ronneberger et al. 2015) on the tensor cores.  Not part of the paper's
 * method, which runs CG unpreconditioned; the preconditioner only changes how
 * fast the same system converges.
 *
 * Volumes use the haloed channels-last BF16 layout: ns samples of
 * nz x ny x nx cells, each padded with a one-cell zero halo, channels
 * innermost; element (s, z, y, x, c) sits at
 *   ((((s*(nz+2) + z+1)*(ny+2) + y+1)*(nx+2) + x+1)*C + c,
 * V = (nx+2)(ny+2)(nz+2) ns voxels.  The caller zeroes a volume once; these
 * calls never write its halo, which is what makes the convolution zero-padded
 * and keeps samples apart.  Weights w[27][cout][ci] with tap
 * t = 9(dz+1) + 3(dy+1) + (dx+1):
 *   y[v][co] = bias[co] + sum_t sum_ci x[v + off_t][ci] w[t][co][ci].
 * Supported (cin, cout): (16,16) (16,32) (32,16) (32,64) (64,32).
 * All pointers dev, 16-byte aligned; V*(nx+2)-sized indices must fit in int.
 * Asynchronous on the stream: a tensor-core wait that gives up is reported by
 * the next tpfa_net_status.
 */
#define TPFA_CONV_RELU 1 /* y = max(y, 0) */
#define TPFA_CONV_MASK 2 /* y = 0 where mask[v][co] <= 0 (ReLU derivative) */
/* y [V][cout] = flags-epilogue(conv(x [V][cin]; w) + bias); bias may be NULL;
 * mask [V][cout] read only with TPFA_CONV_MASK.  x and y must not overlap.
 * The input gradient of a layer is this call with the taps flipped and each
 * tap's matrix transposed (w'[t][ci][co] = w[26-t][co][ci]). */
int tpfa_conv3d_bf16(const uint16_t* x, const uint16_t* w, const float* bias,
                     const uint16_t* mask, uint16_t* y, int nx, int ny, int nz, int ns, int cin,
                     int cout, int flags, void* stream);
/* Weight gradient: dw[t][co][ci] (+)= sum_v dy[v][co] x[v + off_t][ci] over all
 * voxels, FP32 (accumulate != 0 adds to dw).  Allocates a stream-ordered
 * workspace. */
int tpfa_conv3d_wgrad_bf16(const uint16_t* x, const uint16_t* dy, float* dw, int nx, int ny,
                           int nz, int ns, int cin, int cout, int accumulate, void* stream);
/* Forward-convolution kernel for the calls that follow (process-wide):
 * 0 = 128-voxel tiles, each copying the nine row groups it reads;
 * 1 = z-marching: each CTA follows a 128-voxel plane segment through
 *     consecutive planes with a ring of row-group triples, loading each
 *     triple once, 27 MMAs of N = cout per output plane into two alternating
 *     TMEM accumulators;
 * 2 = z-marching with the z-taps folded into N: the loop runs over input
 *     planes, and one MMA of N = 3 cout applies the three z-taps of one
 *     (dy, dx) offset to the three output planes an input plane feeds
 *     (accumulators in a TMEM ring), so every staged input row is read by the
 *     tensor core 9 instead of 27 times;
 * 4 = kernel 2 with warp-specialised roles: a copy warp fills the ring of
 *     triples, one thread issues the MMAs, four epilogue warps drain a ring
 *     of TMEM accumulators, joined by mbarriers instead of block barriers;
 * 3 = per layer shape, the fastest on GB300 (default): 1 for 32 -> 16, 4 for
 *     the others.
 * (cin, cout) = (64, 32) always uses kernel 0.  Returns TPFA_EINVAL for
 * another value. */
int tpfa_conv3d_select(int kernel);
/* Waits for the stream; TPFA_EINTERNAL (and clears the flag) if any
 * tensor-core wait of the convolution kernels gave up since the last call. */
int tpfa_net_status(void* stream);
/* Test hook for that failure path: one block waits, with the same bounded
 * wait the tensor-core kernels use, on an mbarrier phase that nothing
 * completes, gives up after `polls` polls (1 <= polls <= 2^22) and records
 * the timeout as a stalled tensor-core kernel would; the next
 * tpfa_net_status returns TPFA_EINTERNAL and clears it.  Allocates no
 * tensor memory; the context stays usable.  Asynchronous. */
int tpfa_tc_wait_probe(uint32_t polls, void* stream);

/*
 * The 3-level U-Net preconditioner M(r) = rms(r) * net(r / rms(r), ln K):
 *   e0 = relu(conv(in; W0 2->16))          level 0 (full resolution)
 *   e1 = relu(conv(pool(e0); W1 16->32))   level 1 (half, 2x2x2 average pool)
 *   e2 = relu(conv(pool(e1); W2 32->64))   level 2 (quarter)
 *   d2 = relu(conv(e2; W3 64->32))         level 2
 *   s1 = up(d2) + e1                       level 1 (nearest upsampling)
 *   d1 = relu(conv(s1; W4 32->16))         level 1
 *   s0 = up(d1) + e0                       level 0
 *   d0 = relu(conv(s0; W5 16->16))         level 0
 *   z  = conv(d0; W6 16->1)                level 0
 * rms(r) = sqrt(mean of r^2) per sample.  Parameters: one FP32 vector of
 * tpfa_unet_param_count() values, layer by layer W_i[27][cout][cin] then
 * b_i[cout].  Vectors r, ln K, z, gz: FP32, ns samples of nx*ny*nz cells
 * each in the solver's x-fastest order, sample after sample.
 */
typedef struct tpfa_unet tpfa_unet;
int64_t tpfa_unet_param_count(void);
/* nx, ny, nz multiples of 4 (two poolings); ns samples per call; train != 0
 * also allocates what tpfa_unet_backward needs.  Uses the current device. */
int tpfa_unet_create(int nx, int ny, int nz, int ns, int train, tpfa_unet** out);
int tpfa_unet_destroy(tpfa_unet* net);
/* dims4 (host) = {nx, ny, nz, ns} */
int tpfa_unet_shape(const tpfa_unet* net, int* dims4);
/* Converts the FP32 parameters (dev) to the BF16 copies the kernels use
 * (forward layout, and tap-flipped transposed layout for the input gradients). */
int tpfa_unet_set_params(tpfa_unet* net, const float* params, void* stream);
/* z = M(r) for every sample (dev pointers).  Keeps the activations for a
 * following tpfa_unet_backward.  Asynchronous. */
int tpfa_unet_forward(tpfa_unet* net, const float* r, const float* lnk, float* z, void* stream);
/* tpfa_unet_forward on the first ns samples only (1 <= ns <= the network's
 * sample count): r, lnk, z hold ns samples.  Each sample's output is the
 * same as in a full forward pass.  After a pass on fewer samples than the
 * network has, tpfa_unet_backward returns TPFA_EINVAL until the next full
 * forward pass.  Asynchronous. */
int tpfa_unet_forward_samples(tpfa_unet* net, int ns, const float* r, const float* lnk, float* z,
                              void* stream);
/* The network's permeability input: lnk[i] = ln K[i] rounded to FP32, for
 * n cells (K dev FP64 > 0, lnk dev FP32; the current device).  Asynchronous. */
int tpfa_log_perm(const double* K, float* lnk, int64_t n, void* stream);
/* grad (dev, param_count FP32, overwritten) = d(sum gz . z)/d(params) at the
 * last forward pass; gz dev.  Requires train.  Asynchronous. */
int tpfa_unet_backward(tpfa_unet* net, const float* gz, float* grad, void* stream);
/* One Adam step (Kingma and Ba 2015, Algorithm 1), t >= 1 the step number:
 * m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 * p -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).  All dev FP32, n values. */
int tpfa_adam_step(float* params, const float* grad, float* m, float* v, int64_t n, int t,
                   double lr, double b1, double b2, double eps, void* stream);
/* Gradient of the training loss for one sample on the context's grid: the
 * A-norm error of the best multiple of mr,
 *   L = min_c (c mr - e)' A (c mr - e) / (e' A e)
 *     = 1 - a^2 / (b eae),  a = mr' r,  b = mr' A mr,  A e = r,
 * (CG is invariant to the scale of its preconditioner's output).  Writes
 * q = A mr, stats (dev, two doubles) = (a, b) and
 * g = dL/dmr = (2 a / (b eae)) ((a / b) q - r).  coef: the sample's FP32
 * coefficient records; mr, r, q, g dev N floats, pairwise distinct; eae dev
 * double = e' A e.  Asynchronous (stream-ordered workspace). */
int tpfa_anorm_loss_grad(tpfa_ctx* ctx, const float* coef, const float* mr, const float* r,
                         const double* eae, float* q, float* g, double* stats, void* stream);
/* Flexible CG (Notay 2000) with m = TPFA_OPT_FCG_M retained directions,
 * refined in FP64 as cg_solve: outer r = b - A64 x, inner FP32 FCG on
 * A e = r / ||r|| to max(TPFA_OPT_INNER_RTOL, 0.3 tol / (||r||/||b||)),
 * x += e ||r||.  Inner step: z = M(r); p = z - sum_j (z'q_j / p_j'q_j) p_j over
 * the last m directions; q = A p; alpha = p'r / p'q; e += alpha p; r -= alpha q.
 * Preconditioner: net == NULL gives the identity (plain CG); otherwise the
 * Jacobi blend z = D^-1 r + c u with the A-norm-optimal weight
 * c = (u'r - (Au)'D^-1 r) / (u'Au) (one extra operator application), where
 * u = net(r, ln K) if net was created for this grid, or u = P^l net(R^l r, R^l ln K)
 * if it was created for the 2^l coarser grid, l = 1, 2 or 3 (R: mean of each
 * 2x2x2 block, P: nearest prolongation; grid extents divisible by 2^l).  When p'Ap <= 0, a value is
 * not finite, or the smallest r'r of the last 100 iterations is not 1% below
 * the smallest before them, the inner iteration drops the network
 * (TPFA_OPT_FCG_FALLBACK: plain CG by default) and restarts its directions
 * from the current iterate (*fell_back = 1; may be NULL).  net: ns = 1; lnk
 * dev N floats (ignored without net).  coef, coef64, b, x as cg_solve.  Waits
 * for the stream.  Returns TPFA_OK, TPFA_NOTCONV (maxit inner iterations or
 * TPFA_OPT_MAX_OUTER refinements), TPFA_EBREAKDOWN, TPFA_ENONFINITE,
 * TPFA_EINTERNAL (a tensor-core wait gave up) or an argument / CUDA error. */
/* Training target of the network inside the Jacobi blend, for one sample:
 * s = r - A D^-1 r (= A w, w = e - D^-1 r the error left by one Jacobi step)
 * and, when e and wAw are both given, wAw = w' A w.  Pass s as the r argument
 * of tpfa_anorm_loss_grad; the blended loss is (wAw - a^2 / b) / (e' A e).
 * r, e, s dev N floats (s distinct from r and e); wAw dev double.
 * Asynchronous (stream-ordered workspace). */
int tpfa_jacobi_split(tpfa_ctx* ctx, const float* coef, const float* r, const float* e, float* s,
                      double* wAw, void* stream);
/* Restriction to the 2x coarser grid: coarse = scale * (sum of the 8
 * children) (scale 1/8: block mean; scale 1: adjoint of tpfa_prolong2).
 * fine: ns samples of nx x ny x nz (all even) FP32 in the solver's order, dev,
 * 8-byte aligned; coarse: ns (nx/2)(ny/2)(nz/2) FP32, dev.  Asynchronous. */
int tpfa_restrict2(const float* fine, float* coarse, int nx, int ny, int nz, int ns, float scale,
                   void* stream);
/* Nearest prolongation: fine[c] = coarse[parent(c)] (shapes as tpfa_restrict2;
 * fine 8-byte aligned).  Asynchronous. */
int tpfa_prolong2(const float* coarse, float* fine, int nx, int ny, int nz, int ns, void* stream);
/* The 2^levels coarser grid in one pass (levels 1 to 3; extents divisible by
 * 2^levels): coarse = the mean over each 2^levels block, bit-identical to
 * `levels` successive tpfa_restrict2 calls with scale 1/8 (the same sums in
 * the same order).  fine 8-byte aligned; shapes as tpfa_restrict2 with
 * coarse ns (nx/2^l)(ny/2^l)(nz/2^l).  The solvers restrict to and prolong
 * from a network's coarser grid with these passes.  Asynchronous. */
int tpfa_restrict_levels(const float* fine, float* coarse, int nx, int ny, int nz, int ns,
                         int levels, void* stream);
/* fine[c] = coarse value of c's ancestor on the 2^levels coarser grid
 * (`levels` nearest prolongations in one pass).  fine 8-byte aligned.
 * Asynchronous. */
int tpfa_prolong_levels(const float* coarse, float* fine, int nx, int ny, int nz, int ns,
                        int levels, void* stream);
int fcg_solve(tpfa_ctx* ctx, tpfa_unet* net, const float* coef, const double* coef64,
              const float* lnk, const double* b, double* x, double tol, int64_t maxit,
              tpfa_cg_info* info, int* fell_back, void* stream);

/* fcg_solve over the instances of a batch (the learned-preconditioned,
 * mixed-precision, batched form): every instance is refined and iterated as
 * fcg_solve would do it alone, with its own tolerance target, iteration
 * limit, preconditioner mode, fallback and convergence flag, but each FCG
 * step is one launch per vector pass over all instances that still iterate
 * (per-instance partial sums in a fixed order, so an instance's iterates do
 * not depend on the others), and the batched operator application skips
 * finished instances.  The inner solve of an instance stops as soon as its
 * r'r meets its target (not only at the host's periodic look).
 *   nets: host array of n_nets U-Net handles (n_nets = 0: no network; nets
 *         and net_of may then be NULL).  Network k serves the instances i
 *         with net_of[i] == k, which must all have the same grid; its sample
 *         count ns is their number (sample j = the j-th of those instances in
 *         index order) and its grid that grid, or the 2x / 4x / 8x coarser one
 *         (extents divisible) with each extent rounded up to a multiple of 4:
 *         the extra cells are zero padding that the restriction never
 *         writes and the prolongation never reads.  The finest level whose
 *         grid matches is used.  net_of[i] = -1: no network for
 *         instance i (TPFA_OPT_FCG_FALLBACK's preconditioner from the start).
 *   lnk:  dev FP32 ln K over the concatenated cells (8-byte aligned when a
 *         network runs on a coarser grid; ignored without networks).
 *   coef, coef64, b, x: as cg_solve_batch.  Options of the batch:
 *   TPFA_OPT_INNER_RTOL, TPFA_OPT_MAX_OUTER, TPFA_OPT_FCG_M (default 4),
 *   TPFA_OPT_FCG_FALLBACK.  A network instance's cells must start at an even
 *   offset when it runs on a coarser grid.
 *   infos / total: as cg_solve_batch (rel_res_inner is NaN).  fell_back:
 *   host, n_inst ints (1 where the instance dropped its network), or NULL.
 * Calls on one batch must not overlap (they share its workspaces).  Waits for
 * the stream.  Returns as cg_solve_batch, or TPFA_EINTERNAL when a
 * tensor-core wait of a network gave up. */
int fcg_solve_batch(tpfa_batch* batch, tpfa_unet* const* nets, int n_nets, const int* net_of,
                    const float* coef, const double* coef64, const float* lnk, const double* b,
                    double* x, double tol, int64_t maxit, tpfa_cg_info* infos,
                    tpfa_cg_info* total, int* fell_back, void* stream);

/*
 * tpfa_apply_noalloc -- tpfa_apply for callers that cannot allocate device
 * memory.  The paper has no counterpart; this is a library convenience.
 *
 * Who needs it: code that is not allowed to call cudaMalloc / cudaFree, for
 * example a component inside a host application whose allocator owns all
 * device memory and passes in only the input and output buffers, or a loop
 * under a fixed memory budget where allocation (and the device
 * synchronisation cudaFree implies) is not permitted.  tpfa_create
 * allocates, so these callers cannot hold a context; this call needs none.
 *
 * It computes exactly what tpfa_apply computes (the same per-cell
 * arithmetic, always through the cp.async-staged kernel, where tpfa_apply
 * may take the TMA-staged one; pAp may differ from tpfa_apply's in the last
 * bits when the tiling differs) and allocates nothing.  Its reduction workspace is a
 * fixed array of 256 + 16384 * 8 = 131,328 bytes in the library's device
 * image, which every GPU that loads the library holds until the process
 * exits.
 *
 * grid  host pointer to the grid, checked by the same rules as tpfa_create
 *       (nx, ny, nz >= 1, the same size limits, dx, dy, dz, mu finite and
 *       > 0); the geometry fields do not enter the operator application.
 * coef, p, Ap, pAp, stream: as for tpfa_apply.
 *
 * Limits and behaviour:
 *  - the grid must be tiled with at most 16384 blocks of the sweep kernel
 *    (4 warps of 30 x 4 columns each, z-runs lengthened as needed), i.e.
 *    ceil(nx/30) * ceil(ny/4) <= 65536; larger grids get TPFA_EINVAL.
 *  - every call looks up the workspace's device address in the current
 *    context (cudaGetSymbolAddress, no allocation), so a device reset or a
 *    re-created primary context cannot leave a stale address behind.  The
 *    first call on a device may load the library's device code into that
 *    context; make that first call before any stream capture on the device.
 *  - all calls share the one workspace: calls whose kernels overlap on the
 *    GPU (different streams, or different host threads without ordering)
 *    race and give wrong pAp values.  The completion counter is cleared on
 *    the stream before each call that requests pAp.
 */
int tpfa_apply_noalloc(const tpfa_grid* grid, const float* coef, const float* p, float* Ap,
                       double* pAp, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TPFA_H */
