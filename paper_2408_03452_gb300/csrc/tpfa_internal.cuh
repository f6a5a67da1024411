// Internal declarations shared by the CUDA translation units of libtpfa.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sweep_plan.h"
#include "tpfa.h"

namespace tpfa {

constexpr int kWarp = 32;
constexpr int kElemThreads = 256; // threads per block in element-wise / per-cell kernels

// Device-resident scalars of one solve.  Written only by the last block of a
// reduction kernel (or by the prepare kernel), read by every block of the
// following kernels.
struct CgState {
  double alpha;        // alpha_{k-1}: x/r update applied at the start of the next sweep
  double beta;         // beta_{k-1}: direction update applied at the start of the next sweep
  double rho;          // r_k' r_k of the newest residual (true value of the stored vector)
  double rho0;         // r_0' r_0 of the current inner solve
  double rtol2;        // inner relative tolerance squared
  double rho_est;      // ||r_k - alpha_k q_k||^2 from the fused dot products
  double alpha_fin;    // step applied by the finalize kernel
  double scale;        // r32 = scale * r64 for the current inner solve
  double rr64, bb64;   // ||b - A x||^2 and ||b||^2 from the last FP64 residual
  double pap;          // p'Ap of the last tpfa_apply (when requested)
  long long iter;      // CG iterations completed in the current inner solve
  long long maxit;     // iteration limit of the current inner solve
  long long launches;  // sweep launches since prepare (guard against a runaway loop)
  long long guard_limit;
  int parity;          // which vector set (0/1) holds r_k, p_k, q_k
  int done;            // kRunning or one of the Done* codes
  int fault;           // a bounded wait inside a sweep ran out (ends the loop: kGuard)
  int pad1;
};

enum Done : int {
  kRunning = 0,
  kConvEst = 1,      // estimated ||r_{k+1}|| met the tolerance: finalize applies alpha_k
  kConvTrue = 2,     // ||r_k|| already met the tolerance: nothing left to apply
  kMaxit = 3,        // iteration limit: finalize applies alpha_k
  kBreakdown = -4,   // p'Ap <= 0
  kNonFinite = -5,
  kGuard = -6,       // runaway-loop guard tripped
};

bool sweep_config_ok(int vy, int stages);

// One instance of a batched solve: its grid, its sweep tiling, where its
// cells start in the concatenated arrays and which sweep blocks it owns.
struct BatchInst {
  Grid g;
  int64_t nwx, nwy, nwarps;
  int64_t zc;
  int64_t off;      // first cell in the concatenated arrays
  int64_t bstart;   // first sweep block
  int64_t nblocks;  // sweep blocks of this instance
};

// Vector set of the inner CG (two sets, ping-ponged between sweeps).
struct CgVecs {
  float* r[2];
  float* p[2];
  float* q[2];
  float* e;  // correction being accumulated (x of the inner solve)
  // Interleaved layout of the TMA-staged sweep (used instead of the arrays
  // above when set): per cell one record (r, q, p, x), two sets ping-ponged;
  // the set st->parity holds the current iterate, x included.
  float4* v4[2] = {nullptr, nullptr};
};

// Tiling of the TMA-staged CG sweep (sweep_tma.cu): blocks of w compute warps
// (plus one producer warp) own 32 columns x (w * vy) rows and march through
// zc planes with a ring of `stages` shared-memory stages.  b16: BF16 records;
// jac: Jacobi-preconditioned iteration (both use tile 0).
struct TmaPlan {
  int tile;    // index of the (w, vy, stages) choice
  bool b16, jac;
  bool apply;  // the operator application q = A p (tile 0), not a CG sweep
  bool dots;   // ... fused with the flexible-CG dot products (its own ring depth)
  int w, vy, stages, zc;
  int64_t nbx, nby, nbz, nblocks;
};
// Tensor maps of the arrays the TMA sweep reads: both vector-record sets, the
// coefficient records and (BF16 Jacobi) the M^-1 array.
struct TmaMaps {
  CUtensorMap v[2], c, d;
};
// the driver exposes the tensor-map encoder and the record rows have 16-byte
// strides (BF16 records: nx even; BF16 Jacobi: nx % 4 == 0)
bool tma_sweep_ok(const Grid& g, bool b16, bool jac);
int tma_tile_count();
TmaPlan plan_tma(const Grid& g, int tile, int zc_opt, int num_sms, bool b16, bool jac,
                 bool apply = false, bool dots = false);
int tma_blocks_per_sm(const TmaPlan& p);
bool make_tma_maps(const Grid& g, const TmaPlan& p, const void* coef, const float* dinv,
                   const CgVecs& v, TmaMaps* m);

// One instance of a batched TMA-staged sweep (device table): its grid and
// tiling, where its cells and blocks start, and its tensor maps (v[0], v[1],
// c, d of TmaMaps, in device memory).
struct TmaInst {
  Grid g;
  int zc, nbx, nby;
  int id;  // the instance's index in the batch (its scalars, counter, flags)
  int64_t off;
  int64_t bstart;
  int64_t nblocks;
  const CUtensorMap* maps;
};
// Batched CG sweep through the TMA-staged kernel: FP32 records, plain
// (any tile) or Jacobi (tile 0); v.v4 are the batch's record sets.
cudaError_t launch_cg_sweep_tma_batch(const TmaInst* inst, int ninst, int64_t nblocks, int tile,
                                      bool jac, CgVecs v, CgState* st, double* partials,
                                      unsigned int* counters, cudaStream_t s);

// Operator application q = A p (p'q into *pAp when given) through the
// TMA-staged kernel (plan from plan_tma(..., apply = true)).  Needs
// tma_apply_ok (the tensor-map encoder and nx % 4 == 0) and 16-byte aligned p
// and coefficients.  A copy that never lands makes the unwritten cells and p'q
// NaN.
bool tma_apply_ok(const Grid& g, bool b16);
cudaError_t launch_apply_tma(const Grid& g, const TmaPlan& p, const void* coef, const float* pin,
                             float* Ap, double* pAp, double* partials, unsigned int* counter,
                             cudaStream_t s);
// Tensor maps of a batched operator instance: out[0] the coefficient records,
// out[1 + i] the FP32 input in[i] (nin inputs).
bool make_apply_maps(const Grid& g, const TmaPlan& p, const void* coef, const float* const* in,
                     int nin, CUtensorMap* out);
// The batched operator fused with the flexible-CG dot products that read its
// result (A u itself is not stored): for each instance with
// (act[id] & need) == need, with u its input `which`, q = A u and w = M^-1 r:
// u'q into uq[id] and, at dots + id * kApplyDotsStride, u'q, u'r, q'w, then
// w'q_j and u'q_j (j < ndirs <= kApplyMaxDirs).  The instance's maps from
// index own0 on are own-cell maps (make_own_maps) of r, M^-1 and the
// direction slots; q_j is slot qmap[j].  partials: 3 + 2 ndirs doubles per
// block.
constexpr int kApplyMaxDirs = 4;
constexpr int kApplyDotsStride = 3 + 2 * kApplyMaxDirs;
bool make_own_maps(const Grid& g, const TmaPlan& p, const float* const* in, int nin,
                   CUtensorMap* out);
cudaError_t launch_apply_dots_tma_batch(const TmaInst* inst, int ninst, int64_t nblocks,
                                        int which, const int* act, int need, int own0,
                                        const int* qmap, int ndirs, double* uq, double* dots,
                                        double* partials, unsigned int* counters,
                                        cudaStream_t s);
// Batched operator through the TMA-staged kernel: inst[k].maps as from
// make_apply_maps, input `which`; the table may list any subset of the batch's
// instances (inst[k].id, bstart consecutive through the table); only instances
// with (act[id] & need) == need are applied; pAp and counters by id.
cudaError_t launch_apply_tma_batch(const TmaInst* inst, int ninst, int64_t nblocks, int which,
                                   float* Ap, double* pAp, const int* act, int need,
                                   double* partials, unsigned int* counters, cudaStream_t s);

// ---- launchers (kernels_*.cu) ---------------------------------------------

cudaError_t launch_build_trans(const Grid& g, const tpfa_grid& geo, const double* K,
                               const uint8_t* mask, const double* d, double d0, float4* coef,
                               double* coef64, cudaStream_t s);
cudaError_t launch_build_rhs(const Grid& g, const tpfa_grid& geo, const double* K,
                             const uint8_t* mask, const double* q, const double* pD,
                             const int64_t* src_idx, const double* src_val, int64_t n_src,
                             double* b, cudaStream_t s);

// coef: FP32 records (float4) or, with b16, BF16 records (4 x bf16 = uint2)
cudaError_t launch_apply(const Grid& g, const Sweep& sw, const void* coef, bool b16,
                         const float* p, float* Ap, double* pAp, double* partials,
                         unsigned int* counter, cudaStream_t s);
cudaError_t launch_cg_sweep(const Grid& g, const Sweep& sw, const void* coef, bool b16,
                            CgVecs v, CgState* st, double* partials, unsigned int* counter,
                            unsigned long long cond, int use_cond, cudaStream_t s);
// Jacobi-preconditioned CG sweep (stored q, VY = 4).  FP32 records carry D;
// BF16 records need dinv, M^-1 per cell from launch_dinv_bf16.
cudaError_t launch_cg_sweep_jacobi(const Grid& g, const Sweep& sw, const void* coef, bool b16,
                                   const float* dinv, CgVecs v, CgState* st, double* partials,
                                   unsigned int* counter, unsigned long long cond, int use_cond,
                                   cudaStream_t s);
cudaError_t launch_dinv_bf16(const Grid& g, const uint2* coef16, float* dinv, cudaStream_t s);
cudaError_t launch_accumulation(const Grid& g, const uint8_t* mask, const double* d, double d0,
                                const double* p_prev, double* b, cudaStream_t s);
cudaError_t launch_build_trans_bf16(const Grid& g, const tpfa_grid& geo, const double* K,
                                    const uint8_t* mask, const double* d, double d0,
                                    uint2* coef16, cudaStream_t s);
cudaError_t launch_residual64(const Grid& g, const double* coef64, const double* b,
                              const double* x, double* r, double* norms, CgState* st,
                              double* partials, unsigned int* counter, int nblocks,
                              cudaStream_t s);
cudaError_t launch_prepare(const Grid& g, const double* r64, CgVecs v, CgState* st,
                           double rtol, long long maxit, cudaStream_t s);
cudaError_t launch_finalize(const Grid& g, CgVecs v, CgState* st, double* partials,
                            unsigned int* counter, int nblocks, const float4* jac,
                            const float* dinv, cudaStream_t s);
cudaError_t launch_correct(const Grid& g, const CgVecs& v, double* x, const CgState* st,
                           cudaStream_t s);

int sweep_blocks_per_sm(int vy, int stages);
// CG sweep through the TMA-staged kernel (the variant the plan names)
cudaError_t launch_cg_sweep_tma(const Grid& g, const TmaPlan& p, const TmaMaps& m, CgVecs v,
                                CgState* st, double* partials, unsigned int* counter,
                                unsigned long long cond, int use_cond, cudaStream_t s);

// Batched CG sweep over every instance (VY = 4, 4 stages, FP32 records) and
// the one-block kernel that sets the while-loop condition after it.
cudaError_t launch_cg_sweep_batch(const BatchInst* inst, int ninst, int64_t nblocks,
                                  const float4* coef, CgVecs v, CgState* st, double* partials,
                                  unsigned int* counters, bool jac, cudaStream_t s);
cudaError_t launch_batch_cond(const CgState* st, int ninst, unsigned long long cond,
                              long long* sweeps, long long limit, cudaStream_t s);
// Batched operator Ap = A p over every instance i with (act[i] & need) ==
// need (the others are left untouched), pAp[i] = p_i'(A p)_i when pAp is
// given (partials: nblocks doubles; counters: one per instance, zero).
cudaError_t launch_apply_batch(const BatchInst* inst, int ninst, int64_t nblocks,
                               const float4* coef, const float* p, float* Ap, double* pAp,
                               const int* act, int need, double* partials,
                               unsigned int* counters, cudaStream_t s);

// Argument checks shared by the entry points: a device (or managed)
// allocation on `device` that holds [p, p + bytes) and is `align`-aligned.
// context accessors for the solvers outside api.cu
int64_t ctx_cells(const tpfa_ctx* c);
void ctx_dims(const tpfa_ctx* c, int64_t* d3);
double ctx_option(const tpfa_ctx* c, int option);
bool ctx_apply_tma_plan(const tpfa_ctx* c, TmaPlan* p, Grid* g, bool dots = false);
bool dev_ok(const void* p, size_t bytes, size_t align, int device);
bool opt_dev_ok(const void* p, size_t bytes, size_t align, int device);
int elem_blocks(const Grid& g, int num_sms);

}  // namespace tpfa
