// The batch object shared by the batched solvers (batch.cu: plain and
// Jacobi CG sweeps; fcg.cu: flexible CG with the learned preconditioner).
#pragma once

#include <vector>

#include "tpfa_internal.cuh"

struct tpfa_batch {
  int ninst;
  int device;
  int num_sms;
  std::vector<tpfa_grid> geo;
  std::vector<tpfa::Grid> g;
  std::vector<int64_t> off;  // ninst + 1
  std::vector<tpfa::BatchInst> inst;
  int64_t cells;
  int64_t sweep_blocks;
  double inner_rtol;
  int max_outer;
  int precond;
  int fcg_m;         // fcg_solve_batch: retained directions
  int fcg_fallback;  // fcg_solve_batch: 0 = plain CG after a network failure, 1 = Jacobi
  tpfa::BatchInst* inst_dev;
  tpfa::CgState* st;
  tpfa::CgState* host_st;
  double* partials;
  unsigned int* counters;  // ninst for the sweep + 1 for the per-instance helper kernels
  long long* sweeps;
  float* vec;
  double* r64;
  tpfa::CgVecs v;
  // TMA-staged batched sweep (the default): requested z-runs per instance,
  // interleaved vector records, per-instance tilings and tensor maps
  int sweep_sel;  // 0 = automatic (TMA), 1 = cp.async-staged sweep
  int tma_tile;
  std::vector<int> zc_req;
  float4* vec4;
  std::vector<tpfa::TmaInst> tinst;
  tpfa::TmaInst* tinst_dev;
  CUtensorMap* maps_dev;
  int64_t tma_blocks;
  size_t partials_cap;  // doubles
  cudaGraphExec_t loop_exec;
  const void* loop_key_coef;
  int loop_key_precond;
  int loop_key_sweep, loop_key_tile;
  cudaStream_t cap_stream;
  cudaEvent_t ev[4];
};

// Requested z-run of every instance in the batch's TMA-staged sweeps: the
// instance's own request, else the batch-wide automatic length (the batched
// CG sweep and the batched flexible-CG operator use the same runs).
std::vector<int> batch_tma_zc_request(const tpfa_batch* b);
