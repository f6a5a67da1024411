// Batched ensembles: many independent TPFA problems of different sizes solved
// together.  Every per-cell array of a batch is the concatenation of the
// instances' arrays (instance i at cell offset off[i], X innermost inside
// the instance).  The CG iterations of all instances run as one sweep launch
// per iteration inside one CUDA-graph while loop; each instance keeps its
// own scalars, completion counter and convergence flag, and the blocks of a
// converged instance return at once.  Coefficients, right-hand sides, FP64
// residuals and the refinement steps are launched per instance (a handful of
// launches per refinement step).
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "batch_internal.cuh"

using namespace tpfa;


namespace {

#define BK(call)                              \
  do {                                        \
    if ((call) != cudaSuccess) {              \
      cudaGetLastError();                     \
      return TPFA_ECUDA;                      \
    }                                         \
  } while (0)

CgVecs vecs_at(const CgVecs& v, int64_t off) {
  CgVecs o;
  for (int k = 0; k < 2; ++k) {
    o.r[k] = v.r[k] + off;
    o.p[k] = v.p[k] + off;
    o.q[k] = v.q[k] + off;
    o.v4[k] = v.v4[k] != nullptr ? v.v4[k] + off : nullptr;
  }
  o.e = v.e + off;
  return o;
}

// The batched CG loop runs the TMA-staged sweep unless the cp.async sweep is
// requested (or the driver lacks the tensor-map encoder).
bool batch_tma(const tpfa_batch* b) {
  if (b->sweep_sel == 1) return false;
  for (const Grid& g : b->g)
    if (!tma_sweep_ok(g, false, b->precond == 1)) return false;
  return true;
}

// Automatic z-runs of the TMA-staged batched sweep: one common run length,
// the longest (<= 128) that still gives the whole batch about four waves of
// two blocks per SM (per-instance planning would give the small instances
// one-plane runs, each re-reading two halo planes).
int batch_tma_zauto(const tpfa_batch* b) {
  const int64_t target = (int64_t)b->num_sms * 2 * 4;
  int z = 128;
  for (;;) {
    int64_t blocks = 0;
    for (const Grid& g : b->g)
      blocks += plan_tma(g, b->tma_tile, z, b->num_sms, false, b->precond == 1).nblocks;
    if (blocks >= target || z == 1) return z;
    z /= 2;
  }
}

// Per-instance tilings and tensor maps of the TMA-staged batched sweep for
// one coefficient array, the interleaved vector records on first use, and
// partial-sum room for its blocks.
int setup_batch_tma(tpfa_batch* b, const float* coef) {
  const int N = b->ninst;
  const size_t pad = ((size_t)b->cells + 15) / 16 * 16;
  if (b->vec4 == nullptr) {
    if (cudaMalloc(&b->vec4, 2 * pad * sizeof(float4)) != cudaSuccess) {
      cudaGetLastError();
      b->vec4 = nullptr;
      return TPFA_ENOMEM;
    }
  }
  if (b->maps_dev == nullptr) {
    if (cudaMalloc(&b->maps_dev, sizeof(CUtensorMap) * 4 * N) != cudaSuccess ||
        cudaMalloc(&b->tinst_dev, sizeof(TmaInst) * N) != cudaSuccess) {
      cudaGetLastError();
      return TPFA_ENOMEM;
    }
  }
  std::vector<CUtensorMap> maps(4 * (size_t)N);
  b->tinst.assign(N, TmaInst());
  const int zauto = batch_tma_zauto(b);
  int64_t blocks = 0;
  for (int i = 0; i < N; ++i) {
    const TmaPlan p = plan_tma(b->g[i], b->tma_tile, b->zc_req[i] > 0 ? b->zc_req[i] : zauto,
                               b->num_sms, false, b->precond == 1);
    CgVecs vi{};
    vi.v4[0] = b->vec4 + b->off[i];
    vi.v4[1] = b->vec4 + pad + b->off[i];
    TmaMaps m;
    if (!make_tma_maps(b->g[i], p, reinterpret_cast<const float4*>(coef) + b->off[i], nullptr,
                       vi, &m))
      return TPFA_ECUDA;
    maps[4 * i] = m.v[0];
    maps[4 * i + 1] = m.v[1];
    maps[4 * i + 2] = m.c;
    maps[4 * i + 3] = m.c;  // no M^-1 map with FP32 records
    TmaInst& I = b->tinst[i];
    I.g = b->g[i];
    I.zc = p.zc;
    I.nbx = (int)p.nbx;
    I.nby = (int)p.nby;
    I.off = b->off[i];
    I.bstart = blocks;
    I.nblocks = p.nblocks;
    I.id = i;
    I.maps = b->maps_dev + 4 * i;
    blocks += p.nblocks;
  }
  if (blocks > 0x7fffffff) return TPFA_EINVAL;
  b->tma_blocks = blocks;
  if ((size_t)blocks * 4 > b->partials_cap) {
    double* np = nullptr;
    if (cudaMalloc(&np, (size_t)blocks * 4 * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return TPFA_ENOMEM;
    }
    cudaDeviceSynchronize();
    cudaFree(b->partials);
    b->partials = np;
    b->partials_cap = (size_t)blocks * 4;
  }
  BK(cudaMemcpy(b->maps_dev, maps.data(), sizeof(CUtensorMap) * 4 * N, cudaMemcpyHostToDevice));
  BK(cudaMemcpy(b->tinst_dev, b->tinst.data(), sizeof(TmaInst) * N, cudaMemcpyHostToDevice));
  b->v.v4[0] = b->vec4;
  b->v.v4[1] = b->vec4 + pad;
  return TPFA_OK;
}

int use_dev(const tpfa_batch* b) {
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return TPFA_ECUDA;
  if (cur != b->device && cudaSetDevice(b->device) != cudaSuccess) return TPFA_ECUDA;
  return TPFA_OK;
}

bool grid_ok(const tpfa_grid& g) {
  if (g.nx < 1 || g.ny < 1 || g.nz < 1) return false;
  if (!(g.dx > 0) || !(g.dy > 0) || !(g.dz > 0) || !(g.mu > 0)) return false;
  if (!isfinite(g.dx) || !isfinite(g.dy) || !isfinite(g.dz) || !isfinite(g.mu)) return false;
  if ((double)g.nx * (double)g.ny + 2.0 * (double)g.nx > 2147483647.0) return false;
  return (double)g.nx * (double)g.ny * (double)g.nz <= 4.0e12;
}

// While loop {batched sweep; condition} for one coefficient array.
int ensure_batch_loop(tpfa_batch* b, const float* coef) {
  if (b->loop_exec && b->loop_key_coef == coef && b->loop_key_precond == b->precond &&
      b->loop_key_sweep == b->sweep_sel && b->loop_key_tile == b->tma_tile)
    return TPFA_OK;
  if (b->loop_exec) cudaGraphExecDestroy(b->loop_exec);
  b->loop_exec = nullptr;
  const bool tma = batch_tma(b);
  if (tma) {
    const int rc = setup_batch_tma(b, coef);
    if (rc) return rc;
  } else {
    b->v.v4[0] = b->v.v4[1] = nullptr;
  }
  cudaGraph_t graph = nullptr;
  BK(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
  if (e == cudaSuccess) {
    cudaGraph_t body = np.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(b->cap_stream, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e1 =
          tma ? launch_cg_sweep_tma_batch(b->tinst_dev, b->ninst, b->tma_blocks, b->tma_tile,
                                          b->precond == 1, b->v, b->st, b->partials, b->counters,
                                          b->cap_stream)
              : launch_cg_sweep_batch(b->inst_dev, b->ninst, b->sweep_blocks,
                                      reinterpret_cast<const float4*>(coef), b->v, b->st,
                                      b->partials, b->counters, b->precond == 1, b->cap_stream);
      cudaError_t e2 = launch_batch_cond(b->st, b->ninst, h, b->sweeps, 0, b->cap_stream);
      e = cudaStreamEndCapture(b->cap_stream, &body);
      if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : e2;
    }
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->loop_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b->loop_exec = nullptr;
    return TPFA_ECUDA;
  }
  b->loop_key_coef = coef;
  b->loop_key_precond = b->precond;
  b->loop_key_sweep = b->sweep_sel;
  b->loop_key_tile = b->tma_tile;
  return TPFA_OK;
}

}  // namespace

std::vector<int> batch_tma_zc_request(const tpfa_batch* b) {
  const int zauto = batch_tma_zauto(b);
  std::vector<int> z(b->ninst);
  for (int i = 0; i < b->ninst; ++i) z[i] = b->zc_req[i] > 0 ? b->zc_req[i] : zauto;
  return z;
}

extern "C" {

int tpfa_batch_create(const tpfa_grid* grids, int n_inst, const int* zc, tpfa_batch** out) {
  if (out == nullptr) return TPFA_EINVAL;
  *out = nullptr;
  if (grids == nullptr || n_inst < 1 || n_inst > 1 << 20) return TPFA_EINVAL;
  for (int i = 0; i < n_inst; ++i) {
    if (!grid_ok(grids[i])) return TPFA_EINVAL;
    if (zc != nullptr && (zc[i] < 0 || zc[i] > 1 << 20)) return TPFA_EINVAL;
  }
  tpfa_batch* b = new (std::nothrow) tpfa_batch();
  if (!b) return TPFA_ENOMEM;
  b->ninst = n_inst;
  b->inner_rtol = 1e-6;
  b->max_outer = 20;
  b->precond = 0;
  b->fcg_m = 4;
  b->fcg_fallback = 0;
  b->sweep_sel = 0;
  b->tma_tile = 0;
  b->zc_req.assign(n_inst, 0);
  if (zc != nullptr)
    for (int i = 0; i < n_inst; ++i) b->zc_req[i] = zc[i];
  int rc = TPFA_ECUDA;
  size_t pcap = 0;
  int64_t maxelem = 1;
  if (cudaGetDevice(&b->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess)
    goto fail;
  b->geo.assign(grids, grids + n_inst);
  b->off.assign(n_inst + 1, 0);
  for (int i = 0; i < n_inst; ++i) {
    Grid g;
    g.nx = grids[i].nx; g.ny = grids[i].ny; g.nz = grids[i].nz;
    g.plane = g.nx * g.ny;
    g.n = g.plane * g.nz;
    b->g.push_back(g);
    b->off[i + 1] = b->off[i] + g.n;
  }
  b->cells = b->off[n_inst];
  {
    // automatic z-runs: one common run length, the longest (<= 128) that
    // still gives the whole batch about four waves of 8 warps per SM
    int zauto = 128;
    const int64_t target = (int64_t)b->num_sms * 8 * 4;
    for (;;) {
      int64_t w = 0;
      for (int i = 0; i < n_inst; ++i) w += plan_sweep(b->g[i], 4, 4, zauto, b->num_sms).nwarps;
      if (w >= target || zauto == 1) break;
      zauto /= 2;
    }
    int64_t blocks = 0;
    for (int i = 0; i < n_inst; ++i) {
      const int z = (zc != nullptr && zc[i] > 0) ? zc[i] : zauto;
      const Sweep sw = plan_sweep(b->g[i], 4, 4, z, b->num_sms);
      BatchInst I;
      I.g = b->g[i];
      I.nwx = sw.nwx; I.nwy = sw.nwy; I.nwarps = sw.nwarps; I.zc = sw.zc;
      I.off = b->off[i];
      I.bstart = blocks;
      I.nblocks = sw.nblocks;
      blocks += sw.nblocks;
      b->inst.push_back(I);
      const int64_t eb = elem_blocks(b->g[i], b->num_sms);
      if (eb > maxelem) maxelem = eb;
    }
    b->sweep_blocks = blocks;
    if (blocks > 0x7fffffff) { rc = TPFA_EINVAL; goto fail; }
  }
  pcap = (size_t)b->sweep_blocks * 4;
  if ((size_t)maxelem * 2 > pcap) pcap = (size_t)maxelem * 2;
  b->partials_cap = pcap;
  rc = TPFA_ENOMEM;
  if (cudaMalloc(&b->inst_dev, sizeof(BatchInst) * n_inst) != cudaSuccess) goto fail;
  if (cudaMalloc(&b->st, sizeof(CgState) * n_inst) != cudaSuccess) goto fail;
  if (cudaMallocHost(&b->host_st, sizeof(CgState) * n_inst) != cudaSuccess) goto fail;
  if (cudaMalloc(&b->partials, pcap * sizeof(double)) != cudaSuccess) goto fail;
  if (cudaMalloc(&b->counters, sizeof(unsigned int) * (n_inst + 1)) != cudaSuccess) goto fail;
  if (cudaMalloc(&b->sweeps, sizeof(long long)) != cudaSuccess) goto fail;
  {
    const size_t pad = ((size_t)b->cells + 63) / 64 * 64;
    if (cudaMalloc(&b->vec, 7 * pad * sizeof(float)) != cudaSuccess) goto fail;
    if (cudaMalloc(&b->r64, (size_t)b->cells * sizeof(double)) != cudaSuccess) goto fail;
    float* v = b->vec;
    b->v.r[0] = v; b->v.r[1] = v + pad;
    b->v.p[0] = v + 2 * pad; b->v.p[1] = v + 3 * pad;
    b->v.q[0] = v + 4 * pad; b->v.q[1] = v + 5 * pad;
    b->v.e = v + 6 * pad;
  }
  rc = TPFA_ECUDA;
  if (cudaMemcpy(b->inst_dev, b->inst.data(), sizeof(BatchInst) * n_inst,
                 cudaMemcpyHostToDevice) != cudaSuccess)
    goto fail;
  if (cudaMemset(b->st, 0, sizeof(CgState) * n_inst) != cudaSuccess) goto fail;
  if (cudaMemset(b->counters, 0, sizeof(unsigned int) * (n_inst + 1)) != cudaSuccess) goto fail;
  if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) goto fail;
  for (int i = 0; i < 4; ++i)
    if (cudaEventCreate(&b->ev[i]) != cudaSuccess) goto fail;
  if (sweep_blocks_per_sm(4, 4) < 1) goto fail;
  *out = b;
  return TPFA_OK;
fail:
  cudaGetLastError();
  tpfa_batch_destroy(b);
  return rc;
}

int tpfa_batch_destroy(tpfa_batch* b) {
  if (b == nullptr) return TPFA_EINVAL;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != b->device) cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  if (b->loop_exec) cudaGraphExecDestroy(b->loop_exec);
  for (int i = 0; i < 4; ++i)
    if (b->ev[i]) cudaEventDestroy(b->ev[i]);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  cudaFree(b->vec);
  cudaFree(b->vec4);
  cudaFree(b->maps_dev);
  cudaFree(b->tinst_dev);
  cudaFree(b->r64);
  cudaFree(b->partials);
  cudaFree(b->counters);
  cudaFree(b->sweeps);
  cudaFree(b->st);
  cudaFree(b->inst_dev);
  if (b->host_st) cudaFreeHost(b->host_st);
  cudaGetLastError();
  if (cur >= 0 && cur != b->device) cudaSetDevice(cur);
  delete b;
  return TPFA_OK;
}

int tpfa_batch_offsets(const tpfa_batch* b, int64_t* offsets) {
  if (b == nullptr || offsets == nullptr) return TPFA_EINVAL;
  for (int i = 0; i <= b->ninst; ++i) offsets[i] = b->off[i];
  return TPFA_OK;
}

int tpfa_batch_zc(const tpfa_batch* b, int* zc) {
  if (b == nullptr || zc == nullptr) return TPFA_EINVAL;
  const bool tma = batch_tma(b);
  const int zauto = tma ? batch_tma_zauto(b) : 0;
  for (int i = 0; i < b->ninst; ++i) {
    if (tma)
      zc[i] = plan_tma(b->g[i], b->tma_tile, b->zc_req[i] > 0 ? b->zc_req[i] : zauto, b->num_sms,
                       false, b->precond == 1).zc;
    else
      zc[i] = (int)b->inst[i].zc;
  }
  return TPFA_OK;
}


int tpfa_batch_set_option(tpfa_batch* b, int option, double value) {
  if (b == nullptr || !isfinite(value)) return TPFA_EINVAL;
  switch (option) {
    case TPFA_OPT_INNER_RTOL:
      if (!(value > 0.0 && value < 1.0)) return TPFA_EINVAL;
      b->inner_rtol = value;
      return TPFA_OK;
    case TPFA_OPT_MAX_OUTER:
      if (value < 1 || value > 1000) return TPFA_EINVAL;
      b->max_outer = (int)value;
      return TPFA_OK;
    case TPFA_OPT_PRECOND:
      if (value != 0 && value != 1) return TPFA_EINVAL;
      b->precond = (int)value;
      return TPFA_OK;
    case TPFA_OPT_FCG_M:
      if (value != (int)value || value < 1 || value > 16) return TPFA_EINVAL;
      b->fcg_m = (int)value;
      return TPFA_OK;
    case TPFA_OPT_FCG_FALLBACK:
      if (value != 0 && value != 1) return TPFA_EINVAL;
      b->fcg_fallback = (int)value;
      return TPFA_OK;
    case TPFA_OPT_SWEEP:
      if (value != 0 && value != 1) return TPFA_EINVAL;
      b->sweep_sel = (int)value;
      return TPFA_OK;
    case TPFA_OPT_TMA_TILE:
      if (!(value >= 0 && value < tma_tile_count()) || value != floor(value)) return TPFA_EINVAL;
      b->tma_tile = (int)value;
      return TPFA_OK;
    default:
      return TPFA_EINVAL;
  }
}

int tpfa_batch_build_trans(tpfa_batch* b, const double* K, const uint8_t* dirichlet,
                           const double* d, double d_uniform, float* coef, double* coef64,
                           void* stream) {
  if (b == nullptr) return TPFA_EINVAL;
  int rc = use_dev(b);
  if (rc) return rc;
  const size_t n = (size_t)b->cells;
  if (!dev_ok(K, n * 8, 8, b->device) || !opt_dev_ok(dirichlet, n, 1, b->device) ||
      !opt_dev_ok(d, n * 8, 8, b->device) || !dev_ok(coef, n * 16, 16, b->device) ||
      !opt_dev_ok(coef64, n * 32, 16, b->device))
    return TPFA_EINVAL;
  if (d == nullptr && !(d_uniform >= 0.0 && isfinite(d_uniform))) return TPFA_EINVAL;
  for (int i = 0; i < b->ninst; ++i) {
    const int64_t o = b->off[i];
    BK(launch_build_trans(b->g[i], b->geo[i], K + o, dirichlet ? dirichlet + o : nullptr,
                          d ? d + o : nullptr, d_uniform, reinterpret_cast<float4*>(coef) + o,
                          coef64 ? coef64 + 4 * o : nullptr, (cudaStream_t)stream));
  }
  return TPFA_OK;
}

int tpfa_batch_build_rhs(tpfa_batch* b, const double* K, const uint8_t* dirichlet,
                         const double* q, const double* pD, double* rhs, void* stream) {
  if (b == nullptr) return TPFA_EINVAL;
  int rc = use_dev(b);
  if (rc) return rc;
  const size_t n = (size_t)b->cells;
  if (!dev_ok(K, n * 8, 8, b->device) || !opt_dev_ok(dirichlet, n, 1, b->device) ||
      !opt_dev_ok(q, n * 8, 8, b->device) || !opt_dev_ok(pD, n * 8, 8, b->device) ||
      !dev_ok(rhs, n * 8, 8, b->device))
    return TPFA_EINVAL;
  for (int i = 0; i < b->ninst; ++i) {
    const int64_t o = b->off[i];
    BK(launch_build_rhs(b->g[i], b->geo[i], K + o, dirichlet ? dirichlet + o : nullptr,
                        q ? q + o : nullptr, pD ? pD + o : nullptr, nullptr, nullptr, 0, rhs + o,
                        (cudaStream_t)stream));
  }
  return TPFA_OK;
}

int cg_solve_batch(tpfa_batch* b, const float* coef, const double* coef64, const double* rhs,
                   double* x, double tol, int64_t maxit, tpfa_cg_info* infos,
                   tpfa_cg_info* total, void* stream) {
  if (b == nullptr || !(tol > 0.0) || !isfinite(tol) || maxit < 1) return TPFA_EINVAL;
  int rc = use_dev(b);
  if (rc) return rc;
  const size_t n = (size_t)b->cells;
  if (!dev_ok(coef, n * 16, 16, b->device) || !dev_ok(coef64, n * 32, 16, b->device) ||
      !dev_ok(rhs, n * 8, 8, b->device) || !dev_ok(x, n * 8, 8, b->device))
    return TPFA_EINVAL;
  if ((const void*)rhs == (const void*)x) return TPFA_EINVAL;
  rc = ensure_batch_loop(b, coef);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int N = b->ninst;
  const float4* cf = reinterpret_cast<const float4*>(coef);
  unsigned int* ecounter = b->counters + N;  // shared by the per-instance helper kernels
  CgState* hs = b->host_st;
  auto read_states = [&]() -> int {
    BK(cudaMemcpyAsync(hs, b->st, sizeof(CgState) * N, cudaMemcpyDeviceToHost, s));
    BK(cudaStreamSynchronize(s));
    return TPFA_OK;
  };
  auto residual = [&](int i) -> cudaError_t {
    const int64_t o = b->off[i];
    return launch_residual64(b->g[i], coef64 + 4 * o, rhs + o, x + o, b->r64 + o, nullptr,
                             b->st + i, b->partials, ecounter, elem_blocks(b->g[i], b->num_sms),
                             s);
  };

  std::vector<double> bb(N), rel(N), best(N);
  std::vector<int64_t> iters(N, 0);
  std::vector<int> outer(N, 0), status(N, TPFA_OK), stalls(N, 0), active(N, 0);
  std::vector<double> rel_inner(N, NAN);
  int64_t launches = 0;
  double inner_ms = 0.0;

  BK(cudaMemsetAsync(b->counters, 0, sizeof(unsigned int) * (N + 1), s));
  BK(cudaEventRecord(b->ev[0], s));
  for (int i = 0; i < N; ++i) BK(residual(i));
  launches += N;
  rc = read_states();
  if (rc) return rc;
  for (int i = 0; i < N; ++i) {
    bb[i] = hs[i].bb64;
    rel[i] = bb[i] > 0 ? sqrt(hs[i].rr64 / bb[i]) : 0.0;
    best[i] = rel[i];
    if (!isfinite(hs[i].rr64) || !isfinite(bb[i])) {
      status[i] = TPFA_ENONFINITE;
    } else if (bb[i] == 0.0) {
      BK(cudaMemsetAsync(x + b->off[i], 0, sizeof(double) * b->g[i].n, s));
      rel[i] = 0.0;
      ++launches;
    }
  }
  for (int step = 0; step < b->max_outer; ++step) {
    int nact = 0;
    long long mx = 0;
    for (int i = 0; i < N; ++i) {
      active[i] = status[i] == TPFA_OK && rel[i] > tol && iters[i] < maxit;
      if (status[i] == TPFA_OK && rel[i] > tol && iters[i] >= maxit) status[i] = TPFA_NOTCONV;
      if (active[i]) {
        ++nact;
        if (maxit - iters[i] > mx) mx = maxit - iters[i];
      }
    }
    if (nact == 0) break;
    // inactive instances: mark done so their sweep blocks return at once
    for (int i = 0; i < N; ++i)
      if (!active[i]) hs[i].done = kConvTrue;
    BK(cudaMemcpyAsync(b->st, hs, sizeof(CgState) * N, cudaMemcpyHostToDevice, s));
    for (int i = 0; i < N; ++i) {
      if (!active[i]) continue;
      double rtol = 0.5 * tol / rel[i];
      if (rtol < b->inner_rtol) rtol = b->inner_rtol;
      if (rtol > 0.5) rtol = 0.5;
      BK(launch_prepare(b->g[i], b->r64 + b->off[i], vecs_at(b->v, b->off[i]), b->st + i, rtol,
                        (long long)(maxit - iters[i]), s));
      ++launches;
    }
    // while any instance runs: batched sweep + condition (guarded)
    for (int relaunch = 0;; ++relaunch) {
      // the captured condition kernel stops the loop once the sweep counter
      // passes 0: start it at minus the guard limit
      const long long start = -(2 * mx + 64);
      BK(cudaMemcpyAsync(b->sweeps, &start, sizeof(long long), cudaMemcpyHostToDevice, s));
      BK(cudaEventRecord(b->ev[2], s));
      BK(cudaGraphLaunch(b->loop_exec, s));
      BK(cudaEventRecord(b->ev[3], s));
      for (int i = 0; i < N; ++i) {
        if (!active[i]) continue;
        BK(launch_finalize(b->g[i], vecs_at(b->v, b->off[i]), b->st + i, b->partials, ecounter,
                           elem_blocks(b->g[i], b->num_sms),
                           b->precond ? cf + b->off[i] : nullptr, nullptr, s));
        ++launches;
      }
      rc = read_states();
      if (rc) return rc;
      float ms = 0.f;
      BK(cudaEventElapsedTime(&ms, b->ev[2], b->ev[3]));
      inner_ms += ms;
      int again = 0;
      for (int i = 0; i < N; ++i)
        if (active[i] && hs[i].done == kRunning) ++again;
      if (again == 0 || relaunch > 64) break;
    }
    {
      // every batched sweep launch (and the condition kernel after it) is
      // counted once in each instance's state: the most any instance saw
      long long sweeps = 0;
      for (int i = 0; i < N; ++i)
        if (active[i] && hs[i].launches > sweeps) sweeps = hs[i].launches;
      launches += 2 * sweeps;
    }
    for (int i = 0; i < N; ++i) {
      if (!active[i]) continue;
      iters[i] += hs[i].iter;
      rel_inner[i] = hs[i].rho0 > 0 ? sqrt(hs[i].rho / hs[i].rho0) : 0.0;
      const int d = hs[i].done;
      if (d == kGuard || d == kRunning) { status[i] = TPFA_EINTERNAL; active[i] = 0; }
      else if (d == kNonFinite) { status[i] = TPFA_ENONFINITE; active[i] = 0; }
      else if (d == kBreakdown && hs[i].iter == 0) { status[i] = TPFA_EBREAKDOWN; active[i] = 0; }
    }
    for (int i = 0; i < N; ++i) {
      if (!active[i]) continue;
      const int64_t o = b->off[i];
      BK(launch_correct(b->g[i], vecs_at(b->v, o), x + o, b->st + i, s));
      BK(residual(i));
      launches += 2;
      ++outer[i];
    }
    rc = read_states();
    if (rc) return rc;
    for (int i = 0; i < N; ++i) {
      if (!active[i]) continue;
      rel[i] = sqrt(hs[i].rr64 / bb[i]);
      if (!isfinite(rel[i])) { status[i] = TPFA_ENONFINITE; continue; }
      if (hs[i].done == kBreakdown) { status[i] = rel[i] <= tol ? TPFA_OK : TPFA_EBREAKDOWN; continue; }
      if (rel[i] <= tol) continue;
      if (rel[i] > 0.5 * best[i]) {
        if (++stalls[i] >= 3) status[i] = TPFA_ESTAGNATION;
      } else {
        stalls[i] = 0;
      }
      if (rel[i] < best[i]) best[i] = rel[i];
    }
  }
  for (int i = 0; i < N; ++i)
    if (status[i] == TPFA_OK && rel[i] > tol) status[i] = TPFA_NOTCONV;
  BK(cudaEventRecord(b->ev[1], s));
  BK(cudaEventSynchronize(b->ev[1]));
  float tms = 0.f;
  BK(cudaEventElapsedTime(&tms, b->ev[0], b->ev[1]));
  int worst = TPFA_OK;
  int64_t it_sum = 0;
  int out_max = 0;
  double rel_max = 0.0;
  for (int i = 0; i < N; ++i) {
    if (infos) {
      tpfa_cg_info& f = infos[i];
      memset(&f, 0, sizeof(f));
      f.iters = iters[i];
      f.outer = outer[i];
      f.status = status[i];
      f.rel_res_inner = rel_inner[i];
      f.rel_res_fp64 = rel[i];
      f.inner_ms = inner_ms;
      f.total_ms = tms;
      f.kernel_launches = launches;
    }
    if (status[i] < 0 && (worst >= 0 || status[i] < worst)) worst = status[i];
    else if (status[i] > 0 && worst == TPFA_OK) worst = status[i];
    it_sum += iters[i];
    if (outer[i] > out_max) out_max = outer[i];
    if (rel[i] > rel_max) rel_max = rel[i];
  }
  if (total) {
    memset(total, 0, sizeof(*total));
    total->iters = it_sum;
    total->outer = out_max;
    total->status = worst;
    total->rel_res_fp64 = rel_max;
    total->rel_res_inner = NAN;
    total->inner_ms = inner_ms;
    total->total_ms = tms;
    total->kernel_launches = launches;
  }
  return worst;
}

}  // extern "C"
