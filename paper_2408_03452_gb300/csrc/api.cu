// C ABI of libtpfa: argument checking, workspace, CUDA-graph iteration loop
// and the FP64 iterative-refinement driver of cg_solve.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "tpfa_internal.cuh"

using namespace tpfa;

struct tpfa_ctx {
  Grid g;
  tpfa_grid geo;
  int device;
  int num_sms;
  // options
  double inner_rtol;
  double inner_rtol_bf16;
  int max_outer;
  int loop_mode;
  int vy;
  int stages;      // stages of the stored-q sweep and of tpfa_apply
  int precond;     // 0 = none (Alg. 1), 1 = Jacobi
  int fcg_m;       // directions retained by fcg_solve
  int fcg_fallback;  // fcg_solve fallback: 0 = unpreconditioned (default), 1 = Jacobi
  int zc;
  int chunk;
  int sweep_sel;   // CG sweep kernel: 0 = automatic, 1 = cp.async staged, 2 = TMA staged
  int tma_tile;    // tile choice of the TMA-staged sweep
  // reduction workspace
  CgState* st;
  CgState* host_st;  // pinned
  double* partials;
  size_t partials_cap;  // doubles
  unsigned int* counter;
  int elem_nblocks;
  // CG vectors (allocated on first solve)
  float* vec;
  double* r64;
  float* dinv;  // Jacobi with BF16 records: M^-1 per cell (allocated on first use)
  float4* vec4;  // interleaved vector records of the TMA-staged sweep (two sets, on first use)
  CgVecs v;
  // iteration-loop graph
  cudaGraphExec_t loop_exec;
  const void* loop_key_coef;
  bool loop_key_b16;
  int loop_key_precond;
  int loop_key_vy, loop_key_stages;
  int loop_key_zc, loop_key_mode, loop_key_chunk, loop_key_sweep, loop_key_tile;
  TmaMaps* maps;     // tensor maps of the TMA-staged sweep (host copy, built with the loop)
  TmaPlan tplan;
  cudaStream_t cap_stream;
  cudaEvent_t ev[4];
};

namespace tpfa {

typedef int (*AddrRangeFn)(unsigned long long*, size_t*, unsigned long long);

static AddrRangeFn addr_range_fn() {
  static AddrRangeFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<AddrRangeFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// A device (or managed) allocation on the current device that holds
// [p, p + bytes) and starts on an `align`-byte boundary.
bool dev_ok(const void* p, size_t bytes, size_t align, int device) {
  if (p == nullptr) return false;
  if (((uintptr_t)p) % align != 0) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeDevice) {
    if (at.device != device) return false;
  } else if (at.type != cudaMemoryTypeManaged) {
    return false;
  }
  AddrRangeFn fn = addr_range_fn();
  if (fn != nullptr) {
    unsigned long long base = 0;
    size_t size = 0;
    if (fn(&base, &size, (unsigned long long)(uintptr_t)p) == 0) {
      if ((unsigned long long)(uintptr_t)p + bytes > base + size) return false;
    }
  }
  return true;
}

bool opt_dev_ok(const void* p, size_t bytes, size_t align, int device) {
  return p == nullptr || dev_ok(p, bytes, align, device);
}

}  // namespace tpfa

namespace {

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return TPFA_ECUDA;      \
  } while (0)

int use_device(const tpfa_ctx* c) {
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return TPFA_ECUDA;
  if (cur != c->device && cudaSetDevice(c->device) != cudaSuccess) return TPFA_ECUDA;
  return TPFA_OK;
}

Sweep ctx_sweep(const tpfa_ctx* c) { return plan_sweep(c->g, c->vy, c->stages, c->zc, c->num_sms); }

// the sweep the CG loop runs
Sweep ctx_cg_sweep(const tpfa_ctx* c) { return ctx_sweep(c); }

// The CG loop runs the TMA-staged sweep (plain or Jacobi, FP32 or BF16
// records) unless the cp.async sweep is requested or the grid does not allow
// it (BF16 records need an even nx, BF16 Jacobi nx % 4 == 0).
bool use_tma(const tpfa_ctx* c, bool b16) {
  return c->sweep_sel != 1 && c->vy == 4 && tma_sweep_ok(c->g, b16, c->precond == 1);
}

// tpfa_apply: the TMA-staged operator unless the cp.async sweep is selected,
// another VY is, or the grid does not suit the copy engine; the arguments
// must then also be 16-byte aligned (cudaMalloc'd buffers are)
bool use_tma_apply(const tpfa_ctx* c, bool b16) {
  return c->sweep_sel != 1 && c->vy == 4 && tma_apply_ok(c->g, b16);
}
bool aligned16(const void* p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; }

// The CG vectors of a solve: the separate arrays, or with the TMA-staged
// sweep the interleaved records.
CgVecs loop_vecs(const tpfa_ctx* c, bool b16) {
  CgVecs v = c->v;
  if (use_tma(c, b16)) {
    const size_t pad = ((size_t)c->g.n + 15) / 16 * 16;
    v.v4[0] = c->vec4;
    v.v4[1] = c->vec4 + pad;
  }
  return v;
}

cudaError_t launch_cg(const tpfa_ctx* c, const Sweep& sw, const void* coef, bool b16,
                      unsigned long long cond, int use_cond, cudaStream_t s) {
  if (use_tma(c, b16))
    return launch_cg_sweep_tma(c->g, c->tplan, *c->maps, loop_vecs(c, b16), c->st, c->partials,
                               c->counter, cond, use_cond, s);
  if (c->precond == 1)
    return launch_cg_sweep_jacobi(c->g, sw, coef, b16, b16 ? c->dinv : nullptr, c->v, c->st,
                                  c->partials, c->counter, cond, use_cond, s);
  return launch_cg_sweep(c->g, sw, coef, b16, c->v, c->st, c->partials, c->counter, cond,
                         use_cond, s);
}

int ensure_partials(tpfa_ctx* c, size_t need) {
  if (need <= c->partials_cap) return TPFA_OK;
  double* p = nullptr;
  if (cudaMalloc(&p, need * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return TPFA_ENOMEM;
  }
  if (c->partials) {
    cudaDeviceSynchronize();
    cudaFree(c->partials);
  }
  c->partials = p;
  c->partials_cap = need;
  return TPFA_OK;
}

int ensure_vectors(tpfa_ctx* c) {
  if (c->vec != nullptr) return TPFA_OK;
  const size_t n = (size_t)c->g.n;
  // 7 float vectors (r, p, q twice, e), each padded to a 256-byte multiple
  const size_t pad = (n + 63) / 64 * 64;
  if (cudaMalloc(&c->vec, 7 * pad * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    c->vec = nullptr;
    return TPFA_ENOMEM;
  }
  if (cudaMalloc(&c->r64, n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(c->vec);
    c->vec = nullptr;
    c->r64 = nullptr;
    return TPFA_ENOMEM;
  }
  float* b = c->vec;
  c->v.r[0] = b; c->v.r[1] = b + pad;
  c->v.p[0] = b + 2 * pad; c->v.p[1] = b + 3 * pad;
  c->v.q[0] = b + 4 * pad; c->v.q[1] = b + 5 * pad;
  c->v.e = b + 6 * pad;
  return TPFA_OK;
}

void drop_loop(tpfa_ctx* c) {
  if (c->loop_exec) cudaGraphExecDestroy(c->loop_exec);
  c->loop_exec = nullptr;
  c->loop_key_coef = nullptr;
}

// Build (or reuse) the executable graph that runs CG sweeps until the device
// state says stop.  Mode 0: one while-node whose body holds two sweeps (the
// vector sets ping-pong); the last block of each sweep sets the loop
// condition.  Mode 1: `chunk` sweeps back to back, the host polls between
// launches.
int ensure_loop(tpfa_ctx* c, const void* coef, bool b16) {
  if (c->loop_exec && c->loop_key_coef == coef && c->loop_key_b16 == b16 &&
      c->loop_key_precond == c->precond && c->loop_key_vy == c->vy &&
      c->loop_key_stages == c->stages &&
      c->loop_key_zc == c->zc && c->loop_key_mode == c->loop_mode && c->loop_key_chunk == c->chunk &&
      c->loop_key_sweep == c->sweep_sel && c->loop_key_tile == c->tma_tile)
    return TPFA_OK;
  drop_loop(c);
  if ((b16 || c->precond) && c->vy != 4) return TPFA_EINVAL;  // 4-row warp tiles only
  const Sweep sw = ctx_cg_sweep(c);
  const bool tma = use_tma(c, b16);
  if (c->sweep_sel == 2 && !tma) return TPFA_EINVAL;  // TMA sweep requested but not possible
  int rc = TPFA_OK;
  if (tma) {
    c->tplan = plan_tma(c->g, c->tma_tile, c->zc, c->num_sms, b16, c->precond == 1);
    if (c->maps == nullptr) c->maps = new (std::nothrow) TmaMaps();
    if (c->maps == nullptr) return TPFA_ENOMEM;
    if (c->vec4 == nullptr) {
      const size_t pad = ((size_t)c->g.n + 15) / 16 * 16;  // 256-byte aligned second set
      if (cudaMalloc(&c->vec4, 2 * pad * sizeof(float4)) != cudaSuccess) {
        cudaGetLastError();
        c->vec4 = nullptr;
        return TPFA_ENOMEM;
      }
    }
    if (!make_tma_maps(c->g, c->tplan, coef, c->dinv, loop_vecs(c, b16), c->maps))
      return TPFA_ECUDA;
    rc = ensure_partials(c, (size_t)c->tplan.nblocks * 4);
    if (rc) return rc;
    if (tma_blocks_per_sm(c->tplan) < 1) return TPFA_ECUDA;
  } else {
    rc = ensure_partials(c, (size_t)sw.nblocks * 4);
    if (rc) return rc;
    if (sweep_blocks_per_sm(c->vy, c->stages) < 1) return TPFA_ECUDA;
  }
  cudaGraph_t graph = nullptr;
  cudaStream_t cs = c->cap_stream;
  const void* cf = coef;
  if (c->loop_mode == 0) {
    CK(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaGraphDestroy(graph);
      return TPFA_ECUDA;
    }
    cudaGraph_t body = np.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e1 = launch_cg(c, sw, cf, b16, h, 1, cs);
      cudaError_t e2 = launch_cg(c, sw, cf, b16, h, 1, cs);
      e = cudaStreamEndCapture(cs, &body);
      if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : e2;
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaGraphDestroy(graph);
      return TPFA_ECUDA;
    }
  } else {
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t el = cudaSuccess;
    for (int i = 0; i < c->chunk; ++i) {
      cudaError_t e = launch_cg(c, sw, cf, b16, 0, 0, cs);
      if (e != cudaSuccess) el = e;
    }
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (e != cudaSuccess || el != cudaSuccess) {
      cudaGetLastError();
      if (graph) cudaGraphDestroy(graph);
      return TPFA_ECUDA;
    }
  }
  cudaError_t e = cudaGraphInstantiate(&c->loop_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->loop_exec = nullptr;
    return TPFA_ECUDA;
  }
  c->loop_key_coef = coef;
  c->loop_key_b16 = b16;
  c->loop_key_precond = c->precond;
  c->loop_key_vy = c->vy;
  c->loop_key_stages = c->stages;
  c->loop_key_zc = c->zc;
  c->loop_key_mode = c->loop_mode;
  c->loop_key_chunk = c->chunk;
  c->loop_key_sweep = c->sweep_sel;
  c->loop_key_tile = c->tma_tile;
  return TPFA_OK;
}

int read_state(tpfa_ctx* c, cudaStream_t s) {
  CK(cudaMemcpyAsync(c->host_st, c->st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return TPFA_OK;
}

}  // namespace

namespace tpfa {
int64_t ctx_cells(const tpfa_ctx* c) { return c ? c->g.n : 0; }
void ctx_dims(const tpfa_ctx* c, int64_t* d3) {
  d3[0] = c->g.nx;
  d3[1] = c->g.ny;
  d3[2] = c->g.nz;
}
double ctx_option(const tpfa_ctx* c, int option) {
  switch (option) {
    case TPFA_OPT_INNER_RTOL: return c->inner_rtol;
    case TPFA_OPT_MAX_OUTER: return c->max_outer;
    case TPFA_OPT_FCG_M: return c->fcg_m;
    case TPFA_OPT_FCG_FALLBACK: return c->fcg_fallback;
    default: return 0.0;
  }
}

// The TMA-staged operator's plan for tpfa_apply's arguments (coef, p 16-byte
// aligned; dots: the variant fused with the flexible-CG dot products), or
// false when tpfa_apply would take the cp.async kernel.
bool ctx_apply_tma_plan(const tpfa_ctx* c, TmaPlan* p, Grid* g, bool dots) {
  if (!use_tma_apply(c, false)) return false;
  *g = c->g;
  *p = plan_tma(c->g, 0, c->zc, c->num_sms, false, false, true, dots);
  return true;
}
}  // namespace tpfa

extern "C" {

int tpfa_abi_version(void) { return TPFA_ABI_VERSION; }

const char* tpfa_strerror(int code) {
  switch (code) {
    case TPFA_OK: return "success";
    case TPFA_NOTCONV: return "iteration limit reached before the tolerance";
    case TPFA_EINVAL: return "invalid argument (size, NULL, misaligned or non-device pointer, option)";
    case TPFA_ENOMEM: return "device memory allocation failed";
    case TPFA_ECUDA: return "CUDA runtime error";
    case TPFA_EBREAKDOWN: return "CG breakdown: p'Ap <= 0, operator not positive definite";
    case TPFA_ENONFINITE: return "non-finite value in a reduction";
    case TPFA_EINTERNAL: return "internal iteration guard tripped";
    case TPFA_ESTAGNATION: return "iterative refinement stagnated";
    default: return "unknown status";
  }
}

int tpfa_create(const tpfa_grid* grid, tpfa_ctx** out) {
  if (out == nullptr) return TPFA_EINVAL;
  *out = nullptr;
  if (grid == nullptr) return TPFA_EINVAL;
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return TPFA_EINVAL;
  if (!(grid->dx > 0) || !(grid->dy > 0) || !(grid->dz > 0) || !(grid->mu > 0)) return TPFA_EINVAL;
  if (!isfinite(grid->dx) || !isfinite(grid->dy) || !isfinite(grid->dz) || !isfinite(grid->mu))
    return TPFA_EINVAL;
  // cell count must fit comfortably in int64 and in a CUDA grid of warps
  const double n = (double)grid->nx * (double)grid->ny * (double)grid->nz;
  if (n > 4.0e12) return TPFA_EINVAL;
  // the sweep kernels address a z-plane (plus two rows) with 32-bit offsets
  if ((double)grid->nx * (double)grid->ny + 2.0 * (double)grid->nx > 2147483647.0) return TPFA_EINVAL;
  tpfa_ctx* c = new (std::nothrow) tpfa_ctx();
  if (!c) return TPFA_ENOMEM;
  memset((void*)c, 0, sizeof(*c));
  c->geo = *grid;
  c->g.nx = grid->nx; c->g.ny = grid->ny; c->g.nz = grid->nz;
  c->g.plane = grid->nx * grid->ny;
  c->g.n = c->g.plane * grid->nz;
  c->inner_rtol = 1e-6;
  c->inner_rtol_bf16 = 1e-3;
  c->max_outer = 20;
  c->fcg_m = 4;
  c->fcg_fallback = 0;
  c->loop_mode = 0;
  c->vy = 4;
  c->stages = 4;
  c->precond = 0;
  c->zc = 0;
  c->chunk = 32;
  int rc = TPFA_ECUDA;
  if (cudaGetDevice(&c->device) != cudaSuccess) goto fail;
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
    goto fail;
  c->elem_nblocks = elem_blocks(c->g, c->num_sms);
  rc = TPFA_ENOMEM;
  if (cudaMalloc(&c->st, sizeof(CgState)) != cudaSuccess) goto fail;
  if (cudaMalloc(&c->counter, 64) != cudaSuccess) goto fail;
  if (cudaMallocHost(&c->host_st, sizeof(CgState)) != cudaSuccess) goto fail;
  rc = TPFA_ECUDA;
  if (cudaMemset(c->st, 0, sizeof(CgState)) != cudaSuccess) goto fail;
  if (cudaMemset(c->counter, 0, 64) != cudaSuccess) goto fail;
  if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) goto fail;
  for (int i = 0; i < 4; ++i)
    if (cudaEventCreate(&c->ev[i]) != cudaSuccess) goto fail;
  {
    const Sweep sw = ctx_sweep(c);
    size_t need = (size_t)sw.nblocks * 4;
    if (need < (size_t)c->elem_nblocks * 2) need = (size_t)c->elem_nblocks * 2;
    rc = ensure_partials(c, need);
    if (rc) goto fail;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) { rc = TPFA_ECUDA; goto fail; }
  *out = c;
  return TPFA_OK;
fail:
  cudaGetLastError();
  tpfa_destroy(c);
  return rc;
}

int tpfa_destroy(tpfa_ctx* c) {
  if (c == nullptr) return TPFA_EINVAL;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != c->device) cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  drop_loop(c);
  for (int i = 0; i < 4; ++i)
    if (c->ev[i]) cudaEventDestroy(c->ev[i]);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->vec) cudaFree(c->vec);
  if (c->r64) cudaFree(c->r64);
  if (c->dinv) cudaFree(c->dinv);
  if (c->vec4) cudaFree(c->vec4);
  delete c->maps;
  if (c->partials) cudaFree(c->partials);
  if (c->counter) cudaFree(c->counter);
  if (c->st) cudaFree(c->st);
  if (c->host_st) cudaFreeHost(c->host_st);
  cudaGetLastError();
  if (cur >= 0 && cur != c->device) cudaSetDevice(cur);
  delete c;
  return TPFA_OK;
}

int tpfa_set_option(tpfa_ctx* c, int option, double value) {
  if (c == nullptr || !isfinite(value)) return TPFA_EINVAL;
  switch (option) {
    case TPFA_OPT_INNER_RTOL:
      if (!(value > 0.0 && value < 1.0)) return TPFA_EINVAL;
      c->inner_rtol = value;
      return TPFA_OK;
    case TPFA_OPT_INNER_RTOL_BF16:
      if (!(value > 0.0 && value < 1.0)) return TPFA_EINVAL;
      c->inner_rtol_bf16 = value;
      return TPFA_OK;
    case TPFA_OPT_MAX_OUTER:
      if (value < 1 || value > 1000) return TPFA_EINVAL;
      c->max_outer = (int)value;
      return TPFA_OK;
    case TPFA_OPT_LOOP:
      if (value != 0 && value != 1) return TPFA_EINVAL;
      c->loop_mode = (int)value;
      return TPFA_OK;
    case TPFA_OPT_TILE_VY:
      if (!sweep_config_ok((int)value, (int)value == 8 ? 3 : c->stages) || value != floor(value))
        return TPFA_EINVAL;
      c->vy = (int)value;
      if (c->vy == 8) c->stages = 3;
      return TPFA_OK;
    case TPFA_OPT_STAGES:
      if (!sweep_config_ok(c->vy, (int)value) || value != floor(value)) return TPFA_EINVAL;
      c->stages = (int)value;
      return TPFA_OK;
    case TPFA_OPT_PRECOND:
      if (value != 0 && value != 1) return TPFA_EINVAL;
      c->precond = (int)value;
      return TPFA_OK;
    case TPFA_OPT_FCG_M:
      if (!(value >= 1 && value <= 16) || value != floor(value)) return TPFA_EINVAL;
      c->fcg_m = (int)value;
      return TPFA_OK;
    case TPFA_OPT_FCG_FALLBACK:
      if (value != 0 && value != 1) return TPFA_EINVAL;
      c->fcg_fallback = (int)value;
      return TPFA_OK;
    case TPFA_OPT_TILE_ZC:
      if (value < 0 || value > 1 << 20 || value != floor(value)) return TPFA_EINVAL;
      c->zc = (int)value;
      return TPFA_OK;
    case TPFA_OPT_CHUNK:
      if (value < 1 || value > 4096 || value != floor(value)) return TPFA_EINVAL;
      c->chunk = (int)value;
      return TPFA_OK;
    case TPFA_OPT_SWEEP:
      if (value != 0 && value != 1 && value != 2) return TPFA_EINVAL;
      c->sweep_sel = (int)value;
      return TPFA_OK;
    case TPFA_OPT_TMA_TILE:
      if (!(value >= 0 && value < tma_tile_count()) || value != floor(value)) return TPFA_EINVAL;
      c->tma_tile = (int)value;
      return TPFA_OK;
    default:
      return TPFA_EINVAL;
  }
}

int tpfa_sweep_tiling(const tpfa_ctx* c, int which, int64_t* out) {
  if (c == nullptr || out == nullptr || which < 0 || which > 3) return TPFA_EINVAL;
  const Sweep sw = ctx_sweep(c);
  const bool b16 = which == 1 || which == 3;
  if (which >= 2) {
    // the operator (TMA-staged for 16-byte aligned arguments)
    if (use_tma_apply(c, b16)) {
      const TmaPlan p = plan_tma(c->g, 0, c->zc, c->num_sms, b16, false, true);
      out[0] = 2;
      out[1] = p.vy;
      out[2] = p.stages;
      out[3] = p.w;
      out[4] = p.zc;
      out[5] = p.nblocks;
      return TPFA_OK;
    }
  } else if (use_tma(c, b16)) {
    const TmaPlan p = plan_tma(c->g, c->tma_tile, c->zc, c->num_sms, b16, c->precond == 1);
    out[0] = 2;
    out[1] = p.vy;
    out[2] = p.stages;
    out[3] = p.w;
    out[4] = p.zc;
    out[5] = p.nblocks;
    return TPFA_OK;
  }
  if (which < 2 && c->sweep_sel == 2) return TPFA_EINVAL;
  out[0] = 1;
  out[1] = sw.vy;
  out[2] = sw.stages;
  out[3] = sw.warps;
  out[4] = sw.zc;
  out[5] = sw.nblocks;
  return TPFA_OK;
}

int tpfa_build_trans(tpfa_ctx* c, const double* K, const uint8_t* dirichlet, const double* d,
                     double d_uniform, float* coef, double* coef64, void* stream) {
  if (c == nullptr) return TPFA_EINVAL;
  int rc = use_device(c);
  if (rc) return rc;
  const size_t n = (size_t)c->g.n;
  if (!dev_ok(K, n * 8, 8, c->device) || !opt_dev_ok(dirichlet, n, 1, c->device) ||
      !opt_dev_ok(d, n * 8, 8, c->device) || !dev_ok(coef, n * 16, 16, c->device) ||
      !opt_dev_ok(coef64, n * 32, 16, c->device))
    return TPFA_EINVAL;
  if (d == nullptr && !(d_uniform >= 0.0 && isfinite(d_uniform))) return TPFA_EINVAL;
  CK(launch_build_trans(c->g, c->geo, K, dirichlet, d, d_uniform, reinterpret_cast<float4*>(coef),
                        coef64, (cudaStream_t)stream));
  return TPFA_OK;
}

int tpfa_build_rhs(tpfa_ctx* c, const double* K, const uint8_t* dirichlet, const double* q,
                   const double* pD, const int64_t* src_idx, const double* src_val, int64_t n_src,
                   double* b, void* stream) {
  if (c == nullptr || n_src < 0) return TPFA_EINVAL;
  int rc = use_device(c);
  if (rc) return rc;
  const size_t n = (size_t)c->g.n;
  if (!dev_ok(K, n * 8, 8, c->device) || !opt_dev_ok(dirichlet, n, 1, c->device) ||
      !opt_dev_ok(q, n * 8, 8, c->device) || !opt_dev_ok(pD, n * 8, 8, c->device) ||
      !dev_ok(b, n * 8, 8, c->device))
    return TPFA_EINVAL;
  if (n_src > 0 && (!dev_ok(src_idx, (size_t)n_src * 8, 8, c->device) ||
                    !dev_ok(src_val, (size_t)n_src * 8, 8, c->device)))
    return TPFA_EINVAL;
  CK(launch_build_rhs(c->g, c->geo, K, dirichlet, q, pD, src_idx, src_val, n_src, b,
                      (cudaStream_t)stream));
  return TPFA_OK;
}

static int apply_impl(tpfa_ctx* c, const void* coef, bool b16, const float* p, float* Ap,
                      double* pAp, void* stream) {
  if (c == nullptr) return TPFA_EINVAL;
  int rc = use_device(c);
  if (rc) return rc;
  const size_t n = (size_t)c->g.n;
  if (!dev_ok(coef, n * (b16 ? 8 : 16), b16 ? 8 : 16, c->device) ||
      !dev_ok(p, n * 4, 4, c->device) || !dev_ok(Ap, n * 4, 4, c->device) ||
      !opt_dev_ok(pAp, 8, 8, c->device))
    return TPFA_EINVAL;
  if ((const void*)p == (const void*)Ap) return TPFA_EINVAL;
  if (b16 && c->vy != 4) return TPFA_EINVAL;
  if (use_tma_apply(c, b16) && aligned16(coef) && aligned16(p)) {
    const TmaPlan tp = plan_tma(c->g, 0, c->zc, c->num_sms, b16, false, true);
    if (pAp != nullptr) {
      rc = ensure_partials(c, (size_t)tp.nblocks);
      if (rc) return rc;
    }
    CK(launch_apply_tma(c->g, tp, coef, p, Ap, pAp, c->partials, c->counter,
                        (cudaStream_t)stream));
    return TPFA_OK;
  }
  const Sweep sw = ctx_sweep(c);
  if (pAp != nullptr) {
    rc = ensure_partials(c, (size_t)sw.nblocks);
    if (rc) return rc;
  }
  CK(launch_apply(c->g, sw, coef, b16, p, Ap, pAp, c->partials, c->counter, (cudaStream_t)stream));
  return TPFA_OK;
}

int tpfa_build_rhs_transient(tpfa_ctx* c, const double* K, const uint8_t* dirichlet,
                             const double* q, const double* pD, const int64_t* src_idx,
                             const double* src_val, int64_t n_src, const double* d,
                             double d_uniform, const double* p_prev, double* b, void* stream) {
  if (c == nullptr) return TPFA_EINVAL;
  int rc = use_device(c);
  if (rc) return rc;
  const size_t n = (size_t)c->g.n;
  if (!dev_ok(p_prev, n * 8, 8, c->device) || !opt_dev_ok(d, n * 8, 8, c->device)) return TPFA_EINVAL;
  if (d == nullptr && !(d_uniform >= 0.0 && isfinite(d_uniform))) return TPFA_EINVAL;
  if ((const void*)p_prev == (const void*)b) return TPFA_EINVAL;
  rc = tpfa_build_rhs(c, K, dirichlet, q, pD, src_idx, src_val, n_src, b, stream);
  if (rc) return rc;
  CK(launch_accumulation(c->g, dirichlet, d, d_uniform, p_prev, b, (cudaStream_t)stream));
  return TPFA_OK;
}

int tpfa_apply(tpfa_ctx* c, const float* coef, const float* p, float* Ap, double* pAp,
               void* stream) {
  return apply_impl(c, coef, false, p, Ap, pAp, stream);
}

int tpfa_apply_bf16(tpfa_ctx* c, const uint16_t* coef16, const float* p, float* Ap, double* pAp,
                    void* stream) {
  return apply_impl(c, coef16, true, p, Ap, pAp, stream);
}

int tpfa_build_trans_bf16(tpfa_ctx* c, const double* K, const uint8_t* dirichlet, const double* d,
                          double d_uniform, uint16_t* coef16, void* stream) {
  if (c == nullptr) return TPFA_EINVAL;
  int rc = use_device(c);
  if (rc) return rc;
  const size_t n = (size_t)c->g.n;
  if (!dev_ok(K, n * 8, 8, c->device) || !opt_dev_ok(dirichlet, n, 1, c->device) ||
      !opt_dev_ok(d, n * 8, 8, c->device) || !dev_ok(coef16, n * 8, 8, c->device))
    return TPFA_EINVAL;
  if (d == nullptr && !(d_uniform >= 0.0 && isfinite(d_uniform))) return TPFA_EINVAL;
  CK(launch_build_trans_bf16(c->g, c->geo, K, dirichlet, d, d_uniform,
                             reinterpret_cast<uint2*>(coef16), (cudaStream_t)stream));
  return TPFA_OK;
}

int tpfa_residual64(tpfa_ctx* c, const double* coef64, const double* b, const double* x,
                    double* r, double* norms, void* stream) {
  if (c == nullptr) return TPFA_EINVAL;
  int rc = use_device(c);
  if (rc) return rc;
  const size_t n = (size_t)c->g.n;
  if (!dev_ok(coef64, n * 32, 16, c->device) || !dev_ok(b, n * 8, 8, c->device) ||
      !dev_ok(x, n * 8, 8, c->device) || !dev_ok(r, n * 8, 8, c->device) ||
      !opt_dev_ok(norms, 16, 8, c->device))
    return TPFA_EINVAL;
  if ((const void*)r == (const void*)b || (const void*)r == (const void*)x) return TPFA_EINVAL;
  CK(launch_residual64(c->g, coef64, b, x, r, norms, nullptr, c->partials, c->counter,
                       c->elem_nblocks, (cudaStream_t)stream));
  return TPFA_OK;
}

static int solve_impl(tpfa_ctx* c, const void* coef, bool b16, const double* coef64,
                      const double* b, double* x, double tol, int64_t maxit, tpfa_cg_info* info,
                      void* stream) {
  tpfa_cg_info inf;
  memset(&inf, 0, sizeof(inf));
  inf.rel_res_fp64 = NAN;
  inf.rel_res_inner = NAN;
  int rc = TPFA_OK;
  if (info) *info = inf;
  if (c == nullptr || !(tol > 0.0) || !isfinite(tol) || maxit < 1) return TPFA_EINVAL;
  rc = use_device(c);
  if (rc) return rc;
  const size_t n = (size_t)c->g.n;
  if (!dev_ok(coef, n * (b16 ? 8 : 16), b16 ? 8 : 16, c->device) ||
      !dev_ok(coef64, n * 32, 16, c->device) || !dev_ok(b, n * 8, 8, c->device) ||
      !dev_ok(x, n * 8, 8, c->device))
    return TPFA_EINVAL;
  if ((const void*)b == (const void*)x) return TPFA_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  rc = ensure_vectors(c);
  if (rc) return rc;
  if (b16 && c->precond && c->dinv == nullptr) {
    if (cudaMalloc(&c->dinv, n * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      c->dinv = nullptr;
      return TPFA_ENOMEM;
    }
  }
  rc = ensure_loop(c, coef, b16);
  if (rc) return rc;
  const CgVecs vecs = loop_vecs(c, b16);
  CK(cudaMemsetAsync(c->counter, 0, 64, s));
  CK(cudaEventRecord(c->ev[0], s));
  if (b16 && c->precond) {
    // M^-1 from the BF16 records of this call (they may have changed since
    // the last solve with the same pointer)
    CK(launch_dinv_bf16(c->g, static_cast<const uint2*>(coef), c->dinv, s));
  }

  CgState* hs = c->host_st;
  double inner_ms = 0.0;
  int64_t total_iters = 0;
  int64_t launches = 0;
  int outer = 0;
  // r64 = b - A x
  CK(launch_residual64(c->g, coef64, b, x, c->r64, nullptr, c->st, c->partials, c->counter,
                       c->elem_nblocks, s));
  launches += 1;
  rc = read_state(c, s);
  if (rc) return rc;
  const double bb = hs->bb64;
  double rr = hs->rr64;
  double rel = bb > 0 ? sqrt(rr / bb) : 0.0;
  double rel_inner = NAN;
  int status = TPFA_OK;
  if (!isfinite(rr) || !isfinite(bb)) {
    status = TPFA_ENONFINITE;
  } else if (bb == 0.0) {
    CK(cudaMemsetAsync(x, 0, n * sizeof(double), s));
    rel = 0.0;
    launches += 1;
  } else {
    double best = rel;
    int stalls = 0;
    while (rel > tol) {
      if (total_iters >= maxit) { status = TPFA_NOTCONV; break; }
      if (outer >= c->max_outer) { status = TPFA_NOTCONV; break; }
      double rtol = 0.5 * tol / rel;
      const double floor_rtol = b16 ? c->inner_rtol_bf16 : c->inner_rtol;
      if (rtol < floor_rtol) rtol = floor_rtol;
      if (rtol > 0.5) rtol = 0.5;
      CK(launch_prepare(c->g, c->r64, vecs, c->st, rtol, (long long)(maxit - total_iters), s));
      launches += 1;
      int inner_status = kRunning;
      // host-side bound on relaunches (the device guard normally ends the
      // loop first): chunks of sweeps in mode 1, finalize restarts in mode 0
      const long long max_relaunch = (maxit - total_iters) / (c->loop_mode == 1 ? c->chunk : 1) + 64;
      long long relaunch = 0;
      for (;;) {
        if (++relaunch > max_relaunch) { inner_status = kGuard; break; }
        CK(cudaEventRecord(c->ev[2], s));
        CK(cudaGraphLaunch(c->loop_exec, s));
        CK(cudaEventRecord(c->ev[3], s));
        if (c->loop_mode == 1) {
          rc = read_state(c, s);
          if (rc) return rc;
          float ms = 0.f;
          CK(cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]));
          inner_ms += ms;
          if (hs->done == kRunning) continue;
        }
        CK(launch_finalize(c->g, vecs, c->st, c->partials, c->counter, c->elem_nblocks,
                           c->precond && !b16 ? static_cast<const float4*>(coef) : nullptr,
                           c->precond && b16 ? c->dinv : nullptr, s));
        launches += 1;
        rc = read_state(c, s);
        if (rc) return rc;
        if (c->loop_mode == 0) {
          float ms = 0.f;
          CK(cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]));
          inner_ms += ms;
        }
        if (hs->done == kRunning) continue;  // finalize armed a restart
        inner_status = hs->done;
        break;
      }
      total_iters += hs->iter;
      launches += hs->launches;
      rel_inner = hs->rho0 > 0 ? sqrt(hs->rho / hs->rho0) : 0.0;
      if (inner_status == kGuard) { status = TPFA_EINTERNAL; break; }
      if (inner_status == kNonFinite) { status = TPFA_ENONFINITE; break; }
      if (inner_status == kBreakdown && hs->iter == 0) { status = TPFA_EBREAKDOWN; break; }
      // x += e / scale;  r64 = b - A x
      CK(launch_correct(c->g, vecs, x, c->st, s));
      CK(launch_residual64(c->g, coef64, b, x, c->r64, nullptr, c->st, c->partials, c->counter,
                           c->elem_nblocks, s));
      launches += 2;
      ++outer;
      rc = read_state(c, s);
      if (rc) return rc;
      rr = hs->rr64;
      rel = sqrt(rr / bb);
      if (!isfinite(rel)) { status = TPFA_ENONFINITE; break; }
      if (inner_status == kBreakdown) { status = rel <= tol ? TPFA_OK : TPFA_EBREAKDOWN; break; }
      if (rel <= tol) break;
      if (rel > 0.5 * best) {
        if (++stalls >= 3) { status = TPFA_ESTAGNATION; break; }
      } else {
        stalls = 0;
      }
      if (rel < best) best = rel;
    }
  }
  CK(cudaEventRecord(c->ev[1], s));
  CK(cudaEventSynchronize(c->ev[1]));
  float tms = 0.f;
  CK(cudaEventElapsedTime(&tms, c->ev[0], c->ev[1]));
  inf.iters = total_iters;
  inf.outer = outer;
  inf.status = status;
  inf.rel_res_inner = rel_inner;
  inf.rel_res_fp64 = rel;
  inf.inner_ms = inner_ms;
  inf.total_ms = tms;
  inf.kernel_launches = launches;
  if (info) *info = inf;
  return status;
}

int cg_solve(tpfa_ctx* c, const float* coef, const double* coef64, const double* b, double* x,
             double tol, int64_t maxit, tpfa_cg_info* info, void* stream) {
  return solve_impl(c, coef, false, coef64, b, x, tol, maxit, info, stream);
}

int cg_solve_bf16(tpfa_ctx* c, const uint16_t* coef16, const double* coef64, const double* b,
                  double* x, double tol, int64_t maxit, tpfa_cg_info* info, void* stream) {
  return solve_impl(c, coef16, true, coef64, b, x, tol, maxit, info, stream);
}

}  // extern "C"
