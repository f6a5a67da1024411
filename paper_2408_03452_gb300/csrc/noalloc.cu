// tpfa_apply_noalloc: the operator application of tpfa_apply, with its
// reduction workspace in a fixed device array instead of a context.
//
// Some callers cannot allocate device memory: a plugin or solver component
// embedded in a host application whose allocator owns all device memory and
// hands it only the input and output buffers, or a loop with a fixed memory
// budget where cudaMalloc / cudaFree (which may synchronise the device) are
// not allowed.  tpfa_create allocates, so such callers cannot hold a
// context; this entry point needs none and allocates nothing.
#include <math.h>

#include "tpfa_internal.cuh"

namespace {

using namespace tpfa;

// Fixed workspace: one completion counter (first 256 bytes) and one FP64
// partial sum per block.  It bounds the tiling to kNoAllocMaxBlocks blocks
// (sweep_plan.h).
constexpr size_t kCounterBytes = 256;
constexpr size_t kScratchBytes = kCounterBytes + (size_t)kNoAllocMaxBlocks * sizeof(double);

// Held by every GPU that loads the library, until the process exits.  In host
// code this name is only a host-side stand-in; the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_apply_scratch[kScratchBytes];

// The device address of g_apply_scratch in the current device's context.
// It is looked up on every call (a lookup, no allocation): the address
// belongs to the module loaded in the current context, and a host program
// that resets the device or re-creates its primary context gets the module
// loaded again, possibly at another address, so a cached address could be
// stale.
int scratch_address(unsigned char** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_apply_scratch) != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return TPFA_ECUDA;
  }
  *out = static_cast<unsigned char*>(p);
  return TPFA_OK;
}

}  // namespace

extern "C" int tpfa_apply_noalloc(const tpfa_grid* grid, const float* coef, const float* p,
                                  float* Ap, double* pAp, void* stream) {
  if (grid == nullptr) return TPFA_EINVAL;
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return TPFA_EINVAL;
  // geometry is not used by the operator application, but a grid that
  // tpfa_create would refuse is refused here too
  if (!(grid->dx > 0) || !(grid->dy > 0) || !(grid->dz > 0) || !(grid->mu > 0)) return TPFA_EINVAL;
  if (!isfinite(grid->dx) || !isfinite(grid->dy) || !isfinite(grid->dz) || !isfinite(grid->mu))
    return TPFA_EINVAL;
  if ((double)grid->nx * (double)grid->ny + 2.0 * (double)grid->nx > 2147483647.0) return TPFA_EINVAL;
  if ((double)grid->nx * (double)grid->ny * (double)grid->nz > 4.0e12) return TPFA_EINVAL;
  int device = -1, sms = 0;
  if (cudaGetDevice(&device) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    return TPFA_ECUDA;
  }
  Grid g;
  g.nx = grid->nx; g.ny = grid->ny; g.nz = grid->nz;
  g.plane = g.nx * g.ny;
  g.n = g.plane * g.nz;
  const size_t n = (size_t)g.n;
  if (!dev_ok(coef, n * 16, 16, device) || !dev_ok(p, n * 4, 4, device) ||
      !dev_ok(Ap, n * 4, 4, device) || !opt_dev_ok(pAp, 8, 8, device))
    return TPFA_EINVAL;
  if ((const void*)p == (const void*)Ap) return TPFA_EINVAL;
  // Same tiling as tpfa_apply, with longer z-runs if needed so that the
  // block count fits the fixed workspace; grids whose single z-run still
  // needs more blocks are refused.
  Sweep sw;
  if (!plan_noalloc(g, sms, &sw)) return TPFA_EINVAL;
  unsigned char* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc) return rc;
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch);
  double* partials = reinterpret_cast<double*>(scratch + kCounterBytes);
  cudaStream_t s = (cudaStream_t)stream;
  if (pAp != nullptr && cudaMemsetAsync(counter, 0, sizeof(unsigned int), s) != cudaSuccess) {
    cudaGetLastError();
    return TPFA_ECUDA;
  }
  if (launch_apply(g, sw, coef, false, p, Ap, pAp, partials, counter, s) != cudaSuccess) {
    cudaGetLastError();
    return TPFA_ECUDA;
  }
  return TPFA_OK;
}
