// Device helpers shared by the stencil-sweep kernels: compensated FP32
// accumulation, deterministic block and grid reductions, the 7-point product,
// the CG scalar update, and cp.async copies.
#pragma once

#include <math.h>

#include "tpfa_internal.cuh"

namespace tpfa {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Kahan-compensated FP32 accumulator: value = s - c.
struct Acc {
  float s, c;
};

__device__ __forceinline__ void kadd(Acc& a, float v) {
  const float y = __fsub_rn(v, a.c);
  const float t = __fadd_rn(a.s, y);
  a.c = __fsub_rn(__fsub_rn(t, a.s), y);
  a.s = t;
}

__device__ __forceinline__ double kval(const Acc& a) { return (double)a.s - (double)a.c; }

// Sum NV doubles over the block (fixed order) and store the block partial.
template <int NV>
__device__ __forceinline__ void block_partial(double (&v)[NV], double* partials) {
  __shared__ double sm[32][NV];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] += __shfl_down_sync(kFull, v[i], o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) sm[w][i] = v[i];
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    const int nw = blockDim.x >> 5;
    double s = 0.0;
    for (int ww = 0; ww < nw; ++ww) s += sm[ww][threadIdx.x];
    partials[(size_t)blockIdx.x * NV + threadIdx.x] = s;
  }
}

// Returns true in the last of `count` blocks (blocks first .. first+count-1
// of the grid, which share `counter`) to finish; that block then holds the
// fixed-order total of their partials in tot (every thread).
template <int NV>
__device__ __forceinline__ bool last_block_range(const double* partials, unsigned int* counter,
                                                 int64_t first, int64_t count,
                                                 double (&tot)[NV]) {
  __shared__ bool s_last;
  __shared__ double sm[32][NV];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == (unsigned)(count - 1));
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = 0.0;
#pragma unroll 8
  for (int64_t b = threadIdx.x; b < count; b += blockDim.x) {
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] += __ldcg(partials + (size_t)(first + b) * NV + i);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] += __shfl_down_sync(kFull, acc[i], o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) sm[w][i] = acc[i];
  }
  __syncthreads();
  const int nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double s = 0.0;
    for (int ww = 0; ww < nw; ++ww) s += sm[ww][i];
    tot[i] = s;
  }
  if (threadIdx.x == 0) *counter = 0u;  // ready for the next launch
  return true;
}

// The same over the whole grid.
template <int NV>
__device__ __forceinline__ bool last_block_total(const double* partials, unsigned int* counter,
                                                 double (&tot)[NV]) {
  return last_block_range<NV>(partials, counter, 0, gridDim.x, tot);
}

// 7-point product for one cell, fused multiply-adds in a fixed order.
__device__ __forceinline__ float stencil7(float4 c, float txm, float tym, float tzm, float pc,
                                          float pxp, float pxm, float pyp, float pym, float pzp,
                                          float pzm) {
  float q = c.w * pc;
  q = fmaf(-c.x, pxp, q);
  q = fmaf(-txm, pxm, q);
  q = fmaf(-c.y, pyp, q);
  q = fmaf(-tym, pym, q);
  q = fmaf(-c.z, pzp, q);
  q = fmaf(-tzm, pzm, q);
  return q;
}

// CG finish for iteration k (last block, thread 0).  rho = r_k'r_k,
// pq = p_k'q_k, rq = r_k'q_k, qq = q_k'q_k with q_k = A p_k.
//   alpha_k = rho / pq                                  (Alg. 1, line 5)
//   ||r_{k+1}||^2 = rho - 2 alpha rq + alpha^2 qq        (exact identity)
//   beta_k = ||r_{k+1}||^2 / rho                         (Alg. 1, line 9)
// so one reduction per iteration suffices.  The next sweep recomputes the
// true r_{k+1}'r_{k+1} from the stored vector.
__device__ void cg_finish(CgState* st, const double (&t)[4], unsigned long long cond,
                          bool use_cond) {
  const double rho = t[0], pq = t[1], rq = t[2], qq = t[3];
  const long long k = st->iter;
  if (k == 0) st->rho0 = rho;
  st->rho = rho;
  const double thresh = st->rtol2 * st->rho0;
  int done = kRunning;
  if (!isfinite(rho) || !isfinite(pq) || !isfinite(rq) || !isfinite(qq)) {
    done = kNonFinite;
    st->alpha_fin = 0.0;
  } else if (rho <= thresh) {
    done = kConvTrue;
    st->alpha_fin = 0.0;
  } else if (!(pq > 0.0)) {
    done = kBreakdown;
    st->alpha_fin = 0.0;
  } else {
    const double alpha = rho / pq;
    double rn = rho - 2.0 * alpha * rq + alpha * alpha * qq;
    if (rn < 0.0) rn = 0.0;
    st->rho_est = rn;
    st->iter = k + 1;
    if (rn <= thresh) {
      done = kConvEst;
      st->alpha_fin = alpha;
    } else if (k + 1 >= st->maxit) {
      done = kMaxit;
      st->alpha_fin = alpha;
    } else {
      st->alpha = alpha;
      st->beta = rn / rho;
    }
  }
  if (st->launches > st->guard_limit || st->fault) done = kGuard;
  st->parity ^= 1;
  st->done = done;
  if (use_cond) cudaGraphSetConditional(cond, done == kRunning ? 1u : 0u);
}

// ---- asynchronous global -> shared copies (cp.async, zero-filling) --------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
// copy 4 bytes, or write 4 zero bytes when !ok (nothing is read then)
__device__ __forceinline__ void cp4(void* dst, const void* src, bool ok) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
               "r"(ok ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp16(void* dst, const void* src, bool ok) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
               "r"(ok ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp8(void* dst, const void* src, bool ok) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
               "r"(ok ? 8 : 0)
               : "memory");
}
// Jacobi preconditioner M^-1 = diag(jac_inv(D)): one approximate reciprocal
// per cell.  Any fixed positive diagonal is a valid SPD preconditioner; what
// matters is that every kernel uses this same function of D, so z = M^-1 r
// and the M^-1-weighted dot products refer to one and the same M.
__device__ __forceinline__ float jac_inv(float D) { return D != 0.f ? __fdividef(1.0f, D) : 0.f; }

// BF16 halves of a 32-bit word as FP32 (exact)
__device__ __forceinline__ float bf16_lo(unsigned w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(unsigned w) { return __uint_as_float(w & 0xffff0000u); }
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

}  // namespace
}  // namespace tpfa
