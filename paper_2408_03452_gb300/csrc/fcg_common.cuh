// Pieces shared by the two flexible-CG solvers (fcg.cu: one grid; fcg_batch.cu:
// the instances of a batch): block reductions, the retained-direction table,
// the Jacobi diagonal, restriction to and prolongation from the network's
// coarser grid, and the solvers' constants.  Each translation unit gets its
// own copy (anonymous namespace).
#pragma once

#include <stdint.h>

#include "tpfa_internal.cuh"

struct tpfa_unet;
extern "C" int tpfa_unet_forward(tpfa_unet* u, const float* r, const float* lnk, float* z,
                                 void* stream);
extern "C" int tpfa_unet_forward_samples(tpfa_unet* u, int ns, const float* r, const float* lnk,
                                         float* z, void* stream);
extern "C" int tpfa_net_status(void* stream);
extern "C" int tpfa_unet_shape(const tpfa_unet* u, int* dims4);

namespace {

constexpr int kT = 256;

// Block sums of M per-thread FP64 values (warp shuffles, then the warps in
// order): part[slot * M + j].
template <int M>
__device__ __forceinline__ void block_sum_m(const double (&v)[M], double* part,
                                            int64_t slot) {
  __shared__ double sh[M][kT / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < M; ++j) {
    double x = v[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[j][wid] = x;
  }
  __syncthreads();
  if (threadIdx.x < M) {
    double t = 0.0;
    for (int w = 0; w < kT / 32; ++w) t += sh[threadIdx.x][w];
    part[(size_t)slot * M + threadIdx.x] = t;
  }
}
// ... into the slot of this block
template <int M>
__device__ __forceinline__ void block_sum_m(const double (&v)[M], double* part) {
  block_sum_m<M>(v, part, blockIdx.x);
}

constexpr int kMaxDirs = 16;
struct Dirs {
  const float* v[kMaxDirs];
};

// partial sums per block: the most any kernel writes (dots_kernel<kMaxDirs>)
constexpr int kPartPerBlock = 2 + 2 * kMaxDirs;

#define TPFA_FCG_M0(X) \
  X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16)

// dinv = 1 / D (the Jacobi scaling the blend uses)
__global__ void dinv_kernel(const float4* __restrict__ coef, float* __restrict__ dinv, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
    dinv[i] = 1.0f / coef[i].w;
}

// coarse[C] = scale * sum of the 8 children of C (fine grid nx x ny x nz, all
// even, ns samples in the solver's x-fastest order; sample s of the fine
// vector starts at soff[s] when soff is given (even offsets), else at s n).
// The coarse samples are stored qx x qy x qz (>= the coarse extents; 0: not
// padded); padding cells are not written.
__global__ void restrict2_kernel(const float* __restrict__ fine, float* __restrict__ coarse, int nx,
                                 int ny, int nz, int ns, float scale,
                                 const int64_t* __restrict__ soff, int qx, int qy, int qz) {
  const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
  const int px = qx > 0 ? qx : cx, py = qy > 0 ? qy : cy, pz = qz > 0 ? qz : cz;
  const int nc = cx * cy * cz * ns;  // grids with fewer than 2^31 cells
  for (int c = blockIdx.x * kT + threadIdx.x; c < nc; c += gridDim.x * kT) {
    const int i = c % cx;
    int t = c / cx;
    const int j = t % cy;
    t /= cy;
    const int k = t % cz;
    const int s = t / cz;
    const float* f = fine + (soff != nullptr ? (size_t)soff[s] : (size_t)s * nx * ny * nz);
    float acc = 0.f;
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        const float2 v = *reinterpret_cast<const float2*>(
            f + ((size_t)(2 * k + dz) * ny + 2 * j + dy) * nx + 2 * i);
        acc += v.x + v.y;
      }
    coarse[((size_t)(s * pz + k) * py + j) * px + i] = scale * acc;
  }
}

// fine[c] = coarse[parent(c)]; each thread writes two x-neighbours (same
// parent); sample s of the fine vector starts at soff[s] when soff is given
// (even offsets), else at s n; coarse samples stored qx x qy x qz as in
// restrict2_kernel (0: not padded)
__global__ void prolong2_kernel(const float* __restrict__ coarse, float* __restrict__ fine, int nx,
                                int ny, int nz, int ns, const int64_t* __restrict__ soff, int qx,
                                int qy, int qz) {
  const int cx = nx / 2;
  const int px = qx > 0 ? qx : cx, py = qy > 0 ? qy : ny / 2, pz = qz > 0 ? qz : nz / 2;
  const int per = nx / 2 * ny * nz;  // float2 pairs per sample
  const int n2 = per * ns;
  for (int c = blockIdx.x * kT + threadIdx.x; c < n2; c += gridDim.x * kT) {
    const int i = c % cx;
    int t = c / cx;
    const int j = t % ny;
    t /= ny;
    const int k = t % nz;
    const int s = t / nz;
    const float v = coarse[((size_t)(s * pz + k / 2) * py + j / 2) * px + i];
    float* f = fine + (soff != nullptr ? (size_t)soff[s] : (size_t)s * 2 * per);
    *reinterpret_cast<float2*>(f + 2 * (size_t)(c - s * per)) = make_float2(v, v);
  }
}

// Value of one cell of the 2^L coarser grid: the block mean over its 2^L
// children per axis, formed level by level in the order of L successive
// restrict2_kernel passes with scale 1/8.  Each level's product is rounded
// on its own (__fmul_rn, no contraction into a later add), so the result is
// bit-identical to those passes.  (x, y, z): the block's first fine cell.
template <int L>
__device__ __forceinline__ float block_mean(const float* __restrict__ f, int nx, int ny, int x,
                                            int y, int z) {
  float acc = 0.f;
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      if constexpr (L == 1) {
        const float2 v =
            *reinterpret_cast<const float2*>(f + ((size_t)(z + dz) * ny + y + dy) * nx + x);
        acc += v.x + v.y;
      } else {
        constexpr int h = 1 << (L - 1);
        const float a = block_mean<L - 1>(f, nx, ny, x, y + dy * h, z + dz * h);
        const float b = block_mean<L - 1>(f, nx, ny, x + h, y + dy * h, z + dz * h);
        acc += a + b;
      }
    }
  return __fmul_rn(0.125f, acc);
}

// The 2^L coarser grid in one pass (block means, as L restrict2_kernel passes
// with scale 1/8 would give them; fine extents divisible by 2^L).  Sample
// offsets and the padded coarse layout as in restrict2_kernel.
template <int L>
__global__ void restrict_levels_kernel(const float* __restrict__ fine, float* __restrict__ coarse,
                                       int nx, int ny, int nz, int ns,
                                       const int64_t* __restrict__ soff, int qx, int qy, int qz) {
  const int cx = nx >> L, cy = ny >> L, cz = nz >> L;
  const int px = qx > 0 ? qx : cx, py = qy > 0 ? qy : cy, pz = qz > 0 ? qz : cz;
  const int nc = cx * cy * cz * ns;  // grids with fewer than 2^31 cells
  for (int c = blockIdx.x * kT + threadIdx.x; c < nc; c += gridDim.x * kT) {
    const int i = c % cx;
    int t = c / cx;
    const int j = t % cy;
    t /= cy;
    const int k = t % cz;
    const int s = t / cz;
    const float* f = fine + (soff != nullptr ? (size_t)soff[s] : (size_t)s * nx * ny * nz);
    coarse[((size_t)(s * pz + k) * py + j) * px + i] = block_mean<L>(f, nx, ny, i << L, j << L, k << L);
  }
}

// fine[c] = coarse value of c's ancestor on the 2^L coarser grid (L nearest
// prolongations in one pass).  Blocks walk (sample, z) planes along y and the
// groups of V x-neighbours of one plane along x (no per-cell divisions); V = 4
// (one 16-byte store per thread) needs nx % 4 == 0 and sample starts on 16-byte
// boundaries, V = 2 an even nx and 8-byte boundaries.  Sample offsets and the
// padded coarse layout as in prolong2_kernel.
template <int L, int V>
__global__ void prolong_levels_kernel(const float* __restrict__ coarse, float* __restrict__ fine,
                                      int nx, int ny, int nz, int ns,
                                      const int64_t* __restrict__ soff, int qx, int qy, int qz) {
  const int px = qx > 0 ? qx : nx >> L, py = qy > 0 ? qy : ny >> L, pz = qz > 0 ? qz : nz >> L;
  const int gx = nx / V;         // groups per row
  const int per = gx * ny;       // groups per plane
  const int planes = nz * ns;
  for (int pl = blockIdx.y; pl < planes; pl += gridDim.y) {
    const int s = pl / nz, k = pl - s * nz;
    float* f = fine + (soff != nullptr ? (size_t)soff[s] : (size_t)s * nx * ny * nz) +
               (size_t)k * nx * ny;
    const float* c = coarse + (size_t)(s * pz + (k >> L)) * py * px;
    for (int t = blockIdx.x * kT + threadIdx.x; t < per; t += gridDim.x * kT) {
      const int j = t / gx, i = (t - j * gx) * V;
      const float* cr = c + (size_t)(j >> L) * px;
      const float v0 = cr[i >> L];
      if constexpr (V == 4) {
        const float v1 = L >= 2 ? v0 : cr[(i + 2) >> L];
        *reinterpret_cast<float4*>(f + (size_t)j * nx + i) = make_float4(v0, v0, v1, v1);
      } else {
        *reinterpret_cast<float2*>(f + (size_t)j * nx + i) = make_float2(v0, v0);
      }
    }
  }
}

// launchers for L = 1, 2, 3 (kMaxLevels)
inline void launch_restrict_levels(int L, int nb, cudaStream_t st, const float* fine, float* coarse,
                                   int nx, int ny, int nz, int ns, const int64_t* soff, int qx,
                                   int qy, int qz) {
  switch (L) {
    case 1: restrict_levels_kernel<1><<<nb, kT, 0, st>>>(fine, coarse, nx, ny, nz, ns, soff, qx, qy, qz); break;
    case 2: restrict_levels_kernel<2><<<nb, kT, 0, st>>>(fine, coarse, nx, ny, nz, ns, soff, qx, qy, qz); break;
    case 3: restrict_levels_kernel<3><<<nb, kT, 0, st>>>(fine, coarse, nx, ny, nz, ns, soff, qx, qy, qz); break;
    default: break;
  }
}
inline void launch_prolong_levels(int L, int nb, cudaStream_t st, const float* coarse, float* fine,
                                  int nx, int ny, int nz, int ns, const int64_t* soff, int qx,
                                  int qy, int qz, bool starts16 = false) {
  // starts16: every sample starts on a 16-byte boundary (with soff: offsets
  // that are multiples of 4 cells; without: a 16-byte aligned fine)
  const bool v4 = nx % 4 == 0 && starts16 && reinterpret_cast<uintptr_t>(fine) % 16 == 0;
  const int per = (nx / (v4 ? 4 : 2)) * ny;
  const int planes = nz * ns;
  int by = planes < 65535 ? planes : 65535;
  int bx = (per + kT - 1) / kT;
  const int cap = nb / by > 1 ? nb / by : 1;  // about nb blocks in all
  if (bx > cap) bx = cap;
  const dim3 grid((unsigned)bx, (unsigned)by);
#define TPFA_PROLONG(LL)                                                                        \
  if (v4) prolong_levels_kernel<LL, 4><<<grid, kT, 0, st>>>(coarse, fine, nx, ny, nz, ns, soff, qx, qy, qz); \
  else prolong_levels_kernel<LL, 2><<<grid, kT, 0, st>>>(coarse, fine, nx, ny, nz, ns, soff, qx, qy, qz);
  switch (L) {
    case 1: TPFA_PROLONG(1) break;
    case 2: TPFA_PROLONG(2) break;
    case 3: TPFA_PROLONG(3) break;
    default: break;
  }
#undef TPFA_PROLONG
}

// iterations between the host's looks at the device scalars (convergence,
// breakdown, stagnation); at most this many iterations run past the one that
// met the tolerance
constexpr int kCheckEvery = 4;
constexpr int kMaxLevels = 3;  // the network's grid: up to 8x coarser than the solver's

// stagnation window of the fallback test (iterations)
constexpr int kStallWindow = 100;

}  // namespace
