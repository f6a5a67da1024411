// Coefficient and right-hand-side construction (once per solve).
//
// Transmissibility (arXiv 2408.03452, Section II.A, Eq. 4): the flux across
// the face between cells K and L is T_KL (p_L - p_K) with T_KL = Y_KL *
// lambda_KL.  The geometric factor Y is the two-point (half-transmissibility)
// form A_f / (h/(2 k_K) + h/(2 k_L)), which is the harmonic mean of the two
// permeabilities for unit cells; lambda_KL = 1/mu, the arithmetic mean of the
// two (equal) mobilities.  Faces on the outer boundary carry no flow.
// Dirichlet cells (Eq. 3) keep the identity row; their couplings to interior
// cells move to the right-hand side.
#include <cuda_bf16.h>

#include "tpfa_internal.cuh"

namespace tpfa {

namespace {

struct Geo {
  double ax, ay, az;  // face area / mu for x, y, z faces
  double hx, hy, hz;  // cell size along each axis
};

__device__ __forceinline__ double face_trans(double kK, double kL, double a, double h) {
  const double half = 0.5 * h;
  return a / (half / kK + half / kL);
}

__device__ __forceinline__ bool is_dir(const uint8_t* m, int64_t c) { return m != nullptr && m[c] != 0; }

__global__ void __launch_bounds__(kElemThreads)
build_trans_kernel(Grid g, Geo geo, const double* __restrict__ K, const uint8_t* __restrict__ mask,
                   const double* __restrict__ d, double d0, float4* __restrict__ coef,
                   double2* __restrict__ coef64) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < g.n; c += stride) {
    const int64_t i = c % g.nx, j = (c / g.nx) % g.ny, k = c / g.plane;
    double t[3] = {0.0, 0.0, 0.0};
    double diag;
    if (is_dir(mask, c)) {
      diag = 1.0;
    } else {
      const double kc = K[c];
      diag = 0.0;
      // faces in the order -x, +x, -y, +y, -z, +z
      if (i > 0) diag += face_trans(K[c - 1], kc, geo.ax, geo.hx);
      if (i + 1 < g.nx) {
        const double T = face_trans(kc, K[c + 1], geo.ax, geo.hx);
        diag += T;
        if (!is_dir(mask, c + 1)) t[0] = T;
      }
      if (j > 0) diag += face_trans(K[c - g.nx], kc, geo.ay, geo.hy);
      if (j + 1 < g.ny) {
        const double T = face_trans(kc, K[c + g.nx], geo.ay, geo.hy);
        diag += T;
        if (!is_dir(mask, c + g.nx)) t[1] = T;
      }
      if (k > 0) diag += face_trans(K[c - g.plane], kc, geo.az, geo.hz);
      if (k + 1 < g.nz) {
        const double T = face_trans(kc, K[c + g.plane], geo.az, geo.hz);
        diag += T;
        if (!is_dir(mask, c + g.plane)) t[2] = T;
      }
      diag = diag + (d != nullptr ? d[c] : d0);
    }
    coef[c] = make_float4(__double2float_rn(t[0]), __double2float_rn(t[1]),
                          __double2float_rn(t[2]), __double2float_rn(diag));
    if (coef64 != nullptr) {
      coef64[2 * c] = make_double2(t[0], t[1]);
      coef64[2 * c + 1] = make_double2(t[2], diag);
    }
  }
}

// Compact BF16 record for the mixed-precision inner solve: (Tx', Ty', Tz', E),
// each rounded to nearest-even from FP64, with E = d_K + sum of the T_KL to
// Dirichlet neighbours (faces -x..+z in order; E = 1 and T' = 0 on Dirichlet
// cells).  The sweep forms D = sum of the six T' + E in FP32, so the BF16
// operator is the TPFA operator of the rounded face values: symmetric
// positive definite whenever the FP64 one is, with x'Ax within a factor
// (1 +- 2^-9) of the FP64 operator's.
__global__ void __launch_bounds__(kElemThreads)
build_trans_bf16_kernel(Grid g, Geo geo, const double* __restrict__ K,
                        const uint8_t* __restrict__ mask, const double* __restrict__ d, double d0,
                        ushort4* __restrict__ coef16) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < g.n; c += stride) {
    const int64_t i = c % g.nx, j = (c / g.nx) % g.ny, k = c / g.plane;
    double t[3] = {0.0, 0.0, 0.0};
    double e;
    if (is_dir(mask, c)) {
      e = 1.0;
    } else {
      const double kc = K[c];
      e = d != nullptr ? d[c] : d0;
      if (i > 0 && is_dir(mask, c - 1)) e += face_trans(K[c - 1], kc, geo.ax, geo.hx);
      if (i + 1 < g.nx) {
        const double T = face_trans(kc, K[c + 1], geo.ax, geo.hx);
        if (is_dir(mask, c + 1)) e += T; else t[0] = T;
      }
      if (j > 0 && is_dir(mask, c - g.nx)) e += face_trans(K[c - g.nx], kc, geo.ay, geo.hy);
      if (j + 1 < g.ny) {
        const double T = face_trans(kc, K[c + g.nx], geo.ay, geo.hy);
        if (is_dir(mask, c + g.nx)) e += T; else t[1] = T;
      }
      if (k > 0 && is_dir(mask, c - g.plane)) e += face_trans(K[c - g.plane], kc, geo.az, geo.hz);
      if (k + 1 < g.nz) {
        const double T = face_trans(kc, K[c + g.plane], geo.az, geo.hz);
        if (is_dir(mask, c + g.plane)) e += T; else t[2] = T;
      }
    }
    coef16[c] = make_ushort4(__bfloat16_as_ushort(__double2bfloat16(t[0])),
                             __bfloat16_as_ushort(__double2bfloat16(t[1])),
                             __bfloat16_as_ushort(__double2bfloat16(t[2])),
                             __bfloat16_as_ushort(__double2bfloat16(e)));
  }
}

__global__ void __launch_bounds__(kElemThreads)
build_rhs_kernel(Grid g, Geo geo, const double* __restrict__ K, const uint8_t* __restrict__ mask,
                 const double* __restrict__ q, const double* __restrict__ pD,
                 double* __restrict__ b) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < g.n; c += stride) {
    if (is_dir(mask, c)) {
      b[c] = pD != nullptr ? pD[c] : 0.0;
      continue;
    }
    double s = q != nullptr ? q[c] : 0.0;
    if (mask != nullptr) {
      const int64_t i = c % g.nx, j = (c / g.nx) % g.ny, k = c / g.plane;
      const double kc = K[c];
      // lifted couplings to Dirichlet neighbours, faces -x, +x, -y, +y, -z, +z
      const int64_t nb[6] = {c - 1, c + 1, c - g.nx, c + g.nx, c - g.plane, c + g.plane};
      const bool ex[6] = {i > 0, i + 1 < g.nx, j > 0, j + 1 < g.ny, k > 0, k + 1 < g.nz};
      const double ar[3] = {geo.ax, geo.ay, geo.az}, hh[3] = {geo.hx, geo.hy, geo.hz};
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        if (!ex[f] || !is_dir(mask, nb[f])) continue;
        const double T = (f & 1) ? face_trans(kc, K[nb[f]], ar[f >> 1], hh[f >> 1])
                                 : face_trans(K[nb[f]], kc, ar[f >> 1], hh[f >> 1]);
        s += T * (pD != nullptr ? pD[nb[f]] : 0.0);
      }
    }
    b[c] = s;
  }
}

// Point sources, added one after another by a single thread so that
// duplicates accumulate in a fixed order.  Sources on Dirichlet cells and
// indices outside the grid are ignored.
__global__ void add_sources_kernel(Grid g, const uint8_t* __restrict__ mask,
                                   const int64_t* __restrict__ idx, const double* __restrict__ val,
                                   int64_t n, double* __restrict__ b) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int64_t t = 0; t < n; ++t) {
    const int64_t c = idx[t];
    if (c < 0 || c >= g.n || is_dir(mask, c)) continue;
    b[c] += val[t];
  }
}

// Known part of the accumulation term of one backward-Euler step:
// b_K += d_K p_K^n on interior cells.
__global__ void __launch_bounds__(kElemThreads)
accumulation_kernel(Grid g, const uint8_t* __restrict__ mask, const double* __restrict__ d,
                    double d0, const double* __restrict__ p_prev, double* __restrict__ b) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < g.n; c += stride)
    if (!is_dir(mask, c)) b[c] += (d != nullptr ? d[c] : d0) * p_prev[c];
}

Geo make_geo(const tpfa_grid& geo) {
  Geo o;
  o.ax = (geo.dy * geo.dz) / geo.mu;
  o.ay = (geo.dx * geo.dz) / geo.mu;
  o.az = (geo.dx * geo.dy) / geo.mu;
  o.hx = geo.dx; o.hy = geo.dy; o.hz = geo.dz;
  return o;
}

int grid_for(const Grid& g) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return elem_blocks(g, sms);
}

}  // namespace

cudaError_t launch_build_trans(const Grid& g, const tpfa_grid& geo, const double* K,
                               const uint8_t* mask, const double* d, double d0, float4* coef,
                               double* coef64, cudaStream_t s) {
  build_trans_kernel<<<grid_for(g), kElemThreads, 0, s>>>(g, make_geo(geo), K, mask, d, d0, coef,
                                                          reinterpret_cast<double2*>(coef64));
  return cudaGetLastError();
}

cudaError_t launch_accumulation(const Grid& g, const uint8_t* mask, const double* d, double d0,
                                const double* p_prev, double* b, cudaStream_t s) {
  accumulation_kernel<<<grid_for(g), kElemThreads, 0, s>>>(g, mask, d, d0, p_prev, b);
  return cudaGetLastError();
}

cudaError_t launch_build_trans_bf16(const Grid& g, const tpfa_grid& geo, const double* K,
                                    const uint8_t* mask, const double* d, double d0,
                                    uint2* coef16, cudaStream_t s) {
  build_trans_bf16_kernel<<<grid_for(g), kElemThreads, 0, s>>>(
      g, make_geo(geo), K, mask, d, d0, reinterpret_cast<ushort4*>(coef16));
  return cudaGetLastError();
}

cudaError_t launch_build_rhs(const Grid& g, const tpfa_grid& geo, const double* K,
                             const uint8_t* mask, const double* q, const double* pD,
                             const int64_t* src_idx, const double* src_val, int64_t n_src,
                             double* b, cudaStream_t s) {
  build_rhs_kernel<<<grid_for(g), kElemThreads, 0, s>>>(g, make_geo(geo), K, mask, q, pD, b);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || n_src <= 0) return e;
  add_sources_kernel<<<1, 32, 0, s>>>(g, mask, src_idx, src_val, n_src, b);
  return cudaGetLastError();
}

}  // namespace tpfa
