// Flexible conjugate gradients (Notay 2000, m retained directions) with the
// learned U-Net preconditioner, and the gradient of the training loss.
//
// Preconditioner with a network: z = D^-1 r + c u, u = net(r), with the
// A-norm-optimal weight c = (u'r - (Au)'D^-1 r) / (u'Au) (one extra operator
// application), so that each application is at least as good as one Jacobi
// step in the A-norm.
//
// Outer loop (FP64): r = b - A x with the FP64 coefficient records; stop when
// ||r|| <= tol ||b||; otherwise solve A e = r / ||r|| in FP32 by FCG and add
// e ||r|| to x.  Inner FCG:
//   z_k = M(r_k);  p_k = z_k - sum_{j=1..m} (z_k' q_{k-j} / p_{k-j}' q_{k-j}) p_{k-j};
//   q_k = A p_k;  alpha_k = p_k' r_k / p_k' q_k;  e += alpha_k p_k;  r -= alpha_k q_k.
// For a fixed SPD preconditioner this generates the PCG iterates (the extra
// coefficients vanish in exact arithmetic); for the network, which is neither
// linear nor symmetric, the explicit A-orthogonalisation against the last m
// directions keeps much of the Krylov optimality that a single retained
// direction loses.  If p'q <= 0, a value is not finite, or the residual stops
// decreasing, the solve drops the network (Jacobi or the identity) from the
// current iterate.
//
// Dot products: FP32 per-thread sums over a few dozen cells, FP64 block
// partials in a fixed order, added in a fixed order by one-block finish
// kernels that also form the iteration's scalars on the device
// (bit-reproducible; the host reads the r'r history every few iterations).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "batch_internal.cuh"

struct tpfa_unet;
extern "C" int tpfa_unet_forward(tpfa_unet* u, const float* r, const float* lnk, float* z,
                                 void* stream);
extern "C" int tpfa_unet_forward_samples(tpfa_unet* u, int ns, const float* r, const float* lnk,
                                         float* z, void* stream);
extern "C" int tpfa_net_status(void* stream);
extern "C" int tpfa_unet_shape(const tpfa_unet* u, int* dims4);

namespace {

constexpr int kT = 256;

__device__ __forceinline__ void block_sum3(double a, double b, double c, double* out3) {
  __shared__ double sh[3][kT];
  sh[0][threadIdx.x] = a;
  sh[1][threadIdx.x] = b;
  sh[2][threadIdx.x] = c;
  __syncthreads();
  for (int w = kT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
      sh[2][threadIdx.x] += sh[2][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out3[3 * blockIdx.x] = sh[0][0];
    out3[3 * blockIdx.x + 1] = sh[1][0];
    out3[3 * blockIdx.x + 2] = sh[2][0];
  }
}

// r32 = r64 * scale, e = 0; partial r'r
__global__ void start_kernel(const double* __restrict__ r64, double scale, float* __restrict__ r,
                             float* __restrict__ e, int64_t n, double* part) {
  double rr = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
    const float v = (float)(r64[i] * scale);
    r[i] = v;
    e[i] = 0.f;
    rr += (double)v * v;
  }
  block_sum3(rr, 0.0, 0.0, part);
}

// x += e / scale
__global__ void correct_kernel(double* __restrict__ x, const float* __restrict__ e, double inv_scale,
                               int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
    x[i] += inv_scale * (double)e[i];
}

// Block sums of M per-thread FP64 values (warp shuffles, then the warps in
// order): part[blockIdx.x * M + j].
template <int M>
__device__ __forceinline__ void block_sum_m(const double (&v)[M], double* part) {
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
    part[(size_t)blockIdx.x * M + threadIdx.x] = t;
  }
}

constexpr int kMaxDirs = 16;
struct Dirs {
  const float* v[kMaxDirs];
};

// Device-resident scalars of the inner iteration: written by one-block finish
// kernels from fixed-order partial sums, read by the vector kernels, so the
// host need not take part in an iteration.
struct Scal {
  double c;                // blend weight of the current preconditioned residual
  double beta[kMaxDirs];   // coefficients against the retained directions, newest first
  double pq[kMaxDirs];     // p_j'q_j by ring slot
  double alpha;
  double pr;
  int bad;                 // p'q <= 0 or a non-finite value since the host last looked
  int pad;
};

// One pass for the preconditioned residual z = w + c u (w = r / D with Jacobi,
// else r; u the network term when net) and its A-orthogonalisation against M
// retained directions q_j = A p_j:
//   s0 = u'r, s1 = (Au)'w, a_j = w'q_j, b_j = u'q_j   (z'q_j = a_j + c b_j).
template <int M>
__global__ void dots_kernel(const float* __restrict__ r, const float* __restrict__ dinv,
                            const float* __restrict__ u, const float* __restrict__ au, Dirs qd,
                            int jac, int net, int64_t n, double* part) {
  // FP32 sums per thread (about a hundred terms each), FP64 across threads
  // and blocks: FP64 arithmetic per element would cost more than the memory.
  // Four elements per step (float4), a scalar tail for n % 4.
  constexpr int K = 2 + 2 * M;
  float s[K];
#pragma unroll
  for (int j = 0; j < K; ++j) s[j] = 0.f;
  auto one = [&](float ri, float di, float ui, float aui, const float* qv) {
    const float wi = jac ? ri * di : ri;
    if (net) {
      s[0] = fmaf(ui, ri, s[0]);
      s[1] = fmaf(aui, wi, s[1]);
    }
#pragma unroll
    for (int j = 0; j < M; ++j) {
      s[2 + j] = fmaf(wi, qv[j], s[2 + j]);
      s[2 + M + j] = fmaf(ui, qv[j], s[2 + M + j]);
    }
  };
  const int64_t n4 = n / 4;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n4; i += (int64_t)gridDim.x * kT) {
    const float4 r4 = reinterpret_cast<const float4*>(r)[i];
    const float4 d4 = jac ? reinterpret_cast<const float4*>(dinv)[i] : z4;
    const float4 u4 = net ? reinterpret_cast<const float4*>(u)[i] : z4;
    const float4 a4 = net ? reinterpret_cast<const float4*>(au)[i] : z4;
    float4 q4[M > 0 ? M : 1];
#pragma unroll
    for (int j = 0; j < M; ++j) q4[j] = reinterpret_cast<const float4*>(qd.v[j])[i];
    float qv[M > 0 ? M : 1];
#pragma unroll
    for (int j = 0; j < M; ++j) qv[j] = q4[j].x;
    one(r4.x, d4.x, u4.x, a4.x, qv);
#pragma unroll
    for (int j = 0; j < M; ++j) qv[j] = q4[j].y;
    one(r4.y, d4.y, u4.y, a4.y, qv);
#pragma unroll
    for (int j = 0; j < M; ++j) qv[j] = q4[j].z;
    one(r4.z, d4.z, u4.z, a4.z, qv);
#pragma unroll
    for (int j = 0; j < M; ++j) qv[j] = q4[j].w;
    one(r4.w, d4.w, u4.w, a4.w, qv);
  }
  for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * kT + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kT) {
    float qv[M > 0 ? M : 1];
#pragma unroll
    for (int j = 0; j < M; ++j) qv[j] = qd.v[j][i];
    one(r[i], jac ? dinv[i] : 0.f, net ? u[i] : 0.f, net ? au[i] : 0.f, qv);
  }
  double d[K];
#pragma unroll
  for (int j = 0; j < K; ++j) d[j] = s[j];
  block_sum_m<K>(d, part);
}

// c = (u'r - (Au)'w) / u'Au (0 without network, or when u'Au is not positive)
// and beta_j = -(a_j + c b_j) / (p_j'q_j) for the M retained directions
__global__ void finish_dots_kernel(const double* __restrict__ part, int nb, int M, int net,
                                   const double* __restrict__ uau, Scal* sc, int head, int m) {
  __shared__ double tot[2 + 2 * kMaxDirs];
  const int K = 2 + 2 * M;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int k = warp; k < K; k += nw) {
    double t = 0.0;
    for (int b = lane; b < nb; b += 32) t += part[(size_t)b * K + k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) tot[k] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double c = 0.0;
    if (net && nb > 0) {
      const double d = *uau;
      c = (d > 0.0 && isfinite(d)) ? (tot[0] - tot[1]) / d : 0.0;
      if (!isfinite(c)) c = 0.0;
    }
    sc->c = c;
    for (int j = 0; j < M; ++j) {
      const int slot = (head - 1 - j + m) % m;
      double b = -(tot[2 + j] + c * tot[2 + M + j]) / sc->pq[slot];
      if (!isfinite(b)) {
        sc->bad = 1;
        b = 0.0;
      }
      sc->beta[j] = b;
    }
  }
}

// p = w + c u + sum_j beta_j p_j; partial p'r (four elements per step)
template <int M>
__global__ void dir_kernel(const float* __restrict__ r, const float* __restrict__ dinv,
                           const float* __restrict__ u, Dirs pd, const Scal* __restrict__ sc,
                           int jac, int net, float* p, int64_t n, double* part) {
  // p may be the oldest retained direction (read, then overwritten, per element)
  const float c = (float)sc->c;
  float beta[M > 0 ? M : 1];
#pragma unroll
  for (int j = 0; j < M; ++j) beta[j] = (float)sc->beta[j];
  float prf = 0.f;
  auto one = [&](float ri, float di, float ui, const float* pv) {
    float v = jac ? ri * di : ri;
    if (net) v = fmaf(c, ui, v);
#pragma unroll
    for (int j = 0; j < M; ++j) v = fmaf(beta[j], pv[j], v);
    prf = fmaf(v, ri, prf);
    return v;
  };
  const int64_t n4 = n / 4;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n4; i += (int64_t)gridDim.x * kT) {
    const float4 r4 = reinterpret_cast<const float4*>(r)[i];
    const float4 d4 = jac ? reinterpret_cast<const float4*>(dinv)[i] : z4;
    const float4 u4 = net ? reinterpret_cast<const float4*>(u)[i] : z4;
    float4 p4[M > 0 ? M : 1];
#pragma unroll
    for (int j = 0; j < M; ++j) p4[j] = reinterpret_cast<const float4*>(pd.v[j])[i];
    float pv[M > 0 ? M : 1];
    float4 o;
#pragma unroll
    for (int j = 0; j < M; ++j) pv[j] = p4[j].x;
    o.x = one(r4.x, d4.x, u4.x, pv);
#pragma unroll
    for (int j = 0; j < M; ++j) pv[j] = p4[j].y;
    o.y = one(r4.y, d4.y, u4.y, pv);
#pragma unroll
    for (int j = 0; j < M; ++j) pv[j] = p4[j].z;
    o.z = one(r4.z, d4.z, u4.z, pv);
#pragma unroll
    for (int j = 0; j < M; ++j) pv[j] = p4[j].w;
    o.w = one(r4.w, d4.w, u4.w, pv);
    reinterpret_cast<float4*>(p)[i] = o;
  }
  for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * kT + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kT) {
    float pv[M > 0 ? M : 1];
#pragma unroll
    for (int j = 0; j < M; ++j) pv[j] = pd.v[j][i];
    p[i] = one(r[i], jac ? dinv[i] : 0.f, net ? u[i] : 0.f, pv);
  }
  double pr[1] = {prf};
  block_sum_m<1>(pr, part);
}

// fixed-order sum of nb block partials by one block of kT threads
__device__ __forceinline__ double block_total(const double* __restrict__ part, int nb) {
  __shared__ double sh[kT];
  double t = 0.0;
  for (int b = threadIdx.x; b < nb; b += kT) t += part[b];
  sh[threadIdx.x] = t;
  __syncthreads();
  for (int w = kT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  return sh[0];
}

// alpha = p'r / p'q (0 and the bad flag when p'q is not positive or a value
// is not finite); records p'q of the new direction in its slot
__global__ void finish_alpha_kernel(const double* __restrict__ part, int nb,
                                    const double* __restrict__ pq_dev, Scal* sc, int head) {
  const double pr = block_total(part, nb);
  if (threadIdx.x == 0) {
    const double pq = *pq_dev;
    sc->pr = pr;
    if (!(pq > 0.0) || !isfinite(pq) || !isfinite(pr)) {
      sc->bad = 1;
      sc->alpha = 0.0;
      sc->pq[head] = 1.0;
    } else {
      sc->alpha = pr / pq;
      sc->pq[head] = pq;
    }
  }
}

// e += alpha p; r -= alpha q; partial r'r (four elements per step)
__global__ void update_kernel(float* __restrict__ e, float* __restrict__ r,
                              const float* __restrict__ p, const float* __restrict__ q,
                              const Scal* __restrict__ sc, int64_t n, double* part) {
  const float alpha = (float)sc->alpha;
  float rrf = 0.f;
  const int64_t n4 = n / 4;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n4; i += (int64_t)gridDim.x * kT) {
    float4 e4 = reinterpret_cast<float4*>(e)[i];
    float4 r4 = reinterpret_cast<float4*>(r)[i];
    const float4 p4 = reinterpret_cast<const float4*>(p)[i];
    const float4 q4 = reinterpret_cast<const float4*>(q)[i];
    e4.x = fmaf(alpha, p4.x, e4.x);
    e4.y = fmaf(alpha, p4.y, e4.y);
    e4.z = fmaf(alpha, p4.z, e4.z);
    e4.w = fmaf(alpha, p4.w, e4.w);
    r4.x = fmaf(-alpha, q4.x, r4.x);
    r4.y = fmaf(-alpha, q4.y, r4.y);
    r4.z = fmaf(-alpha, q4.z, r4.z);
    r4.w = fmaf(-alpha, q4.w, r4.w);
    reinterpret_cast<float4*>(e)[i] = e4;
    reinterpret_cast<float4*>(r)[i] = r4;
    rrf = fmaf(r4.x, r4.x, rrf);
    rrf = fmaf(r4.y, r4.y, rrf);
    rrf = fmaf(r4.z, r4.z, rrf);
    rrf = fmaf(r4.w, r4.w, rrf);
  }
  for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * kT + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kT) {
    e[i] = fmaf(alpha, p[i], e[i]);
    const float v = fmaf(-alpha, q[i], r[i]);
    r[i] = v;
    rrf = fmaf(v, v, rrf);
  }
  double rr[1] = {rrf};
  block_sum_m<1>(rr, part);
}

// r'r of this iteration into its history slot
__global__ void finish_rr_kernel(const double* __restrict__ part, int nb, double* slot) {
  const double rr = block_total(part, nb);
  if (threadIdx.x == 0) *slot = rr;
}

// partial sums per block: the most any kernel writes (dots_kernel<kMaxDirs>)
constexpr int kPartPerBlock = 2 + 2 * kMaxDirs;

#define TPFA_FCG_M0(X) \
  X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16)

void launch_dots(int m, int nb, cudaStream_t s, const float* r, const float* coef, const float* u,
                 const float* au, const Dirs& qd, int jac, int net, int64_t n, double* part) {
  switch (m) {
#define X(M) \
  case M: dots_kernel<M><<<nb, kT, 0, s>>>(r, coef, u, au, qd, jac, net, n, part); break;
    TPFA_FCG_M0(X)
#undef X
    default: break;
  }
}

void launch_dir(int m, int nb, cudaStream_t s, const float* r, const float* coef, const float* u,
                const Dirs& pd, const Scal* sc, int jac, int net, float* p, int64_t n,
                double* part) {
  switch (m) {
#define X(M) \
  case M: dir_kernel<M><<<nb, kT, 0, s>>>(r, coef, u, pd, sc, jac, net, p, n, part); break;
    TPFA_FCG_M0(X)
#undef X
    default: break;
  }
}

// dinv = 1 / D (the Jacobi scaling the blend uses)
__global__ void dinv_kernel(const float4* __restrict__ coef, float* __restrict__ dinv, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
    dinv[i] = 1.0f / coef[i].w;
}

// y = x / D
__global__ void jacobi_kernel(const float* __restrict__ x, const float4* __restrict__ coef,
                              float* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
    y[i] = x[i] / coef[i].w;
}

// y = a - b (y may alias b)
__global__ void sub_kernel(const float* a, const float* b, float* y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
    y[i] = a[i] - b[i];
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

// partial a'b per block (fixed order); finish: out = sum of partials in block order
__global__ void dot_partial_kernel(const float* __restrict__ a, const float* __restrict__ b,
                                   int64_t n, double* part) {
  __shared__ double sh[kT];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
    s += (double)a[i] * b[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = kT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void dot_finish_kernel(const double* part, int nb, double* out) {
  double s = 0.0;
  for (int i = 0; i < nb; ++i) s += part[i];
  *out = s;
}

// g = (2 a / (b c)) ((a / b) q - r) with a = stats[0], b = stats[1], c = *eae
__global__ void loss_grad_kernel(const float* __restrict__ q, const float* __restrict__ r,
                                 const double* __restrict__ stats, const double* __restrict__ eae,
                                 float* __restrict__ g, int64_t n) {
  const double a = stats[0], b = stats[1], c = *eae;
  const float f = (float)(2.0 * a / (b * c));
  const float ab = (float)(a / b);
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
    g[i] = f * fmaf(ab, q[i], -r[i]);
}

// iterations between the host's looks at the device scalars (convergence,
// breakdown, stagnation); at most this many iterations run past the one that
// met the tolerance
constexpr int kCheckEvery = 4;
constexpr int kMaxLevels = 3;  // the network's grid: up to 8x coarser than the solver's

struct Work {
  cudaStream_t s = nullptr;
  int nb = 0;
  int64_t n = 0;
  int m = 1;                 // retained directions
  float *r = nullptr, *z = nullptr, *e = nullptr, *au = nullptr, *dinv = nullptr;
  float *P = nullptr, *Q = nullptr;  // m directions and their images A p
  double* r64 = nullptr;
  double* uau = nullptr;     // dev, 1
  double* part = nullptr;    // dev, kPartPerBlock * nb
  double* hpart = nullptr;   // pinned host
  double* norms = nullptr;   // dev, 2
  double* hnorms = nullptr;  // pinned
  double* pq = nullptr;      // dev, 1
  Scal* sc = nullptr;        // dev, iteration scalars
  double* hist = nullptr;    // dev, r'r of the iterations since the host last looked
  double* hhist = nullptr;   // pinned copy
  // network on the 2^levels coarser grid: restricted residuals and images per
  // level (level 0 is the solver's grid: r and z), ln K on the network's grid
  int levels = 0;
  int dims[3] = {0, 0, 0};
  float* rl[kMaxLevels + 1] = {};
  float* ul[kMaxLevels + 1] = {};
  float* lnkc = nullptr;
  int64_t launches = 0;

  // distance between retained directions: n rounded up to 4 floats, so that
  // every slot starts on a 16-byte boundary (the vector kernels read float4)
  int64_t slot_stride() const { return (n + 3) / 4 * 4; }

  bool alloc() {
    return cudaMalloc(&r, n * 4) == cudaSuccess && cudaMalloc(&z, n * 4) == cudaSuccess &&
           cudaMalloc(&P, (size_t)m * slot_stride() * 4) == cudaSuccess &&
           cudaMalloc(&Q, (size_t)m * slot_stride() * 4) == cudaSuccess &&
           cudaMalloc(&e, n * 4) == cudaSuccess && cudaMalloc(&r64, n * 8) == cudaSuccess &&
           cudaMalloc(&au, n * 4) == cudaSuccess && cudaMalloc(&uau, 8) == cudaSuccess &&
           cudaMalloc(&dinv, n * 4) == cudaSuccess &&
           cudaMalloc(&part, sizeof(double) * kPartPerBlock * nb) == cudaSuccess &&
           cudaMalloc(&norms, 16) == cudaSuccess && cudaMalloc(&pq, 8) == cudaSuccess &&
           cudaMallocHost(&hpart, sizeof(double) * kPartPerBlock * nb) == cudaSuccess &&
           cudaMallocHost(&hnorms, 16) == cudaSuccess &&
           cudaMalloc(&sc, sizeof(Scal)) == cudaSuccess &&
           cudaMalloc(&hist, sizeof(double) * kCheckEvery) == cudaSuccess &&
           cudaMallocHost(&hhist, sizeof(double) * kCheckEvery) == cudaSuccess &&
           cudaMemset(sc, 0, sizeof(Scal)) == cudaSuccess;
  }
  ~Work() {
    if (s) cudaStreamSynchronize(s);
    cudaFree(r);
    cudaFree(z);
    cudaFree(P);
    cudaFree(Q);
    cudaFree(e);
    cudaFree(au);
    cudaFree(dinv);
    cudaFree(uau);
    cudaFree(r64);
    cudaFree(part);
    cudaFree(norms);
    cudaFree(pq);
    cudaFreeHost(hpart);
    cudaFreeHost(hnorms);
    for (int l = 1; l <= kMaxLevels; ++l) {
      cudaFree(rl[l]);
      cudaFree(ul[l]);
    }
    cudaFree(lnkc);
    cudaFree(sc);
    cudaFree(hist);
    cudaFreeHost(hhist);
  }
  // sums of the three per-block partials, in block order
  bool fetch(double* out3) {
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(hpart, part, sizeof(double) * 3 * nb, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return false;
    out3[0] = out3[1] = out3[2] = 0.0;
    for (int b = 0; b < nb; ++b)
      for (int k = 0; k < 3; ++k) out3[k] += hpart[3 * b + k];
    return true;
  }
};

struct Result {
  int64_t iters = 0;
  int outer = 0;
  double rel = INFINITY, inner_ms = 0.0;
  bool fallback = false;
  int status = TPFA_NOTCONV;
};

enum PrecMode { kIdentity = 0, kJacobi = 1, kBlend = 2 };

// the network term u of the blend (into w.z) and A u (into w.au, u'Au into w.uau)
int network_term(tpfa_ctx* c, tpfa_unet* net, const float* coef, const float* lnk, Work& w) {
  int rc;
  if (w.levels > 0) {
    w.rl[0] = w.r;
    w.ul[0] = w.z;
    for (int l = 1; l <= w.levels; ++l)
      restrict2_kernel<<<w.nb, kT, 0, w.s>>>(w.rl[l - 1], w.rl[l], w.dims[0] >> (l - 1),
                                             w.dims[1] >> (l - 1), w.dims[2] >> (l - 1), 1, 0.125f,
                                             nullptr, 0, 0, 0);
    rc = tpfa_unet_forward(net, w.rl[w.levels], w.lnkc, w.ul[w.levels], w.s);
    if (rc) return rc;
    for (int l = w.levels; l >= 1; --l)
      prolong2_kernel<<<w.nb, kT, 0, w.s>>>(w.ul[l], w.ul[l - 1], w.dims[0] >> (l - 1),
                                            w.dims[1] >> (l - 1), w.dims[2] >> (l - 1), 1, nullptr,
                                            0, 0, 0);
    w.launches += 15 + 2 * w.levels;
  } else {
    rc = tpfa_unet_forward(net, w.r, lnk, w.z, w.s);
    if (rc) return rc;
    w.launches += 15;
  }
  rc = tpfa_apply(c, coef, w.z, w.au, w.uau, w.s);
  ++w.launches;
  return rc;
}

constexpr int kStallWindow = 100;

// Inner FCG on A e = r (r, e already set, r'r = rr0).  All scalars stay on the
// device; every kCheckEvery iterations the host reads the r'r history and the
// bad flag.  Returns a TPFA_* error or TPFA_OK, with res->status =
// TPFA_EBREAKDOWN if the method without network broke down.
int fcg_inner(tpfa_ctx* c, tpfa_unet* net, const float* coef, const float* lnk, Work& w,
              double rr0, double target, int64_t maxit, PrecMode fallback_mode, Result* res) {
  const int m = w.m;
  double rr = rr0;
  int stored = 0, head = 0, pending = 0;
  PrecMode mode = net == nullptr ? kIdentity : (res->fallback ? fallback_mode : kBlend);
  std::vector<double> hist(1, rr);
  if (cudaMemsetAsync(w.sc, 0, sizeof(Scal), w.s) != cudaSuccess) return TPFA_ECUDA;
  while (res->iters < maxit && rr > target * target * rr0) {
    const int jac = mode != kIdentity, with_net = mode == kBlend;
    if (with_net) {
      const int rc = network_term(c, net, coef, lnk, w);
      if (rc) return rc;
    }
    Dirs qd, pd;
    for (int j = 0; j < stored; ++j) {
      const size_t slot = (size_t)((head - 1 - j + m) % m);
      qd.v[j] = w.Q + slot * w.slot_stride();
      pd.v[j] = w.P + slot * w.slot_stride();
    }
    if (stored > 0 || with_net) {
      launch_dots(stored, w.nb, w.s, w.r, w.dinv, w.z, w.au, qd, jac, with_net, w.n, w.part);
      finish_dots_kernel<<<1, kT, 0, w.s>>>(w.part, w.nb, stored, with_net, w.uau, w.sc, head, m);
    } else {
      finish_dots_kernel<<<1, kT, 0, w.s>>>(w.part, 0, 0, 0, w.uau, w.sc, head, m);
    }
    float* p = w.P + (size_t)head * w.slot_stride();
    float* q = w.Q + (size_t)head * w.slot_stride();
    launch_dir(stored, w.nb, w.s, w.r, w.dinv, w.z, pd, w.sc, jac, with_net, p, w.n, w.part);
    int rc = tpfa_apply(c, coef, p, q, w.pq, w.s);
    if (rc) return rc;
    finish_alpha_kernel<<<1, kT, 0, w.s>>>(w.part, w.nb, w.pq, w.sc, head);
    update_kernel<<<w.nb, kT, 0, w.s>>>(w.e, w.r, p, q, w.sc, w.n, w.part);
    finish_rr_kernel<<<1, kT, 0, w.s>>>(w.part, w.nb, w.hist + pending);
    w.launches += 7;
    ++pending;
    ++res->iters;
    head = (head + 1) % m;
    if (stored < m) ++stored;
    if (pending < kCheckEvery && res->iters < maxit) continue;
    // the host looks: r'r history, bad flag
    int bad = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(w.hhist, w.hist, sizeof(double) * pending, cudaMemcpyDeviceToHost,
                        w.s) != cudaSuccess ||
        cudaMemcpyAsync(&bad, &w.sc->bad, sizeof(int), cudaMemcpyDeviceToHost, w.s) !=
            cudaSuccess ||
        cudaStreamSynchronize(w.s) != cudaSuccess)
      return TPFA_ECUDA;
    for (int k = 0; k < pending; ++k) hist.push_back(w.hhist[k]);
    rr = w.hhist[pending - 1];
    pending = 0;
    if (!std::isfinite(rr)) bad = 1;
    // stagnation: the smallest r'r of the last kStallWindow iterations is not
    // 1% below the smallest before them
    bool stalled = false;
    if (mode == kBlend && (int)hist.size() > 2 * kStallWindow) {
      const size_t cut = hist.size() - kStallWindow;
      const double before = *std::min_element(hist.begin(), hist.begin() + cut);
      const double recent = *std::min_element(hist.begin() + cut, hist.end());
      stalled = recent > 0.99 * before;
    }
    if (bad || stalled) {
      if (mode != kBlend) {
        res->status = TPFA_EBREAKDOWN;
        return TPFA_OK;
      }
      mode = fallback_mode;
      res->fallback = true;
      stored = 0;
      hist.assign(1, rr);
      if (cudaMemsetAsync(w.sc, 0, sizeof(Scal), w.s) != cudaSuccess) return TPFA_ECUDA;
    }
  }
  return TPFA_OK;
}

int fcg_outer(tpfa_ctx* c, tpfa_unet* net, const float* coef, const double* coef64,
              const float* lnk, const double* b, double* x, double tol, int64_t maxit,
              double inner_rtol, int max_outer, PrecMode fallback_mode, Work& w, Result* res) {
  for (res->outer = 0; res->outer <= max_outer; ++res->outer) {
    int rc = tpfa_residual64(c, coef64, b, x, w.r64, w.norms, w.s);
    if (rc) return rc;
    ++w.launches;
    if (cudaMemcpyAsync(w.hnorms, w.norms, 16, cudaMemcpyDeviceToHost, w.s) != cudaSuccess ||
        cudaStreamSynchronize(w.s) != cudaSuccess)
      return TPFA_ECUDA;
    const double rr64 = w.hnorms[0], bb64 = w.hnorms[1];
    if (!std::isfinite(rr64)) {
      res->status = TPFA_ENONFINITE;
      return TPFA_OK;
    }
    res->rel = bb64 > 0 ? std::sqrt(rr64 / bb64) : std::sqrt(rr64);
    if (res->rel <= tol || rr64 == 0.0) {
      res->status = TPFA_OK;
      return TPFA_OK;
    }
    if (res->outer == max_outer || res->iters >= maxit) return TPFA_OK;
    const double scale = 1.0 / std::sqrt(rr64);
    const double target = std::fmax(inner_rtol, 0.3 * tol / res->rel);
    const auto ti = std::chrono::steady_clock::now();
    double d3[3];
    start_kernel<<<w.nb, kT, 0, w.s>>>(w.r64, scale, w.r, w.e, w.n, w.part);
    ++w.launches;
    if (!w.fetch(d3)) return TPFA_ECUDA;
    rc = fcg_inner(c, net, coef, lnk, w, d3[0], target, maxit, fallback_mode, res);
    if (rc) return rc;
    correct_kernel<<<w.nb, kT, 0, w.s>>>(x, w.e, 1.0 / scale, w.n);
    ++w.launches;
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(w.s) != cudaSuccess)
      return TPFA_ECUDA;
    res->inner_ms +=
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - ti).count();
    if (res->status == TPFA_EBREAKDOWN) return TPFA_OK;
  }
  return TPFA_OK;
}

}  // namespace

extern "C" int fcg_solve(tpfa_ctx* c, tpfa_unet* net, const float* coef, const double* coef64,
                         const float* lnk, const double* b, double* x, double tol, int64_t maxit,
                         tpfa_cg_info* info, int* fell_back, void* stream) {
  const auto t0 = std::chrono::steady_clock::now();
  if (c == nullptr || !(tol > 0) || maxit < 1) return TPFA_EINVAL;
  const int64_t n = tpfa::ctx_cells(c);
  if (n <= 0) return TPFA_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return TPFA_ECUDA;
  if (!tpfa::dev_ok(coef, n * 16, 16, dev) || !tpfa::dev_ok(coef64, n * 32, 16, dev) ||
      !tpfa::dev_ok(b, n * 8, 8, dev) || !tpfa::dev_ok(x, n * 8, 8, dev) ||
      (net != nullptr && !tpfa::dev_ok(lnk, n * 4, 4, dev)))
    return TPFA_EINVAL;
  int64_t d3[3];
  tpfa::ctx_dims(c, d3);
  // the network's grid: the solver's grid or 2x / 4x / 8x coarser (extents divisible)
  int levels = -1;
  if (net != nullptr) {
    int d4[4];
    tpfa_unet_shape(net, d4);
    for (int l = 0; l <= kMaxLevels && levels < 0; ++l) {
      const int64_t f = 1LL << l;
      if (d3[0] % f == 0 && d3[1] % f == 0 && d3[2] % f == 0 && d4[0] == d3[0] / f &&
          d4[1] == d3[1] / f && d4[2] == d3[2] / f && (l == 0 || n < 2147483647LL))
        levels = l;
    }
    if (levels < 0 || d4[3] != 1) return TPFA_EINVAL;
    // the restriction reads ln K two cells at a time
    if (levels > 0 && reinterpret_cast<uintptr_t>(lnk) % 8 != 0) return TPFA_EINVAL;
  }
  const double inner_rtol = tpfa::ctx_option(c, TPFA_OPT_INNER_RTOL);
  const int max_outer = (int)tpfa::ctx_option(c, TPFA_OPT_MAX_OUTER);
  const PrecMode fallback_mode =
      tpfa::ctx_option(c, TPFA_OPT_FCG_FALLBACK) != 0.0 ? kJacobi : kIdentity;
  Result res;
  int rc;
  int64_t launches = 0;
  {
    Work w;
    w.s = (cudaStream_t)stream;
    w.n = n;
    w.m = (int)tpfa::ctx_option(c, TPFA_OPT_FCG_M);
    w.levels = levels > 0 ? levels : 0;
    for (int i = 0; i < 3; ++i) w.dims[i] = (int)d3[i];
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    w.nb = 4 * nsm;
    bool ok = w.alloc();
    if (ok) {
      dinv_kernel<<<w.nb, kT, 0, w.s>>>(reinterpret_cast<const float4*>(coef), w.dinv, n);
      ok = cudaGetLastError() == cudaSuccess;
    }
    if (ok && w.levels > 0) {
      for (int l = 1; l <= w.levels && ok; ++l) {
        const size_t bytes = (size_t)(n >> (3 * l)) * 4;
        ok = cudaMalloc(&w.rl[l], bytes) == cudaSuccess && cudaMalloc(&w.ul[l], bytes) == cudaSuccess;
      }
      ok = ok && cudaMalloc(&w.lnkc, (size_t)(n >> (3 * w.levels)) * 4) == cudaSuccess;
      if (ok) {
        // ln K on the network's grid (the mean over each 2^levels block), through the
        // image buffers of the intermediate levels
        const float* src = lnk;
        for (int l = 1; l <= w.levels; ++l) {
          float* dst = l == w.levels ? w.lnkc : w.ul[l];
          restrict2_kernel<<<w.nb, kT, 0, w.s>>>(src, dst, w.dims[0] >> (l - 1),
                                                 w.dims[1] >> (l - 1), w.dims[2] >> (l - 1), 1,
                                                 0.125f, nullptr, 0, 0, 0);
          src = dst;
        }
        ok = cudaGetLastError() == cudaSuccess;
      }
    }
    if (!ok) {
      cudaGetLastError();
      rc = TPFA_ENOMEM;
    } else {
      rc = fcg_outer(c, net, coef, coef64, lnk, b, x, tol, maxit, inner_rtol, max_outer,
                     fallback_mode, w, &res);
      if (rc == TPFA_OK && net != nullptr && tpfa_net_status(stream) != TPFA_OK) rc = TPFA_EINTERNAL;
    }
    launches = w.launches;
  }
  if (fell_back) *fell_back = res.fallback ? 1 : 0;
  if (info) {
    info->iters = res.iters;
    info->outer = res.outer;
    info->status = rc ? rc : res.status;
    info->rel_res_inner = 0.0;
    info->rel_res_fp64 = res.rel;
    info->inner_ms = res.inner_ms;
    info->total_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    info->kernel_launches = launches;
  }
  return rc ? rc : res.status;
}

// Gradient of the A-norm loss of the best multiple of mr (see the header):
// q = A mr, stats = (mr' r, mr' A mr), g = (2a/(b eae)) ((a/b) q - r).
extern "C" int tpfa_anorm_loss_grad(tpfa_ctx* c, const float* coef, const float* mr,
                                    const float* r, const double* eae, float* q, float* g,
                                    double* stats, void* stream) {
  const int64_t n = c ? tpfa::ctx_cells(c) : 0;
  if (n <= 0) return TPFA_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return TPFA_ECUDA;
  if (!tpfa::dev_ok(mr, n * 4, 4, dev) || !tpfa::dev_ok(r, n * 4, 4, dev) ||
      !tpfa::dev_ok(eae, 8, 8, dev) || !tpfa::dev_ok(q, n * 4, 4, dev) ||
      !tpfa::dev_ok(g, n * 4, 4, dev) || !tpfa::dev_ok(stats, 16, 8, dev))
    return TPFA_EINVAL;
  if (mr == q || mr == g || r == q || r == g || q == g) return TPFA_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  constexpr int nb = 512;
  double* part = nullptr;
  if (cudaMallocAsync((void**)&part, nb * sizeof(double), s) != cudaSuccess) return TPFA_ENOMEM;
  int rc = tpfa_apply(c, coef, mr, q, stats + 1, stream);
  if (rc == TPFA_OK) {
    dot_partial_kernel<<<nb, kT, 0, s>>>(mr, r, n, part);
    dot_finish_kernel<<<1, 1, 0, s>>>(part, nb, stats);
    loss_grad_kernel<<<nb, kT, 0, s>>>(q, r, stats, eae, g, n);
    if (cudaGetLastError() != cudaSuccess) rc = TPFA_ECUDA;
  }
  cudaFreeAsync(part, s);
  return rc;
}

// s = r - A D^-1 r and, when e and wAw are given, wAw = w' A w with
// w = e - D^-1 r: the training target of the network inside the Jacobi blend.
extern "C" int tpfa_jacobi_split(tpfa_ctx* c, const float* coef, const float* r, const float* e,
                                 float* s, double* wAw, void* stream) {
  const int64_t n = c ? tpfa::ctx_cells(c) : 0;
  if (n <= 0) return TPFA_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return TPFA_ECUDA;
  if (!tpfa::dev_ok(coef, n * 16, 16, dev) || !tpfa::dev_ok(r, n * 4, 4, dev) ||
      !tpfa::dev_ok(s, n * 4, 4, dev) || !tpfa::opt_dev_ok(e, n * 4, 4, dev) ||
      !tpfa::opt_dev_ok(wAw, 8, 8, dev) || (e == nullptr) != (wAw == nullptr))
    return TPFA_EINVAL;
  if (r == s || e == s) return TPFA_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  float *t1 = nullptr, *t2 = nullptr;
  if (cudaMallocAsync((void**)&t1, n * 4, st) != cudaSuccess) return TPFA_ENOMEM;
  if (cudaMallocAsync((void**)&t2, n * 4, st) != cudaSuccess) {
    cudaFreeAsync(t1, st);
    return TPFA_ENOMEM;
  }
  const int nb = (int)((n + kT - 1) / kT < 4096 ? (n + kT - 1) / kT : 4096);
  const float4* c4 = reinterpret_cast<const float4*>(coef);
  jacobi_kernel<<<nb, kT, 0, st>>>(r, c4, t1, n);
  int rc = tpfa_apply(c, coef, t1, t2, nullptr, stream);
  if (rc == TPFA_OK) {
    sub_kernel<<<nb, kT, 0, st>>>(r, t2, s, n);
    if (e != nullptr) {
      sub_kernel<<<nb, kT, 0, st>>>(e, t1, t1, n);
      rc = tpfa_apply(c, coef, t1, t2, wAw, stream);
    }
  }
  if (rc == TPFA_OK && cudaGetLastError() != cudaSuccess) rc = TPFA_ECUDA;
  cudaFreeAsync(t1, st);
  cudaFreeAsync(t2, st);
  return rc;
}

// coarse = scale * (sum of the 8 children) on the 2x coarser grid; fine
// nx x ny x nz (even) per sample, ns samples; dev FP32.  Asynchronous.
extern "C" int tpfa_restrict2(const float* fine, float* coarse, int nx, int ny, int nz, int ns,
                              float scale, void* stream) {
  if (nx < 2 || ny < 2 || nz < 2 || nx % 2 || ny % 2 || nz % 2 || ns < 1) return TPFA_EINVAL;
  if ((double)nx * ny * nz * ns >= 2147483647.0) return TPFA_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return TPFA_ECUDA;
  const size_t n = (size_t)nx * ny * nz * ns;
  if (!tpfa::dev_ok(fine, n * 4, 8, dev) || !tpfa::dev_ok(coarse, n / 8 * 4, 4, dev))
    return TPFA_EINVAL;
  const int nb = (int)((n / 8 + kT - 1) / kT < 4096 ? (n / 8 + kT - 1) / kT : 4096);
  restrict2_kernel<<<nb, kT, 0, (cudaStream_t)stream>>>(fine, coarse, nx, ny, nz, ns, scale,
                                                        nullptr, 0, 0, 0);
  return cudaGetLastError() == cudaSuccess ? TPFA_OK : TPFA_ECUDA;
}

// fine = coarse value of each cell's parent (nearest prolongation).  Asynchronous.
extern "C" int tpfa_prolong2(const float* coarse, float* fine, int nx, int ny, int nz, int ns,
                             void* stream) {
  if (nx < 2 || ny < 2 || nz < 2 || nx % 2 || ny % 2 || nz % 2 || ns < 1) return TPFA_EINVAL;
  if ((double)nx * ny * nz * ns >= 2147483647.0) return TPFA_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return TPFA_ECUDA;
  const size_t n = (size_t)nx * ny * nz * ns;
  if (!tpfa::dev_ok(fine, n * 4, 4, dev) || !tpfa::dev_ok(coarse, n / 8 * 4, 4, dev))
    return TPFA_EINVAL;
  const int nb = (int)((n + kT - 1) / kT < 4096 ? (n + kT - 1) / kT : 4096);
  prolong2_kernel<<<nb, kT, 0, (cudaStream_t)stream>>>(coarse, fine, nx, ny, nz, ns, nullptr, 0,
                                                       0, 0);
  return cudaGetLastError() == cudaSuccess ? TPFA_OK : TPFA_ECUDA;
}

// ---------------------------------------------------------------------------
// Batched flexible CG over the instances of a tpfa_batch (concatenated
// arrays).  The active instances iterate in lockstep: one launch of each
// vector pass covers all of them, block by block over chunks of one
// instance, and one-block-per-instance finish kernels form each instance's
// scalars from its own chunk partials in a fixed order, so an instance's
// iterates do not depend on the other instances.  Each instance has its own
// preconditioner mode, retained-direction count, inner tolerance, iteration
// limit and activity flag (cleared on the device when its inner solve
// converges).  The network term runs per size class: one U-Net over the
// samples of all instances of that grid, fed by a gathering restriction and
// returned by a scattering prolongation.
namespace {

constexpr int kChunk = 8192;  // cells per block of the batched vector passes (a multiple of 4)

enum BatchFlag : int {
  kAct = 1,    // iterating in the current inner solve
  kNet = 2,    // preconditioner: Jacobi blend with the network term
  kJac = 4,    // Jacobi scaling (the blend, or the Jacobi fallback)
  kOuter = 8,  // refined in the current outer step
};

struct BScal {
  double c;
  double beta[kMaxDirs];
  double pq[kMaxDirs];
  double alpha;
  double t2;        // squared inner tolerance relative to rr0
  double thr;       // t2 * rr0: the inner solve stops at r'r <= thr
  double rr0;
  double scale;     // r32 = scale * r64
  long long iters;  // inner iterations of the current outer step
  long long maxit;  // iteration limit of the current outer step
  int stored;       // retained directions (<= m)
  int bad;          // p'q <= 0 or a non-finite value since the host last looked
};

struct BChunk {
  int inst;
  int pad;
  int64_t beg, end;  // cells [beg, end) of the concatenated arrays
};

// The cells of one chunk: four at a time when vec4 (every chunk then starts
// on a multiple of 4 cells, i.e. 16 bytes), and a scalar tail.
template <class F1, class F4>
__device__ __forceinline__ void chunk_cells(const BChunk& ch, int vec4, F1&& f1, F4&& f4) {
  int64_t i0 = ch.beg;
  if (vec4) {
    const int64_t n4 = (ch.end - ch.beg) / 4;
    for (int64_t k = threadIdx.x; k < n4; k += kT) f4(ch.beg / 4 + k);
    i0 = ch.beg + 4 * n4;
  }
  for (int64_t i = i0 + threadIdx.x; i < ch.end; i += kT) f1(i);
}

// tot[k] (shared) = sum over the nc chunks first.. of value k of K per chunk,
// for k < K: one warp per value, lanes over chunks, a fixed shuffle tree
__device__ __forceinline__ void chunk_totals(const double* __restrict__ part, int first, int nc,
                                             int K, double* tot) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = warp; k < K; k += kT / 32) {
    double t = 0.0;
    for (int b = lane; b < nc; b += 32) t += part[(size_t)(first + b) * K + k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) tot[k] = t;
  }
  __syncthreads();
}

__device__ __forceinline__ float4 ld4(const float* p, int64_t k) {
  return reinterpret_cast<const float4*>(p)[k];
}

// r32 = scale r64, e = 0; partial r'r
__global__ void bstart_kernel(const BChunk* __restrict__ chunks, const int* __restrict__ flags,
                              const BScal* __restrict__ sc, const double* __restrict__ r64,
                              float* __restrict__ r, float* __restrict__ e, double* part) {
  const BChunk ch = chunks[blockIdx.x];
  if (!(flags[ch.inst] & kAct)) return;
  const double scale = sc[ch.inst].scale;
  double rr = 0.0;
  for (int64_t i = ch.beg + threadIdx.x; i < ch.end; i += kT) {
    const float v = (float)(r64[i] * scale);
    r[i] = v;
    e[i] = 0.f;
    rr += (double)v * v;
  }
  double d[1] = {rr};
  block_sum_m<1>(d, part);
}

// rr0 and the inner threshold of every active instance
__global__ void bfinish_start_kernel(const int* __restrict__ cfirst, const int* __restrict__ ccount,
                                     const int* __restrict__ flags, const double* __restrict__ part,
                                     BScal* sc) {
  const int i = blockIdx.x;
  if (!(flags[i] & kAct)) return;
  __shared__ double tot[1];
  chunk_totals(part, cfirst[i], ccount[i], 1, tot);
  if (threadIdx.x == 0) {
    sc[i].rr0 = tot[0];
    sc[i].thr = sc[i].t2 * tot[0];
  }
}

// x += e / scale for the instances refined in this outer step
__global__ void bcorrect_kernel(const BChunk* __restrict__ chunks, const int* __restrict__ flags,
                                const BScal* __restrict__ sc, const float* __restrict__ e,
                                double* __restrict__ x) {
  const BChunk ch = chunks[blockIdx.x];
  if (!(flags[ch.inst] & kOuter)) return;
  const double inv = 1.0 / sc[ch.inst].scale;
  for (int64_t i = ch.beg + threadIdx.x; i < ch.end; i += kT) x[i] += inv * (double)e[i];
}

// As dots_kernel, per chunk, with the instance's own preconditioner mode.
template <int M>
__global__ void bdots_kernel(const BChunk* __restrict__ chunks, const int* __restrict__ flags,
                             const float* __restrict__ r, const float* __restrict__ dinv,
                             const float* __restrict__ u, const float* __restrict__ au, Dirs qd,
                             int vec4, double* part) {
  constexpr int K = 2 + 2 * M;
  const BChunk ch = chunks[blockIdx.x];
  const int f = flags[ch.inst];
  if (!(f & kAct)) return;
  const bool jac = (f & kJac) != 0, net = (f & kNet) != 0;
  float s[K];
#pragma unroll
  for (int j = 0; j < K; ++j) s[j] = 0.f;
  auto one = [&](float ri, float di, float ui, float aui, const float* qv) {
    const float wi = jac ? ri * di : ri;
    if (net) {
      s[0] = fmaf(ui, ri, s[0]);
      s[1] = fmaf(aui, wi, s[1]);
    }
#pragma unroll
    for (int j = 0; j < M; ++j) {
      s[2 + j] = fmaf(wi, qv[j], s[2 + j]);
      s[2 + M + j] = fmaf(ui, qv[j], s[2 + M + j]);
    }
  };
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  chunk_cells(
      ch, vec4,
      [&](int64_t i) {
        float qv[M > 0 ? M : 1];
#pragma unroll
        for (int j = 0; j < M; ++j) qv[j] = qd.v[j][i];
        one(r[i], jac ? dinv[i] : 0.f, net ? u[i] : 0.f, net ? au[i] : 0.f, qv);
      },
      [&](int64_t k) {
        const float4 r4 = ld4(r, k);
        const float4 d4 = jac ? ld4(dinv, k) : z4;
        const float4 u4 = net ? ld4(u, k) : z4;
        const float4 a4 = net ? ld4(au, k) : z4;
        float4 q4[M > 0 ? M : 1];
#pragma unroll
        for (int j = 0; j < M; ++j) q4[j] = ld4(qd.v[j], k);
        float qv[M > 0 ? M : 1];
#pragma unroll
        for (int j = 0; j < M; ++j) qv[j] = q4[j].x;
        one(r4.x, d4.x, u4.x, a4.x, qv);
#pragma unroll
        for (int j = 0; j < M; ++j) qv[j] = q4[j].y;
        one(r4.y, d4.y, u4.y, a4.y, qv);
#pragma unroll
        for (int j = 0; j < M; ++j) qv[j] = q4[j].z;
        one(r4.z, d4.z, u4.z, a4.z, qv);
#pragma unroll
        for (int j = 0; j < M; ++j) qv[j] = q4[j].w;
        one(r4.w, d4.w, u4.w, a4.w, qv);
      });
  double d[K];
#pragma unroll
  for (int j = 0; j < K; ++j) d[j] = s[j];
  block_sum_m<K>(d, part);
}

// c and the beta_j of every active instance (beta_j = 0 beyond its own
// retained directions)
__global__ void bfinish_dots_kernel(const int* __restrict__ cfirst, const int* __restrict__ ccount,
                                    const int* __restrict__ flags, const double* __restrict__ part,
                                    int M, const double* __restrict__ uau, BScal* sc, int head,
                                    int m) {
  const int i = blockIdx.x;
  const int f = flags[i];
  if (!(f & kAct)) return;
  __shared__ double tot[2 + 2 * kMaxDirs];
  const int K = 2 + 2 * M;
  chunk_totals(part, cfirst[i], ccount[i], K, tot);
  if (threadIdx.x == 0) {
    BScal& S = sc[i];
    double c = 0.0;
    if (f & kNet) {
      const double d = uau[i];
      c = (d > 0.0 && isfinite(d)) ? (tot[0] - tot[1]) / d : 0.0;
      if (!isfinite(c)) c = 0.0;
    }
    S.c = c;
    for (int j = 0; j < M; ++j) {
      double b = 0.0;
      if (j < S.stored) {
        const int slot = (head - 1 - j + m) % m;
        b = -(tot[2 + j] + c * tot[2 + M + j]) / S.pq[slot];
        if (!isfinite(b)) {
          S.bad = 1;
          b = 0.0;
        }
      }
      S.beta[j] = b;
    }
  }
}

// As dir_kernel, per chunk: p = w + c u + sum over the instance's retained
// directions of beta_j p_j; partial p'r
template <int M>
__global__ void bdir_kernel(const BChunk* __restrict__ chunks, const int* __restrict__ flags,
                            const BScal* __restrict__ sc, const float* __restrict__ r,
                            const float* __restrict__ dinv, const float* __restrict__ u, Dirs pd,
                            float* p, int vec4, double* part) {
  // p may be the oldest retained direction (read, then overwritten, per element)
  const BChunk ch = chunks[blockIdx.x];
  const int f = flags[ch.inst];
  if (!(f & kAct)) return;
  const bool jac = (f & kJac) != 0, net = (f & kNet) != 0;
  const BScal& S = sc[ch.inst];
  const int ns = S.stored;
  const float c = (float)S.c;
  float beta[M > 0 ? M : 1];
#pragma unroll
  for (int j = 0; j < M; ++j) beta[j] = (float)S.beta[j];
  float prf = 0.f;
  auto one = [&](float ri, float di, float ui, const float* pv) {
    float v = jac ? ri * di : ri;
    if (net) v = fmaf(c, ui, v);
#pragma unroll
    for (int j = 0; j < M; ++j)
      if (j < ns) v = fmaf(beta[j], pv[j], v);
    prf = fmaf(v, ri, prf);
    return v;
  };
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  chunk_cells(
      ch, vec4,
      [&](int64_t i) {
        float pv[M > 0 ? M : 1];
#pragma unroll
        for (int j = 0; j < M; ++j) pv[j] = j < ns ? pd.v[j][i] : 0.f;
        p[i] = one(r[i], jac ? dinv[i] : 0.f, net ? u[i] : 0.f, pv);
      },
      [&](int64_t k) {
        const float4 r4 = ld4(r, k);
        const float4 d4 = jac ? ld4(dinv, k) : z4;
        const float4 u4 = net ? ld4(u, k) : z4;
        float4 p4[M > 0 ? M : 1];
#pragma unroll
        for (int j = 0; j < M; ++j) p4[j] = j < ns ? ld4(pd.v[j], k) : z4;
        float pv[M > 0 ? M : 1];
        float4 o;
#pragma unroll
        for (int j = 0; j < M; ++j) pv[j] = p4[j].x;
        o.x = one(r4.x, d4.x, u4.x, pv);
#pragma unroll
        for (int j = 0; j < M; ++j) pv[j] = p4[j].y;
        o.y = one(r4.y, d4.y, u4.y, pv);
#pragma unroll
        for (int j = 0; j < M; ++j) pv[j] = p4[j].z;
        o.z = one(r4.z, d4.z, u4.z, pv);
#pragma unroll
        for (int j = 0; j < M; ++j) pv[j] = p4[j].w;
        o.w = one(r4.w, d4.w, u4.w, pv);
        reinterpret_cast<float4*>(p)[k] = o;
      });
  double pr[1] = {prf};
  block_sum_m<1>(pr, part);
}

// alpha = p'r / p'q per active instance (0 and the bad flag when p'q is not
// positive or a value is not finite); p'q of the new direction into its slot
__global__ void bfinish_alpha_kernel(const int* __restrict__ cfirst, const int* __restrict__ ccount,
                                     const int* __restrict__ flags, const double* __restrict__ part,
                                     const double* __restrict__ pq_dev, BScal* sc, int head, int m) {
  const int i = blockIdx.x;
  if (!(flags[i] & kAct)) return;
  __shared__ double tot[1];
  chunk_totals(part, cfirst[i], ccount[i], 1, tot);
  if (threadIdx.x == 0) {
    BScal& S = sc[i];
    const double pr = tot[0], pq = pq_dev[i];
    if (!(pq > 0.0) || !isfinite(pq) || !isfinite(pr)) {
      S.bad = 1;
      S.alpha = 0.0;
      S.pq[head] = 1.0;
    } else {
      S.alpha = pr / pq;
      S.pq[head] = pq;
    }
    if (S.stored < m) ++S.stored;
  }
}

// e += alpha p; r -= alpha q; partial r'r
__global__ void bupdate_kernel(const BChunk* __restrict__ chunks, const int* __restrict__ flags,
                               const BScal* __restrict__ sc, float* __restrict__ e,
                               float* __restrict__ r, const float* __restrict__ p,
                               const float* __restrict__ q, int vec4, double* part) {
  const BChunk ch = chunks[blockIdx.x];
  if (!(flags[ch.inst] & kAct)) return;
  const float alpha = (float)sc[ch.inst].alpha;
  float rrf = 0.f;
  chunk_cells(
      ch, vec4,
      [&](int64_t i) {
        e[i] = fmaf(alpha, p[i], e[i]);
        const float v = fmaf(-alpha, q[i], r[i]);
        r[i] = v;
        rrf = fmaf(v, v, rrf);
      },
      [&](int64_t k) {
        float4 e4 = ld4(e, k), r4 = ld4(r, k);
        const float4 p4 = ld4(p, k), q4 = ld4(q, k);
        e4.x = fmaf(alpha, p4.x, e4.x);
        e4.y = fmaf(alpha, p4.y, e4.y);
        e4.z = fmaf(alpha, p4.z, e4.z);
        e4.w = fmaf(alpha, p4.w, e4.w);
        r4.x = fmaf(-alpha, q4.x, r4.x);
        r4.y = fmaf(-alpha, q4.y, r4.y);
        r4.z = fmaf(-alpha, q4.z, r4.z);
        r4.w = fmaf(-alpha, q4.w, r4.w);
        reinterpret_cast<float4*>(e)[k] = e4;
        reinterpret_cast<float4*>(r)[k] = r4;
        rrf = fmaf(r4.x, r4.x, rrf);
        rrf = fmaf(r4.y, r4.y, rrf);
        rrf = fmaf(r4.z, r4.z, rrf);
        rrf = fmaf(r4.w, r4.w, rrf);
      });
  double rr[1] = {rrf};
  block_sum_m<1>(rr, part);
}

// r'r of this iteration into the instance's history slot (-1 for an instance
// that did not iterate); an instance whose r'r met its threshold (or is not
// a number), or that reached its iteration limit, stops iterating
__global__ void bfinish_rr_kernel(const int* __restrict__ cfirst, const int* __restrict__ ccount,
                                  int* flags, const double* __restrict__ part, BScal* sc,
                                  double* hist, int pending) {
  const int i = blockIdx.x;
  const int f = flags[i];
  if (!(f & kAct)) {
    if (threadIdx.x == 0) hist[(size_t)i * kCheckEvery + pending] = -1.0;
    return;
  }
  __shared__ double tot[1];
  chunk_totals(part, cfirst[i], ccount[i], 1, tot);
  if (threadIdx.x == 0) {
    BScal& S = sc[i];
    const double rr = tot[0];
    hist[(size_t)i * kCheckEvery + pending] = rr;
    S.iters += 1;
    if (!(rr > S.thr) || S.iters >= S.maxit) flags[i] = f & ~kAct;
  }
}

// dst[s][c] = src[soff[s] + c] (gather), or dst[soff[s] + c] = src[s][c]
// (scatter); n cells per sample, ns samples
__global__ void gather_kernel(const float* __restrict__ src, const int64_t* __restrict__ soff,
                              float* __restrict__ dst, int64_t n, int ns, int scatter) {
  const int64_t tot = n * ns;
  for (int64_t c = (int64_t)blockIdx.x * kT + threadIdx.x; c < tot; c += (int64_t)gridDim.x * kT) {
    const int64_t s = c / n, i = c - s * n;
    if (scatter) dst[soff[s] + i] = src[c];
    else dst[c] = src[soff[s] + i];
  }
}

void launch_bdots(int M, unsigned nchunks, cudaStream_t s, const BChunk* ch, const int* flags,
                  const float* r, const float* dinv, const float* u, const float* au,
                  const Dirs& qd, int vec4, double* part) {
  switch (M) {
#define X(MM)                                                                                 \
  case MM:                                                                                    \
    bdots_kernel<MM><<<nchunks, kT, 0, s>>>(ch, flags, r, dinv, u, au, qd, vec4, part); \
    break;
    TPFA_FCG_M0(X)
#undef X
    default: break;
  }
}

void launch_bdir(int M, unsigned nchunks, cudaStream_t s, const BChunk* ch, const int* flags,
                 const BScal* sc, const float* r, const float* dinv, const float* u,
                 const Dirs& pd, float* p, int vec4, double* part) {
  switch (M) {
#define X(MM)                                                                                    \
  case MM:                                                                                       \
    bdir_kernel<MM><<<nchunks, kT, 0, s>>>(ch, flags, sc, r, dinv, u, pd, p, vec4, part); \
    break;
    TPFA_FCG_M0(X)
#undef X
    default: break;
  }
}

// One network of the batched solve: the instances (members) that share it,
// which all have the same grid; the network runs on the 2^levels coarser grid,
// and only on the members that still iterate with it (the active ones, as a
// prefix of its samples).
struct BNet {
  tpfa_unet* net = nullptr;
  int levels = 0;
  int dims[3] = {0, 0, 0};  // the members' grid
  int pdims[3] = {0, 0, 0}; // the network's grid: the 2^levels coarser grid, each extent
                            // rounded up to a multiple of 4 (zero padding beyond the grid)
  int64_t ncoarse = 0;      // cells of one sample on the network's grid
  // stored extents of level l (0: unpadded), for the restriction into level l
  // and the prolongation out of it
  int qx(int l) const { return l == levels ? pdims[0] : 0; }
  int qy(int l) const { return l == levels ? pdims[1] : 0; }
  int qz(int l) const { return l == levels ? pdims[2] : 0; }
  std::vector<int> members;
  std::vector<int> active;  // indices into members of the samples the network runs on
  int64_t* soff = nullptr;  // dev: cell offset of each active member in the concatenated arrays
  int64_t* coff = nullptr;  // dev: offset of each active member's sample in lnk_all
  float* rl[kMaxLevels + 1] = {};  // restricted residuals per level (level 0: gathered copy)
  float* ul[kMaxLevels + 1] = {};  // network term per level (level 0: before the scatter)
  float* lnk_all = nullptr;        // ln K on the network's grid, member after member
  float* lnkc = nullptr;           // the same for the active members, in their order
  cudaStream_t st = nullptr;       // the networks are independent: each runs on its own stream
  cudaEvent_t done = nullptr;
  BNet() = default;
  BNet(const BNet&) = delete;
  BNet& operator=(const BNet&) = delete;
  ~BNet() {
    if (st) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
    if (done) cudaEventDestroy(done);
    cudaFree(soff);
    cudaFree(coff);
    cudaFree(lnk_all);
    for (int l = 0; l <= kMaxLevels; ++l) {
      cudaFree(rl[l]);
      cudaFree(ul[l]);
    }
    cudaFree(lnkc);
  }
};

struct BWork {
  cudaStream_t s = nullptr;
  int ninst = 0, m = 1, vec4 = 0, nb = 0;
  int64_t cells = 0, stride = 0;
  std::vector<BChunk> chunks;
  std::vector<int> cfirst, ccount;
  BChunk* chunks_dev = nullptr;
  int *cfirst_dev = nullptr, *ccount_dev = nullptr, *flags = nullptr, *hflags = nullptr;
  BScal *sc = nullptr, *hsc = nullptr;
  float *r = nullptr, *z = nullptr, *e = nullptr, *au = nullptr, *dinv = nullptr;
  float *P = nullptr, *Q = nullptr;
  double *part = nullptr, *uau = nullptr, *pq = nullptr, *norms = nullptr, *hnorms = nullptr;
  double *hist = nullptr, *hhist = nullptr;
  cudaEvent_t fork = nullptr;  // the networks' streams start after it
  int64_t launches = 0;

  bool alloc() {
    const size_t v = (size_t)stride * 4;
    const size_t nc = chunks.size();
    bool ok = cudaMalloc(&chunks_dev, sizeof(BChunk) * nc) == cudaSuccess &&
              cudaMalloc(&cfirst_dev, sizeof(int) * ninst) == cudaSuccess &&
              cudaMalloc(&ccount_dev, sizeof(int) * ninst) == cudaSuccess &&
              cudaMalloc(&flags, sizeof(int) * ninst) == cudaSuccess &&
              cudaMallocHost(&hflags, sizeof(int) * ninst) == cudaSuccess &&
              cudaMalloc(&sc, sizeof(BScal) * ninst) == cudaSuccess &&
              cudaMallocHost(&hsc, sizeof(BScal) * ninst) == cudaSuccess &&
              cudaMalloc(&r, v) == cudaSuccess && cudaMalloc(&z, v) == cudaSuccess &&
              cudaMalloc(&e, v) == cudaSuccess && cudaMalloc(&au, v) == cudaSuccess &&
              cudaMalloc(&dinv, v) == cudaSuccess &&
              cudaMalloc(&P, v * m) == cudaSuccess && cudaMalloc(&Q, v * m) == cudaSuccess &&
              cudaMalloc(&part, sizeof(double) * kPartPerBlock * nc) == cudaSuccess &&
              cudaMalloc(&uau, sizeof(double) * ninst) == cudaSuccess &&
              cudaMalloc(&pq, sizeof(double) * ninst) == cudaSuccess &&
              cudaMalloc(&norms, sizeof(double) * 2 * ninst) == cudaSuccess &&
              cudaMallocHost(&hnorms, sizeof(double) * 2 * ninst) == cudaSuccess &&
              cudaMalloc(&hist, sizeof(double) * kCheckEvery * ninst) == cudaSuccess &&
              cudaMallocHost(&hhist, sizeof(double) * kCheckEvery * ninst) == cudaSuccess &&
              cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess;
    // defined contents everywhere (the network also reads the residuals of
    // instances that are not iterating)
    ok = ok && cudaMemsetAsync(r, 0, v, s) == cudaSuccess &&
         cudaMemsetAsync(z, 0, v, s) == cudaSuccess && cudaMemsetAsync(e, 0, v, s) == cudaSuccess &&
         cudaMemsetAsync(flags, 0, sizeof(int) * ninst, s) == cudaSuccess &&
         cudaMemcpyAsync(chunks_dev, chunks.data(), sizeof(BChunk) * nc, cudaMemcpyHostToDevice,
                         s) == cudaSuccess &&
         cudaMemcpyAsync(cfirst_dev, cfirst.data(), sizeof(int) * ninst, cudaMemcpyHostToDevice,
                         s) == cudaSuccess &&
         cudaMemcpyAsync(ccount_dev, ccount.data(), sizeof(int) * ninst, cudaMemcpyHostToDevice,
                         s) == cudaSuccess &&
         cudaStreamSynchronize(s) == cudaSuccess;
    return ok;
  }
  ~BWork() {
    if (s) cudaStreamSynchronize(s);
    cudaFree(chunks_dev);
    cudaFree(cfirst_dev);
    cudaFree(ccount_dev);
    cudaFree(flags);
    cudaFreeHost(hflags);
    cudaFree(sc);
    cudaFreeHost(hsc);
    cudaFree(r);
    cudaFree(z);
    cudaFree(e);
    cudaFree(au);
    cudaFree(dinv);
    cudaFree(P);
    cudaFree(Q);
    cudaFree(part);
    cudaFree(uau);
    cudaFree(pq);
    cudaFree(norms);
    cudaFreeHost(hnorms);
    cudaFree(hist);
    cudaFreeHost(hhist);
    if (fork) cudaEventDestroy(fork);
  }
  unsigned nchunks() const { return (unsigned)chunks.size(); }
};

// The members of each network that iterate in blend mode (blend[i]): when
// the set changes, their cell offsets and the offsets of their ln K samples
// are uploaded and their ln K gathered into the network's input prefix.
// Called with every stream idle (outer-step start, the host's looks).
int update_active(std::vector<BNet>& nets, const std::vector<int>& blend,
                  const std::vector<int64_t>& off, BWork& w) {
  for (BNet& N : nets) {
    std::vector<int> act;
    for (int j = 0; j < (int)N.members.size(); ++j)
      if (blend[N.members[j]]) act.push_back(j);
    if (act == N.active) continue;
    N.active = act;
    if (act.empty()) continue;
    const int ns = (int)act.size();
    std::vector<int64_t> so(ns), co(ns);
    for (int k = 0; k < ns; ++k) {
      so[k] = off[N.members[act[k]]];
      co[k] = (int64_t)act[k] * N.ncoarse;
    }
    if (cudaMemcpyAsync(N.soff, so.data(), sizeof(int64_t) * ns, cudaMemcpyHostToDevice, w.s) !=
            cudaSuccess ||
        cudaMemcpyAsync(N.coff, co.data(), sizeof(int64_t) * ns, cudaMemcpyHostToDevice, w.s) !=
            cudaSuccess)
      return TPFA_ECUDA;
    gather_kernel<<<w.nb, kT, 0, w.s>>>(N.lnk_all, N.coff, N.lnkc, N.ncoarse, ns, 0);
    ++w.launches;
    if (cudaGetLastError() != cudaSuccess) return TPFA_ECUDA;
  }
  return TPFA_OK;
}

// u = P^l net(R^l r, R^l ln K) for the active members of one network, on w.s
int network_class(BNet& N, BWork& w) {
  const int ns = (int)N.active.size();
  int rc;
  if (N.levels > 0) {
    for (int l = 1; l <= N.levels; ++l)
      restrict2_kernel<<<w.nb, kT, 0, w.s>>>(l == 1 ? w.r : N.rl[l - 1], N.rl[l],
                                             N.dims[0] >> (l - 1), N.dims[1] >> (l - 1),
                                             N.dims[2] >> (l - 1), ns, 0.125f,
                                             l == 1 ? N.soff : nullptr, N.qx(l), N.qy(l), N.qz(l));
    rc = tpfa_unet_forward_samples(N.net, ns, N.rl[N.levels], N.lnkc, N.ul[N.levels], w.s);
    if (rc) return rc;
    for (int l = N.levels; l >= 1; --l)
      prolong2_kernel<<<w.nb, kT, 0, w.s>>>(N.ul[l], l == 1 ? w.z : N.ul[l - 1],
                                            N.dims[0] >> (l - 1), N.dims[1] >> (l - 1),
                                            N.dims[2] >> (l - 1), ns, l == 1 ? N.soff : nullptr,
                                            N.qx(l), N.qy(l), N.qz(l));
    w.launches += 15 + 2 * N.levels;
  } else {
    const int64_t n = (int64_t)N.dims[0] * N.dims[1] * N.dims[2];
    gather_kernel<<<w.nb, kT, 0, w.s>>>(w.r, N.soff, N.rl[0], n, ns, 0);
    rc = tpfa_unet_forward_samples(N.net, ns, N.rl[0], N.lnkc, N.ul[0], w.s);
    if (rc) return rc;
    gather_kernel<<<w.nb, kT, 0, w.s>>>(N.ul[0], N.soff, w.z, n, ns, 1);
    w.launches += 17;
  }
  return cudaGetLastError() == cudaSuccess ? TPFA_OK : TPFA_ECUDA;
}

// u = network term of every network with a member that iterates in blend
// mode (into w.z at the members' cells).  The networks touch disjoint cells
// and their own buffers only: each runs on its own stream, forked from and
// joined back to w.s, so that the small, latency-bound layers of the size
// classes overlap.
int batch_network_term(std::vector<BNet>& nets, BWork& w) {
  if (cudaEventRecord(w.fork, w.s) != cudaSuccess) return TPFA_ECUDA;
  const cudaStream_t main = w.s;
  for (BNet& N : nets) {
    if (N.active.empty()) continue;
    if (cudaStreamWaitEvent(N.st, w.fork, 0) != cudaSuccess) return TPFA_ECUDA;
    w.s = N.st;
    const int rc = network_class(N, w);
    w.s = main;
    if (rc) return rc;
    if (cudaEventRecord(N.done, N.st) != cudaSuccess ||
        cudaStreamWaitEvent(main, N.done, 0) != cudaSuccess)
      return TPFA_ECUDA;
  }
  return TPFA_OK;
}

}  // namespace

// Arguments and results: see the header.  Instance results match what
// fcg_solve computes for the instance alone up to the order of the dot
// products' partial sums; the instances of one call do not influence each
// other's iterates.
extern "C" int fcg_solve_batch(tpfa_batch* batch, tpfa_unet* const* nets, int n_nets,
                               const int* net_of, const float* coef, const double* coef64,
                               const float* lnk, const double* b, double* x, double tol,
                               int64_t maxit, tpfa_cg_info* infos, tpfa_cg_info* total,
                               int* fell_back, void* stream) {
  using namespace tpfa;
  const auto t0 = std::chrono::steady_clock::now();
  if (batch == nullptr || !(tol > 0) || !std::isfinite(tol) || maxit < 1 || n_nets < 0 ||
      (n_nets > 0 && (nets == nullptr || net_of == nullptr)))
    return TPFA_EINVAL;
  const int N = batch->ninst;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return TPFA_ECUDA;
  if (cur != batch->device && cudaSetDevice(batch->device) != cudaSuccess) return TPFA_ECUDA;
  const int dev = batch->device;
  const size_t n = (size_t)batch->cells;
  if (!dev_ok(coef, n * 16, 16, dev) || !dev_ok(coef64, n * 32, 16, dev) ||
      !dev_ok(b, n * 8, 8, dev) || !dev_ok(x, n * 8, 8, dev) ||
      (n_nets > 0 && !dev_ok(lnk, n * 4, 4, dev)))
    return TPFA_EINVAL;
  if ((const void*)b == (const void*)x) return TPFA_EINVAL;
  // networks: members, level, shape
  std::vector<BNet> bn(n_nets);
  std::vector<int> of(N, -1);
  for (int i = 0; i < N && n_nets > 0; ++i) {
    if (net_of[i] < -1 || net_of[i] >= n_nets) return TPFA_EINVAL;
    of[i] = net_of[i];
    if (of[i] >= 0) bn[of[i]].members.push_back(i);
  }
  for (int k = 0; k < n_nets; ++k) {
    BNet& B = bn[k];
    B.net = nets[k];
    if (B.net == nullptr || B.members.empty()) return TPFA_EINVAL;
    const Grid& g0 = batch->g[B.members[0]];
    int d4[4];
    if (tpfa_unet_shape(B.net, d4) != TPFA_OK || d4[3] != (int)B.members.size()) return TPFA_EINVAL;
    // the network's level: its grid is the members' grid (l = 0) or the 2^l
    // coarser one with each extent rounded up to a multiple of 4; the finest
    // level that fits is taken
    B.levels = -1;
    auto up4 = [](int64_t v) { return (v + 3) / 4 * 4; };
    for (int l = 0; l <= kMaxLevels && B.levels < 0; ++l) {
      const int64_t f = 1LL << l;
      if (g0.nx % f != 0 || g0.ny % f != 0 || g0.nz % f != 0) continue;
      const int64_t c[3] = {g0.nx / f, g0.ny / f, g0.nz / f};
      bool fits = true;
      for (int a = 0; a < 3; ++a) fits = fits && d4[a] == (l == 0 ? c[a] : up4(c[a]));
      if (fits) B.levels = l;
    }
    if (B.levels < 0) return TPFA_EINVAL;
    for (int a = 0; a < 3; ++a) B.pdims[a] = d4[a];
    if ((double)g0.n * B.members.size() >= 2147483647.0) return TPFA_EINVAL;
    for (int i : B.members) {
      const Grid& gi = batch->g[i];
      if (gi.nx != g0.nx || gi.ny != g0.ny || gi.nz != g0.nz) return TPFA_EINVAL;
      if (B.levels > 0 && batch->off[i] % 2 != 0) return TPFA_EINVAL;
    }
    B.dims[0] = (int)g0.nx;
    B.dims[1] = (int)g0.ny;
    B.dims[2] = (int)g0.nz;
    // the restriction reads ln K two cells at a time
    if (B.levels > 0 && reinterpret_cast<uintptr_t>(lnk) % 8 != 0) return TPFA_EINVAL;
  }
  const double inner_rtol = batch->inner_rtol;
  const int max_outer = batch->max_outer;
  const int fb_bits = batch->fcg_fallback ? kJac : 0;
  cudaStream_t s = (cudaStream_t)stream;

  std::vector<int64_t> iters(N, 0);
  std::vector<int> outer(N, 0), status(N, TPFA_OK), fb(N, 0);
  std::vector<double> rel(N, INFINITY);
  double inner_ms = 0.0;
  int rc = TPFA_OK;
  int64_t launches = 0;
  {
    BWork w;
    w.s = s;
    w.ninst = N;
    w.m = batch->fcg_m;
    w.cells = batch->cells;
    w.stride = (batch->cells + 3) / 4 * 4;
    w.nb = 4 * batch->num_sms;
    w.vec4 = 1;
    w.cfirst.resize(N);
    w.ccount.resize(N);
    for (int i = 0; i < N; ++i) {
      if (batch->off[i] % 4 != 0) w.vec4 = 0;
      w.cfirst[i] = (int)w.chunks.size();
      for (int64_t c0 = batch->off[i]; c0 < batch->off[i + 1]; c0 += kChunk) {
        BChunk ch;
        ch.inst = i;
        ch.pad = 0;
        ch.beg = c0;
        ch.end = std::min<int64_t>(c0 + kChunk, batch->off[i + 1]);
        w.chunks.push_back(ch);
      }
      w.ccount[i] = (int)w.chunks.size() - w.cfirst[i];
    }
    if (w.chunks.size() > 0x7fffffffu) return TPFA_EINVAL;
    bool ok = w.alloc();
    if (ok) {
      dinv_kernel<<<w.nb, kT, 0, s>>>(reinterpret_cast<const float4*>(coef), w.dinv, w.cells);
      ok = cudaGetLastError() == cudaSuccess;
    }
    for (BNet& B : bn) {
      if (!ok) break;
      const int ns = (int)B.members.size();
      std::vector<int64_t> so(ns);
      for (int j = 0; j < ns; ++j) so[j] = batch->off[B.members[j]];
      const int64_t nf = (int64_t)B.dims[0] * B.dims[1] * B.dims[2];
      ok = cudaStreamCreateWithFlags(&B.st, cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&B.done, cudaEventDisableTiming) == cudaSuccess &&
           cudaMalloc(&B.soff, sizeof(int64_t) * ns) == cudaSuccess &&
           cudaMemcpyAsync(B.soff, so.data(), sizeof(int64_t) * ns, cudaMemcpyHostToDevice, s) ==
               cudaSuccess;
      // the network's level is stored padded; its padding stays zero (the
      // restriction writes only the grid's cells)
      B.ncoarse = (int64_t)B.pdims[0] * B.pdims[1] * B.pdims[2];
      for (int l = B.levels > 0 ? 1 : 0; l <= B.levels && ok; ++l) {
        const size_t bytes = (l == B.levels ? (size_t)B.ncoarse : (size_t)(nf >> (3 * l))) * ns * 4;
        ok = cudaMalloc(&B.rl[l], bytes) == cudaSuccess && cudaMalloc(&B.ul[l], bytes) == cudaSuccess &&
             cudaMemsetAsync(B.rl[l], 0, bytes, s) == cudaSuccess;
      }
      ok = ok && cudaMalloc(&B.lnkc, (size_t)B.ncoarse * ns * 4) == cudaSuccess &&
           cudaMalloc(&B.lnk_all, (size_t)B.ncoarse * ns * 4) == cudaSuccess &&
           cudaMemsetAsync(B.lnk_all, 0, (size_t)B.ncoarse * ns * 4, s) == cudaSuccess &&
           cudaMalloc(&B.coff, sizeof(int64_t) * ns) == cudaSuccess;
      if (!ok) break;
      // ln K on the network's grid (mean over each 2^levels block), member
      // after member, through the image buffers of the intermediate levels
      if (B.levels == 0) {
        gather_kernel<<<w.nb, kT, 0, s>>>(lnk, B.soff, B.lnk_all, nf, ns, 0);
      } else {
        for (int l = 1; l <= B.levels; ++l)
          restrict2_kernel<<<w.nb, kT, 0, s>>>(l == 1 ? lnk : B.ul[l - 1],
                                               l == B.levels ? B.lnk_all : B.ul[l],
                                               B.dims[0] >> (l - 1), B.dims[1] >> (l - 1),
                                               B.dims[2] >> (l - 1), ns, 0.125f,
                                               l == 1 ? B.soff : nullptr, B.qx(l), B.qy(l),
                                               B.qz(l));
      }
      ok = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(s) == cudaSuccess;
    }
    ok = ok && cudaMemsetAsync(batch->counters, 0, sizeof(unsigned int) * (N + 1), s) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      return TPFA_ENOMEM;
    }
    const float4* cf4 = reinterpret_cast<const float4*>(coef);
    unsigned int* ecounter = batch->counters + N;
    auto residuals = [&](const std::vector<int>& which) -> int {
      for (int i = 0; i < N; ++i) {
        if (!which[i]) continue;
        const int64_t o = batch->off[i];
        if (launch_residual64(batch->g[i], coef64 + 4 * o, b + o, x + o, batch->r64 + o,
                              w.norms + 2 * i, nullptr, batch->partials, ecounter,
                              elem_blocks(batch->g[i], batch->num_sms), s) != cudaSuccess)
          return TPFA_ECUDA;
        ++w.launches;
      }
      if (cudaMemcpyAsync(w.hnorms, w.norms, sizeof(double) * 2 * N, cudaMemcpyDeviceToHost, s) !=
              cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        return TPFA_ECUDA;
      for (int i = 0; i < N; ++i) {
        if (!which[i]) continue;
        const double rr64 = w.hnorms[2 * i], bb64 = w.hnorms[2 * i + 1];
        if (!std::isfinite(rr64)) {
          status[i] = TPFA_ENONFINITE;
          continue;
        }
        rel[i] = bb64 > 0 ? std::sqrt(rr64 / bb64) : std::sqrt(rr64);
        w.hsc[i].scale = rr64 > 0 ? 1.0 / std::sqrt(rr64) : 1.0;
      }
      return TPFA_OK;
    };
    std::vector<int> todo(N, 1), blend(N, 0);
    std::vector<std::vector<double>> hist(N);
    std::memset(w.hsc, 0, sizeof(BScal) * N);
    rc = residuals(todo);
    for (int step = 0; rc == TPFA_OK && step <= max_outer; ++step) {
      // instances refined in this outer step
      int nact = 0;
      for (int i = 0; i < N; ++i) {
        todo[i] = status[i] == TPFA_OK && rel[i] > tol && iters[i] < maxit && step < max_outer;
        w.hflags[i] = 0;
        if (!todo[i]) continue;
        ++nact;
        BScal& S = w.hsc[i];
        const double scale = S.scale;
        std::memset(&S, 0, sizeof(BScal));
        S.scale = scale;
        const double target = std::fmax(inner_rtol, 0.3 * tol / rel[i]);
        S.t2 = target * target;
        S.maxit = maxit - iters[i];
        w.hflags[i] = kOuter | kAct | (of[i] >= 0 && !fb[i] ? (kNet | kJac) : fb_bits);
        hist[i].clear();
      }
      if (nact == 0) break;
      const auto ti = std::chrono::steady_clock::now();
      if (cudaMemcpyAsync(w.sc, w.hsc, sizeof(BScal) * N, cudaMemcpyHostToDevice, s) !=
              cudaSuccess ||
          cudaMemcpyAsync(w.flags, w.hflags, sizeof(int) * N, cudaMemcpyHostToDevice, s) !=
              cudaSuccess) {
        rc = TPFA_ECUDA;
        break;
      }
      bstart_kernel<<<w.nchunks(), kT, 0, s>>>(w.chunks_dev, w.flags, w.sc, batch->r64, w.r, w.e,
                                               w.part);
      bfinish_start_kernel<<<N, kT, 0, s>>>(w.cfirst_dev, w.ccount_dev, w.flags, w.part, w.sc);
      w.launches += 2;
      // inner FCG, all refined instances in lockstep
      int head = 0, gstored = 0, pending = 0;
      int64_t giters = 0;
      bool running = true;
      for (int i = 0; i < N; ++i) blend[i] = (w.hflags[i] & kNet) != 0;
      rc = update_active(bn, blend, batch->off, w);
      if (rc) break;
      bool first = true;
      while (running && rc == TPFA_OK) {
        bool any_blend = false;
        for (int i = 0; i < N; ++i) any_blend = any_blend || blend[i];
        if (any_blend) {
          rc = batch_network_term(bn, w);
          if (rc) break;
          if (launch_apply_batch(batch->inst_dev, N, batch->sweep_blocks, cf4, w.z, w.au, w.uau,
                                 w.flags, kAct | kNet, batch->partials, batch->counters,
                                 s) != cudaSuccess) {
            rc = TPFA_ECUDA;
            break;
          }
          ++w.launches;
        }
        Dirs qd, pd;
        for (int j = 0; j < gstored; ++j) {
          const size_t slot = (size_t)((head - 1 - j + w.m) % w.m);
          qd.v[j] = w.Q + slot * w.stride;
          pd.v[j] = w.P + slot * w.stride;
        }
        float* p = w.P + (size_t)head * w.stride;
        float* q = w.Q + (size_t)head * w.stride;
        launch_bdots(gstored, w.nchunks(), s, w.chunks_dev, w.flags, w.r, w.dinv, w.z, w.au, qd,
                     w.vec4, w.part);
        bfinish_dots_kernel<<<N, kT, 0, s>>>(w.cfirst_dev, w.ccount_dev, w.flags, w.part, gstored,
                                             w.uau, w.sc, head, w.m);
        launch_bdir(gstored, w.nchunks(), s, w.chunks_dev, w.flags, w.sc, w.r, w.dinv, w.z, pd, p,
                    w.vec4, w.part);
        if (launch_apply_batch(batch->inst_dev, N, batch->sweep_blocks, cf4, p, q, w.pq, w.flags,
                               kAct, batch->partials, batch->counters, s) != cudaSuccess) {
          rc = TPFA_ECUDA;
          break;
        }
        bfinish_alpha_kernel<<<N, kT, 0, s>>>(w.cfirst_dev, w.ccount_dev, w.flags, w.part, w.pq,
                                              w.sc, head, w.m);
        bupdate_kernel<<<w.nchunks(), kT, 0, s>>>(w.chunks_dev, w.flags, w.sc, w.e, w.r, p, q,
                                                  w.vec4, w.part);
        bfinish_rr_kernel<<<N, kT, 0, s>>>(w.cfirst_dev, w.ccount_dev, w.flags, w.part, w.sc,
                                           w.hist, pending);
        w.launches += 7;
        ++pending;
        ++giters;
        head = (head + 1) % w.m;
        if (gstored < w.m) ++gstored;
        if (pending < kCheckEvery) continue;
        // the host looks: r'r histories, flags, bad flags
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(w.hhist, w.hist, sizeof(double) * kCheckEvery * N,
                            cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(w.hflags, w.flags, sizeof(int) * N, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaMemcpyAsync(w.hsc, w.sc, sizeof(BScal) * N, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
          rc = TPFA_ECUDA;
          break;
        }
        bool changed = false;
        running = false;
        for (int i = 0; i < N; ++i) {
          blend[i] = 0;
          if (!(w.hflags[i] & kOuter) || status[i] != TPFA_OK) continue;
          BScal& S = w.hsc[i];
          if (first) hist[i].assign(1, S.rr0);
          double last = hist[i].empty() ? S.rr0 : hist[i].back();
          for (int k = 0; k < pending; ++k) {
            const double v = w.hhist[(size_t)i * kCheckEvery + k];
            if (v >= 0.0 || !std::isfinite(v)) {
              hist[i].push_back(v);
              last = v;
            }
          }
          const bool is_blend = (w.hflags[i] & kNet) != 0;
          const bool bad = S.bad != 0;
          // stagnation: the smallest r'r of the last kStallWindow iterations
          // is not 1% below the smallest before them
          bool stalled = false;
          if (is_blend && (w.hflags[i] & kAct) && (int)hist[i].size() > 2 * kStallWindow) {
            const size_t cut = hist[i].size() - kStallWindow;
            const double before = *std::min_element(hist[i].begin(), hist[i].begin() + cut);
            const double recent = *std::min_element(hist[i].begin() + cut, hist[i].end());
            stalled = recent > 0.99 * before;
          }
          if (!std::isfinite(last)) {
            if (is_blend) fb[i] = 1;
            status[i] = TPFA_ENONFINITE;
            w.hflags[i] &= ~kAct;
            changed = true;
          } else if (bad || stalled) {
            if (!is_blend) {
              status[i] = TPFA_EBREAKDOWN;
              w.hflags[i] &= ~kAct;
            } else {
              // drop the network for this instance from its current iterate
              fb[i] = 1;
              w.hflags[i] = (w.hflags[i] & (kAct | kOuter)) | fb_bits;
              S.stored = 0;
              S.bad = 0;
              S.c = 0.0;
              hist[i].assign(1, last);
            }
            changed = true;
          }
          blend[i] = (w.hflags[i] & kAct) && (w.hflags[i] & kNet);
          if (w.hflags[i] & kAct) running = true;
        }
        first = false;
        pending = 0;
        if (changed &&
            (cudaMemcpyAsync(w.sc, w.hsc, sizeof(BScal) * N, cudaMemcpyHostToDevice, s) !=
                 cudaSuccess ||
             cudaMemcpyAsync(w.flags, w.hflags, sizeof(int) * N, cudaMemcpyHostToDevice, s) !=
                 cudaSuccess)) {
          rc = TPFA_ECUDA;
          break;
        }
        // the networks run on the members that still iterate with them
        rc = update_active(bn, blend, batch->off, w);
        if (rc) break;
        if (giters > maxit + kCheckEvery) break;  // every instance has its own limit below this
      }
      if (rc) break;
      // a partial check window: fetch the iteration counts
      if (cudaMemcpyAsync(w.hsc, w.sc, sizeof(BScal) * N, cudaMemcpyDeviceToHost, s) !=
              cudaSuccess ||
          cudaMemcpyAsync(w.hflags, w.flags, sizeof(int) * N, cudaMemcpyDeviceToHost, s) !=
              cudaSuccess) {
        rc = TPFA_ECUDA;
        break;
      }
      bcorrect_kernel<<<w.nchunks(), kT, 0, s>>>(w.chunks_dev, w.flags, w.sc, w.e, x);
      ++w.launches;
      if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
        rc = TPFA_ECUDA;
        break;
      }
      inner_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - ti)
                      .count();
      for (int i = 0; i < N; ++i) {
        if (!todo[i]) continue;
        iters[i] += w.hsc[i].iters;
        ++outer[i];
        if (status[i] != TPFA_OK) todo[i] = 0;  // broke down: no further residual
      }
      rc = residuals(todo);
    }
    if (rc == TPFA_OK && n_nets > 0 && tpfa_net_status(stream) != TPFA_OK) rc = TPFA_EINTERNAL;
    launches = w.launches;
  }
  for (int i = 0; i < N; ++i)
    if (status[i] == TPFA_OK && !(rel[i] <= tol)) status[i] = TPFA_NOTCONV;
  const double ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  int worst = TPFA_OK;
  int64_t it_sum = 0;
  int out_max = 0;
  double rel_max = 0.0;
  for (int i = 0; i < N; ++i) {
    if (infos) {
      tpfa_cg_info& f = infos[i];
      std::memset(&f, 0, sizeof(f));
      f.iters = iters[i];
      f.outer = outer[i];
      f.status = rc ? rc : status[i];
      f.rel_res_inner = NAN;
      f.rel_res_fp64 = rel[i];
      f.inner_ms = inner_ms;
      f.total_ms = ms;
      f.kernel_launches = launches;
    }
    if (fell_back) fell_back[i] = fb[i];
    if (status[i] < 0 && (worst >= 0 || status[i] < worst)) worst = status[i];
    else if (status[i] > 0 && worst == TPFA_OK) worst = status[i];
    it_sum += iters[i];
    if (outer[i] > out_max) out_max = outer[i];
    if (rel[i] > rel_max) rel_max = rel[i];
  }
  if (total) {
    std::memset(total, 0, sizeof(*total));
    total->iters = it_sum;
    total->outer = out_max;
    total->status = rc ? rc : worst;
    total->rel_res_fp64 = rel_max;
    total->rel_res_inner = NAN;
    total->inner_ms = inner_ms;
    total->total_ms = ms;
    total->kernel_launches = launches;
  }
  return rc ? rc : worst;
}
