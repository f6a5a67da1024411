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

#include "fcg_common.cuh"

namespace {

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
// fdots: the totals from the fused operator (u'Au, then s0, s1, a_j, b_j)
// instead of the block partials
__global__ void finish_dots_kernel(const double* __restrict__ part, int nb, int M, int net,
                                   const double* __restrict__ uau, Scal* sc, int head, int m,
                                   const double* __restrict__ fdots) {
  __shared__ double tot[2 + 2 * kMaxDirs];
  const int K = 2 + 2 * M;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (fdots != nullptr) {
    if (threadIdx.x < K) tot[threadIdx.x] = fdots[1 + threadIdx.x];
  } else {
    for (int k = warp; k < K; k += nw) {
      double t = 0.0;
      for (int b = lane; b < nb; b += 32) t += part[(size_t)b * K + k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      if (lane == 0) tot[k] = t;
    }
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
  // network on the 2^levels coarser grid: the restricted residual and the
  // network's output there (index levels), ln K on the network's grid
  int levels = 0;
  int dims[3] = {0, 0, 0};
  float* rl[kMaxLevels + 1] = {};
  float* ul[kMaxLevels + 1] = {};
  float* lnkc = nullptr;
  int64_t launches = 0;
  // the TMA-staged operator fused with the blend's dot products (a batch of
  // one): maps {coefficients, z, P slots, r, M^-1, Q slots}
  bool fused = false;
  CUtensorMap* fmaps = nullptr;
  tpfa::TmaInst* finst = nullptr;
  int* fact = nullptr;
  unsigned int* fcnt = nullptr;
  double* fpart = nullptr;
  double* fdots = nullptr;
  int64_t fblocks = 0;
  int own0 = 0;

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
    cudaFree(fmaps);
    cudaFree(finst);
    cudaFree(fact);
    cudaFree(fcnt);
    cudaFree(fpart);
    cudaFree(fdots);
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

// the network term u of the blend (into w.z) and, unless the fused operator
// takes it, A u (into w.au, u'Au into w.uau)
int network_term(tpfa_ctx* c, tpfa_unet* net, const float* coef, const float* lnk, Work& w,
                 bool with_apply) {
  int rc;
  if (w.levels > 0) {
    const int L = w.levels;
    launch_restrict_levels(L, w.nb, w.s, w.r, w.rl[L], w.dims[0], w.dims[1], w.dims[2], 1,
                           nullptr, 0, 0, 0);
    rc = tpfa_unet_forward(net, w.rl[L], w.lnkc, w.ul[L], w.s);
    if (rc) return rc;
    launch_prolong_levels(L, w.nb, w.s, w.ul[L], w.z, w.dims[0], w.dims[1], w.dims[2], 1, nullptr,
                          0, 0, 0, true);
    w.launches += 17;
  } else {
    rc = tpfa_unet_forward(net, w.r, lnk, w.z, w.s);
    if (rc) return rc;
    w.launches += 15;
  }
  if (!with_apply) return TPFA_OK;
  rc = tpfa_apply(c, coef, w.z, w.au, w.uau, w.s);
  ++w.launches;
  return rc;
}

// Set up the fused operator when tpfa_apply would take the TMA-staged kernel.
int setup_fused(const tpfa_ctx* c, const float* coef, Work& w) {
  using namespace tpfa;
  TmaPlan p;
  Grid g;
  if (!ctx_apply_tma_plan(c, &p, &g, true) || reinterpret_cast<uintptr_t>(coef) % 16 != 0 ||
      w.m > kMaxDirs)
    return TPFA_OK;
  const int per = 4 + 2 * w.m;
  std::vector<CUtensorMap> maps(per);
  std::vector<const float*> in(1 + w.m), own(2 + w.m);
  in[0] = w.z;
  own[0] = w.r;
  own[1] = w.dinv;
  for (int k = 0; k < w.m; ++k) {
    in[1 + k] = w.P + (size_t)k * w.slot_stride();
    own[2 + k] = w.Q + (size_t)k * w.slot_stride();
  }
  if (!make_apply_maps(g, p, coef, in.data(), 1 + w.m, maps.data()) ||
      !make_own_maps(g, p, own.data(), 2 + w.m, maps.data() + 2 + w.m))
    return TPFA_OK;  // the unfused passes
  TmaInst I{};
  I.g = g;
  I.zc = p.zc;
  I.nbx = (int)p.nbx;
  I.nby = (int)p.nby;
  I.id = 0;
  I.off = 0;
  I.bstart = 0;
  I.nblocks = p.nblocks;
  const int one = 1;
  if (cudaMalloc(&w.fmaps, sizeof(CUtensorMap) * per) != cudaSuccess ||
      cudaMalloc(&w.finst, sizeof(TmaInst)) != cudaSuccess ||
      cudaMalloc(&w.fact, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&w.fcnt, sizeof(unsigned int)) != cudaSuccess ||
      cudaMalloc(&w.fpart, sizeof(double) * p.nblocks * (3 + 2 * kApplyMaxDirs)) != cudaSuccess ||
      cudaMalloc(&w.fdots, sizeof(double) * kApplyDotsStride) != cudaSuccess) {
    cudaGetLastError();
    return TPFA_ENOMEM;
  }
  I.maps = w.fmaps;
  if (cudaMemcpyAsync(w.fmaps, maps.data(), sizeof(CUtensorMap) * per, cudaMemcpyHostToDevice,
                      w.s) != cudaSuccess ||
      cudaMemcpyAsync(w.finst, &I, sizeof(TmaInst), cudaMemcpyHostToDevice, w.s) != cudaSuccess ||
      cudaMemcpyAsync(w.fact, &one, sizeof(int), cudaMemcpyHostToDevice, w.s) != cudaSuccess ||
      cudaMemsetAsync(w.fcnt, 0, sizeof(unsigned int), w.s) != cudaSuccess ||
      cudaStreamSynchronize(w.s) != cudaSuccess)
    return TPFA_ECUDA;
  w.fused = true;
  w.fblocks = p.nblocks;
  w.own0 = 2 + w.m;
  return TPFA_OK;
}

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
    Dirs qd, pd;
    int qmap[kMaxDirs];
    for (int j = 0; j < stored; ++j) {
      const size_t slot = (size_t)((head - 1 - j + m) % m);
      qd.v[j] = w.Q + slot * w.slot_stride();
      pd.v[j] = w.P + slot * w.slot_stride();
      qmap[j] = (int)slot;
    }
    // with the network, the TMA-staged operator A u also forms the dot
    // products (A u itself is not stored)
    const bool fused = with_net && w.fused && stored <= tpfa::kApplyMaxDirs;
    if (with_net) {
      int rc = network_term(c, net, coef, lnk, w, !fused);
      if (rc) return rc;
      if (fused) {
        if (launch_apply_dots_tma_batch(w.finst, 1, w.fblocks, 0, w.fact, 1, w.own0, qmap, stored,
                                        w.uau, w.fdots, w.fpart, w.fcnt, w.s) != cudaSuccess)
          return TPFA_ECUDA;
        ++w.launches;
      }
    }
    if (fused) {
      finish_dots_kernel<<<1, kT, 0, w.s>>>(w.part, w.nb, stored, 1, w.uau, w.sc, head, m, w.fdots);
    } else if (stored > 0 || with_net) {
      launch_dots(stored, w.nb, w.s, w.r, w.dinv, w.z, w.au, qd, jac, with_net, w.n, w.part);
      finish_dots_kernel<<<1, kT, 0, w.s>>>(w.part, w.nb, stored, with_net, w.uau, w.sc, head, m,
                                            nullptr);
    } else {
      finish_dots_kernel<<<1, kT, 0, w.s>>>(w.part, 0, 0, 0, w.uau, w.sc, head, m, nullptr);
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
      const int L = w.levels;
      const size_t bytes = (size_t)(n >> (3 * L)) * 4;
      ok = cudaMalloc(&w.rl[L], bytes) == cudaSuccess && cudaMalloc(&w.ul[L], bytes) == cudaSuccess &&
           cudaMalloc(&w.lnkc, bytes) == cudaSuccess;
      if (ok) {
        // ln K on the network's grid: the mean over each 2^levels block
        launch_restrict_levels(L, w.nb, w.s, lnk, w.lnkc, w.dims[0], w.dims[1], w.dims[2], 1,
                               nullptr, 0, 0, 0);
        ok = cudaGetLastError() == cudaSuccess;
      }
    }
    if (ok && net != nullptr) ok = setup_fused(c, coef, w) == TPFA_OK;
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
  // the kernel writes two x-neighbours at a time
  if (!tpfa::dev_ok(fine, n * 4, 8, dev) || !tpfa::dev_ok(coarse, n / 8 * 4, 4, dev))
    return TPFA_EINVAL;
  const int nb = (int)((n + kT - 1) / kT < 4096 ? (n + kT - 1) / kT : 4096);
  prolong2_kernel<<<nb, kT, 0, (cudaStream_t)stream>>>(coarse, fine, nx, ny, nz, ns, nullptr, 0,
                                                       0, 0);
  return cudaGetLastError() == cudaSuccess ? TPFA_OK : TPFA_ECUDA;
}

// The 2^levels coarser grid in one pass: the block means, bit-identical to
// `levels` successive tpfa_restrict2 calls with scale 1/8.  Asynchronous.
extern "C" int tpfa_restrict_levels(const float* fine, float* coarse, int nx, int ny, int nz, int ns,
                                    int levels, void* stream) {
  if (levels < 1 || levels > kMaxLevels || ns < 1) return TPFA_EINVAL;
  const int f = 1 << levels;
  if (nx < f || ny < f || nz < f || nx % f || ny % f || nz % f) return TPFA_EINVAL;
  if ((double)nx * ny * nz * ns >= 2147483647.0) return TPFA_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return TPFA_ECUDA;
  const size_t n = (size_t)nx * ny * nz * ns, nc = n >> (3 * levels);
  if (!tpfa::dev_ok(fine, n * 4, 8, dev) || !tpfa::dev_ok(coarse, nc * 4, 4, dev))
    return TPFA_EINVAL;
  const int nb = (int)((nc + kT - 1) / kT < 4096 ? (nc + kT - 1) / kT : 4096);
  launch_restrict_levels(levels, nb, (cudaStream_t)stream, fine, coarse, nx, ny, nz, ns, nullptr, 0,
                         0, 0);
  return cudaGetLastError() == cudaSuccess ? TPFA_OK : TPFA_ECUDA;
}

// fine = value of each cell's ancestor on the 2^levels coarser grid (levels
// nearest prolongations in one pass).  Asynchronous.
extern "C" int tpfa_prolong_levels(const float* coarse, float* fine, int nx, int ny, int nz, int ns,
                                   int levels, void* stream) {
  if (levels < 1 || levels > kMaxLevels || ns < 1) return TPFA_EINVAL;
  const int f = 1 << levels;
  if (nx < f || ny < f || nz < f || nx % f || ny % f || nz % f) return TPFA_EINVAL;
  if ((double)nx * ny * nz * ns >= 2147483647.0) return TPFA_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return TPFA_ECUDA;
  const size_t n = (size_t)nx * ny * nz * ns, nc = n >> (3 * levels);
  if (!tpfa::dev_ok(fine, n * 4, 8, dev) || !tpfa::dev_ok(coarse, nc * 4, 4, dev))
    return TPFA_EINVAL;
  const int nb = (int)((n / 2 + kT - 1) / kT < 4096 ? (n / 2 + kT - 1) / kT : 4096);
  launch_prolong_levels(levels, nb, (cudaStream_t)stream, coarse, fine, nx, ny, nz, ns, nullptr, 0,
                        0, 0, true);
  return cudaGetLastError() == cudaSuccess ? TPFA_OK : TPFA_ECUDA;
}
