// Flexible conjugate gradients (Notay 2000, one retained direction) with the
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
//   z_k = M(r_k);  p_0 = z_0,  p_k = z_k - (z_k' q_{k-1} / p_{k-1}' q_{k-1}) p_{k-1};
//   q_k = A p_k;  alpha_k = p_k' r_k / p_k' q_k;  e += alpha_k p_k;  r -= alpha_k q_k.
// For a fixed SPD preconditioner this generates the PCG iterates; for the
// network, which is neither linear nor symmetric, the explicit
// A-orthogonalisation against the previous direction keeps the method
// convergent.  If p'q <= 0, a value is not finite, or the residual stops
// decreasing, the solve falls back to the identity preconditioner (plain CG)
// from the current iterate.
//
// Dot products: FP64 per-thread sums, per-block partials in a fixed order,
// added on the host in block order (bit-reproducible).
#include <chrono>
#include <cmath>
#include <vector>

#include "tpfa_internal.cuh"

struct tpfa_unet;
extern "C" int tpfa_unet_forward(tpfa_unet* u, const float* r, const float* lnk, float* z,
                                 void* stream);
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

// partial a'b
__global__ void dot_kernel(const float* __restrict__ a, const float* __restrict__ b, int64_t n,
                           double* part) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
    s += (double)a[i] * b[i];
  block_sum3(s, 0.0, 0.0, part);
}

// p = z + beta p (p = z when first); partial p'r
__global__ void dir_kernel(const float* __restrict__ z, float* __restrict__ p,
                           const float* __restrict__ r, float beta, int first, int64_t n,
                           double* part) {
  double pr = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
    const float v = first ? z[i] : fmaf(beta, p[i], z[i]);
    p[i] = v;
    pr += (double)v * r[i];
  }
  block_sum3(pr, 0.0, 0.0, part);
}

// e += alpha p; r -= alpha q; partial r'r
__global__ void update_kernel(float* __restrict__ e, float* __restrict__ r,
                              const float* __restrict__ p, const float* __restrict__ q, float alpha,
                              int64_t n, double* part) {
  double rr = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
    e[i] = fmaf(alpha, p[i], e[i]);
    const float v = fmaf(-alpha, q[i], r[i]);
    r[i] = v;
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

__global__ void copy_kernel(const float* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
    b[i] = a[i];
}

// partials of u'r and (Au)'(r / D)
__global__ void blend_dots_kernel(const float* __restrict__ u, const float* __restrict__ r,
                                  const float* __restrict__ au, const float4* __restrict__ coef,
                                  int64_t n, double* part) {
  double s0 = 0.0, s1 = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
    const float ri = r[i];
    s0 += (double)u[i] * ri;
    s1 += (double)au[i] * (ri / coef[i].w);
  }
  block_sum3(s0, s1, 0.0, part);
}

// z = r / D + c u (in place over u)
__global__ void blend_kernel(float* __restrict__ uz, const float* __restrict__ r,
                             const float4* __restrict__ coef, float c, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
    uz[i] = fmaf(c, uz[i], r[i] / coef[i].w);
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
  float *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *e = nullptr, *au = nullptr;
  double* r64 = nullptr;
  double* uau = nullptr;     // dev, 1
  double* part = nullptr;    // dev, 3 * nb
  double* hpart = nullptr;   // pinned host
  double* norms = nullptr;   // dev, 2
  double* hnorms = nullptr;  // pinned
  double* pq = nullptr;      // dev, 1
  int64_t launches = 0;

  bool alloc() {
    return cudaMalloc(&r, n * 4) == cudaSuccess && cudaMalloc(&z, n * 4) == cudaSuccess &&
           cudaMalloc(&p, n * 4) == cudaSuccess && cudaMalloc(&q, n * 4) == cudaSuccess &&
           cudaMalloc(&e, n * 4) == cudaSuccess && cudaMalloc(&r64, n * 8) == cudaSuccess &&
           cudaMalloc(&au, n * 4) == cudaSuccess && cudaMalloc(&uau, 8) == cudaSuccess &&
           cudaMalloc(&part, sizeof(double) * 3 * nb) == cudaSuccess &&
           cudaMalloc(&norms, 16) == cudaSuccess && cudaMalloc(&pq, 8) == cudaSuccess &&
           cudaMallocHost(&hpart, sizeof(double) * 3 * nb) == cudaSuccess &&
           cudaMallocHost(&hnorms, 16) == cudaSuccess;
  }
  ~Work() {
    if (s) cudaStreamSynchronize(s);
    cudaFree(r);
    cudaFree(z);
    cudaFree(p);
    cudaFree(q);
    cudaFree(e);
    cudaFree(au);
    cudaFree(uau);
    cudaFree(r64);
    cudaFree(part);
    cudaFree(norms);
    cudaFree(pq);
    cudaFreeHost(hpart);
    cudaFreeHost(hnorms);
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
  bool fetch_scalar(const double* dev, double* out) {
    if (cudaMemcpyAsync(hnorms, dev, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return false;
    *out = hnorms[0];
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

// Inner FCG on A e = r (r, e already set, r'r = rr0); returns a TPFA_* error or
// TPFA_OK, with res->status = TPFA_EBREAKDOWN if plain CG itself broke down.
int fcg_inner(tpfa_ctx* c, tpfa_unet* net, const float* coef, const float* lnk, Work& w,
              double rr0, double target, int64_t maxit, Result* res) {
  double d3[3];
  double rr = rr0, pq_prev = 0.0;
  bool first = true;
  bool precond_on = net != nullptr && !res->fallback;
  std::vector<double> hist(1, rr);
  while (res->iters < maxit && rr > target * target * rr0) {
    if (precond_on) {
      // z = D^-1 r + c u, u = net(r), c the A-norm-optimal weight
      int rc = tpfa_unet_forward(net, w.r, lnk, w.z, w.s);
      if (rc) return rc;
      w.launches += 15;
      rc = tpfa_apply(c, coef, w.z, w.au, w.uau, w.s);
      if (rc) return rc;
      blend_dots_kernel<<<w.nb, kT, 0, w.s>>>(w.z, w.r, w.au, reinterpret_cast<const float4*>(coef),
                                               w.n, w.part);
      w.launches += 2;
      double uau = 0.0;
      if (!w.fetch(d3) || !w.fetch_scalar(w.uau, &uau)) return TPFA_ECUDA;
      double cw = uau > 0.0 && std::isfinite(uau) ? (d3[0] - d3[1]) / uau : 0.0;
      if (!std::isfinite(cw)) cw = 0.0;
      blend_kernel<<<w.nb, kT, 0, w.s>>>(w.z, w.r, reinterpret_cast<const float4*>(coef), (float)cw,
                                          w.n);
      ++w.launches;
    } else {
      copy_kernel<<<w.nb, kT, 0, w.s>>>(w.r, w.z, w.n);
      ++w.launches;
    }
    float beta = 0.f;
    if (!first) {
      dot_kernel<<<w.nb, kT, 0, w.s>>>(w.z, w.q, w.n, w.part);
      ++w.launches;
      if (!w.fetch(d3)) return TPFA_ECUDA;
      beta = (float)(-d3[0] / pq_prev);
    }
    dir_kernel<<<w.nb, kT, 0, w.s>>>(w.z, w.p, w.r, beta, first ? 1 : 0, w.n, w.part);
    ++w.launches;
    if (!w.fetch(d3)) return TPFA_ECUDA;
    const double pr = d3[0];
    int rc = tpfa_apply(c, coef, w.p, w.q, w.pq, w.s);
    if (rc) return rc;
    ++w.launches;
    double pq = 0.0;
    if (!w.fetch_scalar(w.pq, &pq)) return TPFA_ECUDA;
    const bool bad = !(pq > 0.0) || !std::isfinite(pq) || !std::isfinite(pr) ||
                     !std::isfinite((double)beta);
    // stagnation: less than 1% reduction of r'r over the last 50 iterations
    const bool stalled = precond_on && hist.size() > 50 && rr > 0.99 * hist[hist.size() - 51];
    if (bad || stalled) {
      if (!precond_on) {
        res->status = TPFA_EBREAKDOWN;
        return TPFA_OK;
      }
      precond_on = false;  // plain CG from the current iterate
      res->fallback = true;
      first = true;
      continue;
    }
    const float alpha = (float)(pr / pq);
    update_kernel<<<w.nb, kT, 0, w.s>>>(w.e, w.r, w.p, w.q, alpha, w.n, w.part);
    ++w.launches;
    if (!w.fetch(d3)) return TPFA_ECUDA;
    rr = d3[0];
    hist.push_back(rr);
    pq_prev = pq;
    first = false;
    ++res->iters;
  }
  return TPFA_OK;
}

int fcg_outer(tpfa_ctx* c, tpfa_unet* net, const float* coef, const double* coef64,
              const float* lnk, const double* b, double* x, double tol, int64_t maxit,
              double inner_rtol, int max_outer, Work& w, Result* res) {
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
    rc = fcg_inner(c, net, coef, lnk, w, d3[0], target, maxit, res);
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
  if (net != nullptr) {
    int d4[4];
    int64_t d3[3];
    tpfa_unet_shape(net, d4);
    tpfa::ctx_dims(c, d3);
    if (d4[0] != d3[0] || d4[1] != d3[1] || d4[2] != d3[2] || d4[3] != 1) return TPFA_EINVAL;
  }
  const double inner_rtol = tpfa::ctx_option(c, TPFA_OPT_INNER_RTOL);
  const int max_outer = (int)tpfa::ctx_option(c, TPFA_OPT_MAX_OUTER);
  Result res;
  int rc;
  int64_t launches = 0;
  {
    Work w;
    w.s = (cudaStream_t)stream;
    w.n = n;
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    w.nb = 4 * nsm;
    if (!w.alloc()) {
      cudaGetLastError();
      rc = TPFA_ENOMEM;
    } else {
      rc = fcg_outer(c, net, coef, coef64, lnk, b, x, tol, maxit, inner_rtol, max_outer, w, &res);
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
