// The learned preconditioner's network: a 3-level 3D U-Net (Ronneberger,
// Fischer and Brox 2015) with 16/32/64 channels, 3x3x3 convolutions, 2x2x2
// average pooling, nearest upsampling and additive skip connections:
//
//   e0 = relu(conv(in; W0 2->16))          level 0 (full resolution)
//   e1 = relu(conv(pool(e0); W1 16->32))   level 1 (half)
//   e2 = relu(conv(pool(e1); W2 32->64))   level 2 (quarter)
//   d2 = relu(conv(e2; W3 64->32))         level 2
//   s1 = up(d2) + e1                       level 1
//   d1 = relu(conv(s1; W4 32->16))         level 1
//   s0 = up(d1) + e0                       level 0
//   d0 = relu(conv(s0; W5 16->16))         level 0
//   z  = conv(d0; W6 16->1)                level 0
//
// with in = (r / rms(r), ln K) and M(r) = rms(r) z, so that M is homogeneous
// of degree one in r.  Every convolution runs on the tensor cores (conv3d.cu);
// the 2-channel input and the 1-channel output are carried as 16 channels
// whose extra weights are zero.  Activations are BF16 in the haloed
// channels-last layout (net_internal.cuh); parameters are an FP32 vector,
// converted to BF16 (forward layout and tap-flipped transposed layout for the
// input gradients) by tpfa_unet_set_params.
#include <cuda_bf16.h>

#include <cstring>
#include <new>

#include "net_internal.cuh"
#include "tpfa_internal.cuh"

using tpfa::net::Vol;
using tpfa::net::make_vol;

namespace {

constexpr int kLayers = 7;
struct LayerDef {
  int cin, cout;    // true shape
  int cip, cop;     // shape the kernels run (16-channel padding)
  int level;
};
constexpr LayerDef kDefs[kLayers] = {{2, 16, 16, 16, 0},  {16, 32, 16, 32, 1}, {32, 64, 32, 64, 2},
                                     {64, 32, 64, 32, 2}, {32, 16, 32, 16, 1}, {16, 16, 16, 16, 0},
                                     {16, 1, 16, 16, 0}};

constexpr int kThreads = 256;

// offsets of W_i and b_i in the flat FP32 parameter vector
struct ParamLayout {
  int64_t w[kLayers], b[kLayers], total;
  ParamLayout() {
    int64_t o = 0;
    for (int i = 0; i < kLayers; ++i) {
      w[i] = o;
      o += 27LL * kDefs[i].cout * kDefs[i].cin;
      b[i] = o;
      o += kDefs[i].cout;
    }
    total = o;
  }
};
const ParamLayout kParams;

__device__ __forceinline__ float bf(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }
__device__ __forceinline__ uint16_t tobf(float f) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(f));
}
__device__ __forceinline__ bool positive(uint16_t h) { return (h & 0x8000u) == 0 && (h & 0x7fffu); }

// compact cell index c = i + nx (j + ny (k + nz s)) -> haloed voxel index
__device__ __forceinline__ int halo_index(const Vol& g, int c, int* sample) {
  const int i = c % g.nx;
  int t = c / g.nx;
  const int j = t % g.ny;
  t /= g.ny;
  const int k = t % g.nz;
  const int s = t / g.nz;
  if (sample) *sample = s;
  return ((s * g.dp + k + 1) * g.hp + j + 1) * g.wp + i + 1;
}

// parent (coarse) voxel of fine compact cell c
__device__ __forceinline__ int parent_index(const Vol& gf, const Vol& gc, int c) {
  const int i = c % gf.nx;
  int t = c / gf.nx;
  const int j = t % gf.ny;
  t /= gf.ny;
  const int k = t % gf.nz;
  const int s = t / gf.nz;
  return ((s * gc.dp + k / 2 + 1) * gc.hp + j / 2 + 1) * gc.wp + i / 2 + 1;
}

__host__ __device__ __forceinline__ int cells(const Vol& g) { return g.nx * g.ny * g.nz * g.ns; }
int blocks_for(long long n) { return (int)((n + kThreads - 1) / kThreads); }

// ---- per-sample root mean square (fixed-order reduction) ------------------
constexpr int kRmsBlocks = 1024;  // most blocks per sample

// blocks per sample of the sum of squares: about eight cells per thread, so
// that small samples do not launch mostly idle blocks (depends only on the
// sample's size, so a sample's rms is the same alone or in a batch)
int rms_blocks(int per) {
  const int b = (per + kThreads * 8 - 1) / (kThreads * 8);
  return b < 1 ? 1 : (b > kRmsBlocks ? kRmsBlocks : b);
}

__global__ void sumsq_partial_kernel(const float* __restrict__ r, int n, double* partials) {
  __shared__ double sh[kThreads];
  const int s = blockIdx.y;
  const float* rs = r + (size_t)s * n;
  double acc = 0.0;
  for (int c = blockIdx.x * kThreads + threadIdx.x; c < n; c += gridDim.x * kThreads) {
    const double v = rs[c];
    acc += v * v;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[s * gridDim.x + blockIdx.x] = sh[0];
}

// one block per sample: strided sums, then a tree, in a fixed order
__global__ void rms_finish_kernel(const double* partials, int nb, int n, float* rms) {
  __shared__ double sh[kThreads];
  const int s = blockIdx.x;
  double t = 0.0;
  for (int b = threadIdx.x; b < nb; b += kThreads) t += partials[s * nb + b];
  sh[threadIdx.x] = t;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double v = sqrt(sh[0] / n);
    rms[s] = v > 0.0 ? (float)v : 1.0f;  // a zero residual maps to a zero input
  }
}

// ---- element-wise kernels ----------------------------------------------------
// in16[v] = (bf16(r/rms), bf16(ln K), 0, ..., 0)
__global__ void prep_input_kernel(const float* __restrict__ r, const float* __restrict__ lnk,
                                  const float* __restrict__ rms, uint16_t* __restrict__ in16,
                                  Vol g) {
  const int c = blockIdx.x * kThreads + threadIdx.x;
  if (c >= cells(g)) return;
  int s;
  const int v = halo_index(g, c, &s);
  const uint32_t w0 = (uint32_t)tobf(r[c] / rms[s]) | ((uint32_t)tobf(lnk[c]) << 16);
  uint4* o = reinterpret_cast<uint4*>(in16 + (size_t)v * 16);
  o[0] = make_uint4(w0, 0, 0, 0);
  o[1] = make_uint4(0, 0, 0, 0);
}

// z[c] = rms * out16[v][0]
__global__ void out_extract_kernel(const uint16_t* __restrict__ o16, const float* __restrict__ rms,
                                   float* __restrict__ z, Vol g) {
  const int c = blockIdx.x * kThreads + threadIdx.x;
  if (c >= cells(g)) return;
  int s;
  const int v = halo_index(g, c, &s);
  z[c] = rms[s] * bf(o16[(size_t)v * 16]);
}

// g16[v] = (bf16(rms * gz[c]), 0, ..., 0): gradient of the network output
__global__ void grad_in_kernel(const float* __restrict__ gz, const float* __restrict__ rms,
                               uint16_t* __restrict__ g16, Vol g) {
  const int c = blockIdx.x * kThreads + threadIdx.x;
  if (c >= cells(g)) return;
  int s;
  const int v = halo_index(g, c, &s);
  uint4* o = reinterpret_cast<uint4*>(g16 + (size_t)v * 16);
  o[0] = make_uint4((uint32_t)tobf(rms[s] * gz[c]), 0, 0, 0);
  o[1] = make_uint4(0, 0, 0, 0);
}

// coarse[V] = mean of the 8 children; one thread per (coarse cell, 8 channels)
__global__ void pool_kernel(const uint16_t* __restrict__ fine, uint16_t* __restrict__ coarse,
                            int C, Vol gf, Vol gc) {
  const int kc = C / 8;
  const int id = blockIdx.x * kThreads + threadIdx.x;
  if (id >= cells(gc) * kc) return;
  const int cc = id / kc, ch = (id % kc) * 8;
  const int i = cc % gc.nx;
  int t = cc / gc.nx;
  const int j = t % gc.ny;
  t /= gc.ny;
  const int k = t % gc.nz;
  const int s = t / gc.nz;
  float a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        const int vf = ((s * gf.dp + 2 * k + dz + 1) * gf.hp + 2 * j + dy + 1) * gf.wp + 2 * i + dx + 1;
        const uint4 u = *reinterpret_cast<const uint4*>(fine + (size_t)vf * C + ch);
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          a[2 * h] += bf((uint16_t)(w[h] & 0xffff));
          a[2 * h + 1] += bf((uint16_t)(w[h] >> 16));
        }
      }
  const int vc = ((s * gc.dp + k + 1) * gc.hp + j + 1) * gc.wp + i + 1;
  uint32_t o[4];
#pragma unroll
  for (int h = 0; h < 4; ++h)
    o[h] = (uint32_t)tobf(a[2 * h] * 0.125f) | ((uint32_t)tobf(a[2 * h + 1] * 0.125f) << 16);
  *reinterpret_cast<uint4*>(coarse + (size_t)vc * C + ch) = make_uint4(o[0], o[1], o[2], o[3]);
}

// out[v] = skip[v] + coarse[parent(v)]  (nearest upsampling plus skip)
__global__ void upadd_kernel(const uint16_t* __restrict__ coarse, const uint16_t* __restrict__ skip,
                             uint16_t* __restrict__ out, int C, Vol gf, Vol gc) {
  const int kc = C / 8;
  const int id = blockIdx.x * kThreads + threadIdx.x;
  if (id >= cells(gf) * kc) return;
  const int c = id / kc, ch = (id % kc) * 8;
  const int vf = halo_index(gf, c, nullptr);
  const int vc = parent_index(gf, gc, c);
  const uint4 a = *reinterpret_cast<const uint4*>(skip + (size_t)vf * C + ch);
  const uint4 b = *reinterpret_cast<const uint4*>(coarse + (size_t)vc * C + ch);
  const uint32_t wa[4] = {a.x, a.y, a.z, a.w}, wb[4] = {b.x, b.y, b.z, b.w};
  uint32_t o[4];
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const float lo = bf((uint16_t)(wa[h] & 0xffff)) + bf((uint16_t)(wb[h] & 0xffff));
    const float hi = bf((uint16_t)(wa[h] >> 16)) + bf((uint16_t)(wb[h] >> 16));
    o[h] = (uint32_t)tobf(lo) | ((uint32_t)tobf(hi) << 16);
  }
  *reinterpret_cast<uint4*>(out + (size_t)vf * C + ch) = make_uint4(o[0], o[1], o[2], o[3]);
}

// coarse[V] = (sum of the 8 children of fine) * (mask[V] > 0): adjoint of the
// upsampling followed by the ReLU derivative of the coarse layer
__global__ void upadj_mask_kernel(const uint16_t* __restrict__ fine, const uint16_t* __restrict__ mask,
                                  uint16_t* __restrict__ coarse, int C, Vol gf, Vol gc) {
  const int kc = C / 8;
  const int id = blockIdx.x * kThreads + threadIdx.x;
  if (id >= cells(gc) * kc) return;
  const int cc = id / kc, ch = (id % kc) * 8;
  const int i = cc % gc.nx;
  int t = cc / gc.nx;
  const int j = t % gc.ny;
  t /= gc.ny;
  const int k = t % gc.nz;
  const int s = t / gc.nz;
  float a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        const int vf = ((s * gf.dp + 2 * k + dz + 1) * gf.hp + 2 * j + dy + 1) * gf.wp + 2 * i + dx + 1;
        const uint4 u = *reinterpret_cast<const uint4*>(fine + (size_t)vf * C + ch);
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          a[2 * h] += bf((uint16_t)(w[h] & 0xffff));
          a[2 * h + 1] += bf((uint16_t)(w[h] >> 16));
        }
      }
  const int vc = ((s * gc.dp + k + 1) * gc.hp + j + 1) * gc.wp + i + 1;
  const uint4 m = *reinterpret_cast<const uint4*>(mask + (size_t)vc * C + ch);
  const uint32_t wm[4] = {m.x, m.y, m.z, m.w};
  uint32_t o[4];
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const float lo = positive((uint16_t)(wm[h] & 0xffff)) ? a[2 * h] : 0.f;
    const float hi = positive((uint16_t)(wm[h] >> 16)) ? a[2 * h + 1] : 0.f;
    o[h] = (uint32_t)tobf(lo) | ((uint32_t)tobf(hi) << 16);
  }
  *reinterpret_cast<uint4*>(coarse + (size_t)vc * C + ch) = make_uint4(o[0], o[1], o[2], o[3]);
}

// out[v] = (skip[v] + coarse[parent(v)] / 8) * (mask[v] > 0): the skip
// gradient plus the adjoint of average pooling, then the ReLU derivative
__global__ void pooladj_add_mask_kernel(const uint16_t* __restrict__ skip,
                                        const uint16_t* __restrict__ coarse,
                                        const uint16_t* __restrict__ mask, uint16_t* __restrict__ out,
                                        int C, Vol gf, Vol gc) {
  const int kc = C / 8;
  const int id = blockIdx.x * kThreads + threadIdx.x;
  if (id >= cells(gf) * kc) return;
  const int c = id / kc, ch = (id % kc) * 8;
  const int vf = halo_index(gf, c, nullptr);
  const int vc = parent_index(gf, gc, c);
  const uint4 a = *reinterpret_cast<const uint4*>(skip + (size_t)vf * C + ch);
  const uint4 b = *reinterpret_cast<const uint4*>(coarse + (size_t)vc * C + ch);
  const uint4 m = *reinterpret_cast<const uint4*>(mask + (size_t)vf * C + ch);
  const uint32_t wa[4] = {a.x, a.y, a.z, a.w}, wb[4] = {b.x, b.y, b.z, b.w},
                 wm[4] = {m.x, m.y, m.z, m.w};
  uint32_t o[4];
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    float lo = bf((uint16_t)(wa[h] & 0xffff)) + 0.125f * bf((uint16_t)(wb[h] & 0xffff));
    float hi = bf((uint16_t)(wa[h] >> 16)) + 0.125f * bf((uint16_t)(wb[h] >> 16));
    if (!positive((uint16_t)(wm[h] & 0xffff))) lo = 0.f;
    if (!positive((uint16_t)(wm[h] >> 16))) hi = 0.f;
    o[h] = (uint32_t)tobf(lo) | ((uint32_t)tobf(hi) << 16);
  }
  *reinterpret_cast<uint4*>(out + (size_t)vf * C + ch) = make_uint4(o[0], o[1], o[2], o[3]);
}

// ---- bias gradients: per-channel sums over the interior (fixed order) -----
constexpr int kBiasBlocks = 64;

__global__ void chansum_partial_kernel(const uint16_t* __restrict__ t, int C, Vol g,
                                       double* partials) {
  // one block per (chunk of cells); each thread accumulates all C channels of its cells
  __shared__ double sh[kThreads];
  const int n = cells(g);
  for (int ch = 0; ch < C; ++ch) {
    double acc = 0.0;
    for (int c = blockIdx.x * kThreads + threadIdx.x; c < n; c += gridDim.x * kThreads)
      acc += bf(t[(size_t)halo_index(g, c, nullptr) * C + ch]);
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) partials[ch * gridDim.x + blockIdx.x] = sh[0];
    __syncthreads();
  }
}

__global__ void chansum_finish_kernel(const double* partials, int nb, int cout, float* out) {
  const int ch = threadIdx.x;
  if (ch >= cout) return;
  double t = 0.0;
  for (int b = 0; b < nb; ++b) t += partials[ch * nb + b];
  out[ch] = (float)t;
}

// ---- parameters --------------------------------------------------------------
// wf[t][co][ci] (padded cop x cip) and wb[t][ci][co] = W[26 - t][co][ci]
__global__ void prepare_weights_kernel(const float* __restrict__ w, int cin, int cout, int cip,
                                       int cop, uint16_t* __restrict__ wf, uint16_t* __restrict__ wb) {
  const int id = blockIdx.x * kThreads + threadIdx.x;
  if (id >= 27 * cop * cip) return;
  const int ci = id % cip, co = (id / cip) % cop, t = id / (cip * cop);
  const float v = (ci < cin && co < cout) ? w[((size_t)t * cout + co) * cin + ci] : 0.f;
  const uint16_t h = tobf(v);
  wf[id] = h;
  if (wb) wb[((size_t)(26 - t) * cip + ci) * cop + co] = h;
}

__global__ void prepare_bias_kernel(const float* __restrict__ b, int cout, int cop, float* bp) {
  const int i = threadIdx.x;
  if (i < cop) bp[i] = i < cout ? b[i] : 0.f;
}

// grad[t][co][ci] = padded[t][co][ci] for the true shape
__global__ void extract_wgrad_kernel(const float* __restrict__ padded, int cin, int cout, int cip,
                                     int cop, float* __restrict__ grad) {
  const int id = blockIdx.x * kThreads + threadIdx.x;
  if (id >= 27 * cout * cin) return;
  const int ci = id % cin, co = (id / cin) % cout, t = id / (cin * cout);
  grad[id] = padded[((size_t)t * cop + co) * cip + ci];
}

// Adam (Kingma and Ba 2015, Algorithm 1) with bias corrections bc1 = 1 - b1^t,
// bc2 = 1 - b2^t
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                            float bc1, float bc2) {
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

}  // namespace

struct tpfa_unet {
  int device;
  int train;
  Vol g[3];  // levels 0, 1, 2
  uint16_t* wf[kLayers];
  uint16_t* wb[kLayers];
  float* bias[kLayers];
  // forward activations
  uint16_t *in16, *e0, *s0, *d0, *o16;  // level 0
  uint16_t *p0, *e1, *s1, *d1;          // level 1
  uint16_t *p1, *e2, *d2;               // level 2
  // backward
  uint16_t *g16, *dd0, *ds0, *de0;      // level 0
  uint16_t *dd1, *ds1, *dp0, *de1;      // level 1
  uint16_t *dd2, *de2, *dp1;            // level 2
  float* wpad;     // padded weight gradient [27][16][16]
  float* ws;       // weight-gradient workspace
  size_t ws_bytes;
  float* rms;
  double* partials;
  bool have_params, have_forward;
};

namespace {

void unet_free(tpfa_unet* u) {
  cudaSetDevice(u->device);
  uint16_t** bufs[] = {&u->in16, &u->e0, &u->s0, &u->d0, &u->o16, &u->p0, &u->e1, &u->s1,
                       &u->d1,   &u->p1, &u->e2, &u->d2, &u->g16, &u->dd0, &u->ds0, &u->de0,
                       &u->dd1,  &u->ds1, &u->dp0, &u->de1, &u->dd2, &u->de2, &u->dp1};
  for (auto b : bufs) cudaFree(*b);
  for (int i = 0; i < kLayers; ++i) {
    cudaFree(u->wf[i]);
    cudaFree(u->wb[i]);
    cudaFree(u->bias[i]);
  }
  cudaFree(u->wpad);
  cudaFree(u->ws);
  cudaFree(u->rms);
  cudaFree(u->partials);
  delete u;
}

bool alloc_zero(void** p, size_t bytes) {
  if (cudaMalloc(p, bytes) != cudaSuccess) return false;
  return cudaMemset(*p, 0, bytes) == cudaSuccess;
}

bool vol_buf(uint16_t** p, const Vol& g, int C) {
  return alloc_zero((void**)p, (size_t)g.vp * C * sizeof(uint16_t));
}

#define CKE(x)                                  \
  do {                                          \
    if ((x) != cudaSuccess) return TPFA_ECUDA;  \
  } while (0)

int conv(tpfa_unet* u, const Vol* gv, int layer, const uint16_t* x, const uint16_t* mask,
         uint16_t* y, int flags, bool backward, cudaStream_t s) {
  const LayerDef& d = kDefs[layer];
  const Vol& g = gv[d.level];
  cudaError_t e;
  if (!backward)
    e = tpfa::net::conv_fwd(x, u->wf[layer], u->bias[layer], mask, y, g, d.cip, d.cop, flags, s);
  else
    e = tpfa::net::conv_fwd(x, u->wb[layer], nullptr, mask, y, g, d.cop, d.cip, flags, s);
  return e == cudaSuccess ? TPFA_OK : TPFA_ECUDA;
}

int layer_grads(tpfa_unet* u, int layer, const uint16_t* x, const uint16_t* dpre, float* grad,
                cudaStream_t s) {
  const LayerDef& d = kDefs[layer];
  const Vol& g = u->g[d.level];
  const bool padded = d.cin != d.cip || d.cout != d.cop;
  float* dw = padded ? u->wpad : grad + kParams.w[layer];
  CKE(tpfa::net::conv_wgrad(x, dpre, dw, u->ws, g, d.cip, d.cop, 0, s));
  if (padded) {
    extract_wgrad_kernel<<<blocks_for(27LL * d.cout * d.cin), kThreads, 0, s>>>(
        u->wpad, d.cin, d.cout, d.cip, d.cop, grad + kParams.w[layer]);
    CKE(cudaGetLastError());
  }
  chansum_partial_kernel<<<kBiasBlocks, kThreads, 0, s>>>(dpre, d.cop, g, u->partials);
  CKE(cudaGetLastError());
  chansum_finish_kernel<<<1, 64, 0, s>>>(u->partials, kBiasBlocks, d.cout, grad + kParams.b[layer]);
  CKE(cudaGetLastError());
  return TPFA_OK;
}

int elem_launch_ok() { return cudaGetLastError() == cudaSuccess ? TPFA_OK : TPFA_ECUDA; }

// lnk = (float) ln K, the network's second input channel
__global__ void log_perm_kernel(const double* __restrict__ K, float* __restrict__ lnk, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    lnk[i] = (float)log(K[i]);
}

}  // namespace

extern "C" {

int64_t tpfa_unet_param_count(void) { return kParams.total; }

int tpfa_log_perm(const double* K, float* lnk, int64_t n, void* stream) {
  int dev = -1;
  if (n < 1 || cudaGetDevice(&dev) != cudaSuccess) return n < 1 ? TPFA_EINVAL : TPFA_ECUDA;
  if (!tpfa::dev_ok(K, (size_t)n * 8, 8, dev) || !tpfa::dev_ok(lnk, (size_t)n * 4, 4, dev))
    return TPFA_EINVAL;
  const int64_t nb = (n + kThreads - 1) / kThreads;
  log_perm_kernel<<<(unsigned)(nb < 4096 ? nb : 4096), kThreads, 0, (cudaStream_t)stream>>>(K, lnk, n);
  return elem_launch_ok();
}

int tpfa_unet_create(int nx, int ny, int nz, int ns, int train, tpfa_unet** out) {
  if (out == nullptr) return TPFA_EINVAL;
  *out = nullptr;
  if (nx < 4 || ny < 4 || nz < 4 || nx % 4 || ny % 4 || nz % 4 || ns < 1) return TPFA_EINVAL;
  if (!tpfa::net::vol_ok(nx, ny, nz, ns) || (long long)nx * ny * nz * ns > (1LL << 30))
    return TPFA_EINVAL;
  tpfa_unet* u = new (std::nothrow) tpfa_unet;
  if (u == nullptr) return TPFA_ENOMEM;
  std::memset(u, 0, sizeof(*u));
  if (cudaGetDevice(&u->device) != cudaSuccess) {
    delete u;
    return TPFA_ECUDA;
  }
  u->train = train ? 1 : 0;
  u->g[0] = make_vol(nx, ny, nz, ns);
  u->g[1] = make_vol(nx / 2, ny / 2, nz / 2, ns);
  u->g[2] = make_vol(nx / 4, ny / 4, nz / 4, ns);
  bool ok = true;
  for (int i = 0; i < kLayers && ok; ++i) {
    const size_t nw = 27ULL * kDefs[i].cip * kDefs[i].cop * 2;
    ok = alloc_zero((void**)&u->wf[i], nw) && alloc_zero((void**)&u->bias[i], kDefs[i].cop * 4);
    if (ok && train && i > 0) ok = alloc_zero((void**)&u->wb[i], nw);
  }
  const Vol &g0 = u->g[0], &g1 = u->g[1], &g2 = u->g[2];
  ok = ok && vol_buf(&u->in16, g0, 16) && vol_buf(&u->e0, g0, 16) && vol_buf(&u->s0, g0, 16) &&
       vol_buf(&u->d0, g0, 16) && vol_buf(&u->o16, g0, 16) && vol_buf(&u->p0, g1, 16) &&
       vol_buf(&u->e1, g1, 32) && vol_buf(&u->s1, g1, 32) && vol_buf(&u->d1, g1, 16) &&
       vol_buf(&u->p1, g2, 32) && vol_buf(&u->e2, g2, 64) && vol_buf(&u->d2, g2, 32);
  if (ok && train) {
    ok = vol_buf(&u->g16, g0, 16) && vol_buf(&u->dd0, g0, 16) && vol_buf(&u->ds0, g0, 16) &&
         vol_buf(&u->de0, g0, 16) && vol_buf(&u->dd1, g1, 16) && vol_buf(&u->ds1, g1, 32) &&
         vol_buf(&u->dp0, g1, 16) && vol_buf(&u->de1, g1, 32) && vol_buf(&u->dd2, g2, 32) &&
         vol_buf(&u->de2, g2, 64) && vol_buf(&u->dp1, g2, 32) &&
         alloc_zero((void**)&u->wpad, 27 * 16 * 16 * 4);
    size_t wsb = 0;
    for (int i = 0; i < kLayers; ++i) {
      const size_t b = tpfa::net::conv_wgrad_ws_bytes(u->g[kDefs[i].level], kDefs[i].cip, kDefs[i].cop);
      if (b > wsb) wsb = b;
    }
    u->ws_bytes = wsb;
    ok = ok && alloc_zero((void**)&u->ws, wsb);
  }
  const size_t np = (size_t)ns * kRmsBlocks > 64 * kBiasBlocks ? (size_t)ns * kRmsBlocks
                                                                  : 64 * kBiasBlocks;
  ok = ok && alloc_zero((void**)&u->rms, (size_t)ns * 4) && alloc_zero((void**)&u->partials, np * 8);
  if (!ok) {
    cudaGetLastError();
    unet_free(u);
    return TPFA_ENOMEM;
  }
  *out = u;
  return TPFA_OK;
}

int tpfa_unet_shape(const tpfa_unet* u, int* dims4) {
  if (u == nullptr || dims4 == nullptr) return TPFA_EINVAL;
  dims4[0] = u->g[0].nx;
  dims4[1] = u->g[0].ny;
  dims4[2] = u->g[0].nz;
  dims4[3] = u->g[0].ns;
  return TPFA_OK;
}

int tpfa_unet_destroy(tpfa_unet* u) {
  if (u == nullptr) return TPFA_EINVAL;
  unet_free(u);
  return TPFA_OK;
}

int tpfa_unet_set_params(tpfa_unet* u, const float* params, void* stream) {
  if (u == nullptr) return TPFA_EINVAL;
  if (cudaSetDevice(u->device) != cudaSuccess) return TPFA_ECUDA;
  if (!tpfa::dev_ok(params, (size_t)kParams.total * 4, 4, u->device)) return TPFA_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  for (int i = 0; i < kLayers; ++i) {
    const LayerDef& d = kDefs[i];
    prepare_weights_kernel<<<blocks_for(27LL * d.cip * d.cop), kThreads, 0, s>>>(
        params + kParams.w[i], d.cin, d.cout, d.cip, d.cop, u->wf[i], u->wb[i]);
    prepare_bias_kernel<<<1, 64, 0, s>>>(params + kParams.b[i], d.cout, d.cop, u->bias[i]);
  }
  if (elem_launch_ok()) return TPFA_ECUDA;
  u->have_params = true;
  return TPFA_OK;
}

int tpfa_unet_forward_samples(tpfa_unet* u, int ns, const float* r, const float* lnk, float* z,
                              void* stream) {
  if (u == nullptr || !u->have_params || ns < 1 || ns > u->g[0].ns) return TPFA_EINVAL;
  if (cudaSetDevice(u->device) != cudaSuccess) return TPFA_ECUDA;
  // the first ns samples: a prefix of every volume (samples are whole haloed blocks)
  Vol gv[3];
  for (int l = 0; l < 3; ++l) gv[l] = make_vol(u->g[l].nx, u->g[l].ny, u->g[l].nz, ns);
  const Vol &g0 = gv[0], &g1 = gv[1], &g2 = gv[2];
  const int n0 = cells(g0);
  if (!tpfa::dev_ok(r, (size_t)n0 * 4, 4, u->device) || !tpfa::dev_ok(lnk, (size_t)n0 * 4, 4, u->device) ||
      !tpfa::dev_ok(z, (size_t)n0 * 4, 4, u->device))
    return TPFA_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int per = g0.nx * g0.ny * g0.nz;
  const int nrb = rms_blocks(per);
  sumsq_partial_kernel<<<dim3(nrb, g0.ns), kThreads, 0, s>>>(r, per, u->partials);
  rms_finish_kernel<<<g0.ns, kThreads, 0, s>>>(u->partials, nrb, per, u->rms);
  prep_input_kernel<<<blocks_for(n0), kThreads, 0, s>>>(r, lnk, u->rms, u->in16, g0);
  if (elem_launch_ok()) return TPFA_ECUDA;
  using tpfa::net::kConvRelu;
  int rc;
  u->have_forward = false;
  if ((rc = conv(u, gv, 0, u->in16, nullptr, u->e0, kConvRelu, false, s))) return rc;
  pool_kernel<<<blocks_for((long long)cells(g1) * 2), kThreads, 0, s>>>(u->e0, u->p0, 16, g0, g1);
  if ((rc = elem_launch_ok())) return rc;
  if ((rc = conv(u, gv, 1, u->p0, nullptr, u->e1, kConvRelu, false, s))) return rc;
  pool_kernel<<<blocks_for((long long)cells(g2) * 4), kThreads, 0, s>>>(u->e1, u->p1, 32, g1, g2);
  if ((rc = elem_launch_ok())) return rc;
  if ((rc = conv(u, gv, 2, u->p1, nullptr, u->e2, kConvRelu, false, s))) return rc;
  if ((rc = conv(u, gv, 3, u->e2, nullptr, u->d2, kConvRelu, false, s))) return rc;
  upadd_kernel<<<blocks_for((long long)cells(g1) * 4), kThreads, 0, s>>>(u->d2, u->e1, u->s1, 32, g1, g2);
  if ((rc = elem_launch_ok())) return rc;
  if ((rc = conv(u, gv, 4, u->s1, nullptr, u->d1, kConvRelu, false, s))) return rc;
  upadd_kernel<<<blocks_for((long long)n0 * 2), kThreads, 0, s>>>(u->d1, u->e0, u->s0, 16, g0, g1);
  if ((rc = elem_launch_ok())) return rc;
  if ((rc = conv(u, gv, 5, u->s0, nullptr, u->d0, kConvRelu, false, s))) return rc;
  if ((rc = conv(u, gv, 6, u->d0, nullptr, u->o16, 0, false, s))) return rc;
  out_extract_kernel<<<blocks_for(n0), kThreads, 0, s>>>(u->o16, u->rms, z, g0);
  if ((rc = elem_launch_ok())) return rc;
  // the backward pass needs the activations of every sample
  u->have_forward = ns == u->g[0].ns;
  return TPFA_OK;
}

int tpfa_unet_forward(tpfa_unet* u, const float* r, const float* lnk, float* z, void* stream) {
  if (u == nullptr) return TPFA_EINVAL;
  return tpfa_unet_forward_samples(u, u->g[0].ns, r, lnk, z, stream);
}

int tpfa_unet_backward(tpfa_unet* u, const float* gz, float* grad, void* stream) {
  if (u == nullptr || !u->train || !u->have_forward) return TPFA_EINVAL;
  if (cudaSetDevice(u->device) != cudaSuccess) return TPFA_ECUDA;
  const Vol &g0 = u->g[0], &g1 = u->g[1], &g2 = u->g[2];
  const int n0 = cells(g0);
  if (!tpfa::dev_ok(gz, (size_t)n0 * 4, 4, u->device) ||
      !tpfa::dev_ok(grad, (size_t)kParams.total * 4, 4, u->device))
    return TPFA_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  using tpfa::net::kConvMask;
  int rc;
  grad_in_kernel<<<blocks_for(n0), kThreads, 0, s>>>(gz, u->rms, u->g16, g0);
  if ((rc = elem_launch_ok())) return rc;
  // layer 6: z = conv(d0)
  if ((rc = layer_grads(u, 6, u->d0, u->g16, grad, s))) return rc;
  if ((rc = conv(u, u->g, 6, u->g16, u->d0, u->dd0, kConvMask, true, s))) return rc;
  // layer 5: d0 = relu(conv(s0))
  if ((rc = layer_grads(u, 5, u->s0, u->dd0, grad, s))) return rc;
  if ((rc = conv(u, u->g, 5, u->dd0, nullptr, u->ds0, 0, true, s))) return rc;
  // s0 = up(d1) + e0
  upadj_mask_kernel<<<blocks_for((long long)cells(g1) * 2), kThreads, 0, s>>>(u->ds0, u->d1, u->dd1, 16, g0, g1);
  if ((rc = elem_launch_ok())) return rc;
  // layer 4: d1 = relu(conv(s1))
  if ((rc = layer_grads(u, 4, u->s1, u->dd1, grad, s))) return rc;
  if ((rc = conv(u, u->g, 4, u->dd1, nullptr, u->ds1, 0, true, s))) return rc;
  // s1 = up(d2) + e1
  upadj_mask_kernel<<<blocks_for((long long)cells(g2) * 4), kThreads, 0, s>>>(u->ds1, u->d2, u->dd2, 32, g1, g2);
  if ((rc = elem_launch_ok())) return rc;
  // layer 3: d2 = relu(conv(e2))
  if ((rc = layer_grads(u, 3, u->e2, u->dd2, grad, s))) return rc;
  if ((rc = conv(u, u->g, 3, u->dd2, u->e2, u->de2, kConvMask, true, s))) return rc;
  // layer 2: e2 = relu(conv(p1))
  if ((rc = layer_grads(u, 2, u->p1, u->de2, grad, s))) return rc;
  if ((rc = conv(u, u->g, 2, u->de2, nullptr, u->dp1, 0, true, s))) return rc;
  // e1 feeds s1 (skip) and p1 = pool(e1)
  pooladj_add_mask_kernel<<<blocks_for((long long)cells(g1) * 4), kThreads, 0, s>>>(
      u->ds1, u->dp1, u->e1, u->de1, 32, g1, g2);
  if ((rc = elem_launch_ok())) return rc;
  // layer 1: e1 = relu(conv(p0))
  if ((rc = layer_grads(u, 1, u->p0, u->de1, grad, s))) return rc;
  if ((rc = conv(u, u->g, 1, u->de1, nullptr, u->dp0, 0, true, s))) return rc;
  // e0 feeds s0 (skip) and p0 = pool(e0)
  pooladj_add_mask_kernel<<<blocks_for((long long)n0 * 2), kThreads, 0, s>>>(
      u->ds0, u->dp0, u->e0, u->de0, 16, g0, g1);
  if ((rc = elem_launch_ok())) return rc;
  // layer 0: e0 = relu(conv(in))
  if ((rc = layer_grads(u, 0, u->in16, u->de0, grad, s))) return rc;
  return TPFA_OK;
}

int tpfa_adam_step(float* params, const float* grad, float* m, float* v, int64_t n, int t,
                   double lr, double b1, double b2, double eps, void* stream) {
  if (n < 1 || t < 1 || !(lr > 0) || !(b1 >= 0 && b1 < 1) || !(b2 >= 0 && b2 < 1) || !(eps >= 0))
    return TPFA_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return TPFA_ECUDA;
  const size_t bytes = (size_t)n * 4;
  if (!tpfa::dev_ok(params, bytes, 4, dev) || !tpfa::dev_ok(grad, bytes, 4, dev) ||
      !tpfa::dev_ok(m, bytes, 4, dev) || !tpfa::dev_ok(v, bytes, 4, dev))
    return TPFA_EINVAL;
  const double bc1 = 1.0 - pow(b1, t), bc2 = 1.0 - pow(b2, t);
  adam_kernel<<<blocks_for(n), kThreads, 0, (cudaStream_t)stream>>>(
      params, grad, m, v, n, (float)lr, (float)b1, (float)b2, (float)eps, (float)bc1, (float)bc2);
  return elem_launch_ok();
}

}  // extern "C"
