// Batched flexible CG (fcg_solve_batch): the learned-preconditioned,
// mixed-precision, batched form of the solve.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "batch_internal.cuh"
#include "fcg_common.cuh"

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
  int id;            // index in the batch's full chunk list (its partial-sum slot)
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
  block_sum_m<1>(d, part, ch.id);
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
                             int vec4, double* part, int skip_net) {
  constexpr int K = 2 + 2 * M;
  const BChunk ch = chunks[blockIdx.x];
  const int f = flags[ch.inst];
  if (skip_net && (f & kNet)) return;  // the fused operator took this instance's dots
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
  block_sum_m<K>(d, part, ch.id);
}

// c and the beta_j of every active instance (beta_j = 0 beyond its own
// retained directions)
__global__ void bfinish_dots_kernel(const int* __restrict__ cfirst, const int* __restrict__ ccount,
                                    const int* __restrict__ flags, const double* __restrict__ part,
                                    int M, const double* __restrict__ uau, BScal* sc, int head,
                                    int m, const double* __restrict__ fdots) {
  const int i = blockIdx.x;
  const int f = flags[i];
  if (!(f & kAct)) return;
  __shared__ double tot[2 + 2 * kMaxDirs];
  const int K = 2 + 2 * M;
  if (fdots != nullptr && (f & kNet)) {
    // from the fused operator: u'q, then u'r, q'w, w'q_j, u'q_j
    if (threadIdx.x < K)
      tot[threadIdx.x] = fdots[(size_t)i * tpfa::kApplyDotsStride + 1 + threadIdx.x];
    __syncthreads();
  } else {
    chunk_totals(part, cfirst[i], ccount[i], K, tot);
  }
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
  block_sum_m<1>(pr, part, ch.id);
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
  block_sum_m<1>(rr, part, ch.id);
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
                  const Dirs& qd, int vec4, double* part, int skip_net) {
  switch (M) {
#define X(MM)                                                                                  \
  case MM:                                                                                     \
    bdots_kernel<MM><<<nchunks, kT, 0, s>>>(ch, flags, r, dinv, u, au, qd, vec4, part, skip_net); \
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
  std::vector<int> members;
  std::vector<int> active;  // indices into members of the samples the network runs on
  int64_t* soff = nullptr;  // dev: cell offset of each active member in the concatenated arrays
  int64_t* coff = nullptr;  // dev: offset of each active member's sample in lnk_all
  float* rl[kMaxLevels + 1] = {};  // rl[levels]: restricted residuals (level 0: gathered copy)
  float* ul[kMaxLevels + 1] = {};  // ul[levels]: network output (level 0: before the scatter)
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
  // TMA-staged operator (set up when every instance suits it): per-instance
  // tilings and tensor maps {coefficients, z, P slot 0 .. m-1}, block partials
  bool tma = false;
  CUtensorMap* amaps = nullptr;
  std::vector<tpfa::TmaInst> ainst_all;  // every instance (host)
  tpfa::TmaInst* ainst = nullptr;         // the instances of aset (device)
  int own0 = 0;                           // first own-cell map of an instance
  double* dots = nullptr;                 // fused operator: per-instance dot products
  int nainst = 0;
  int64_t ablocks = 0;
  double* apart = nullptr;
  // The per-iteration passes launch only over the instances that were
  // iterating at the host's last look (aset): their chunks and operator
  // blocks.  An instance that stops on the device in between keeps its
  // blocks until the next look; they return at once.
  std::vector<int> aset;
  std::vector<BChunk> achunks;
  BChunk* achunks_dev = nullptr;
  unsigned nach = 0;

  bool alloc() {
    const size_t v = (size_t)stride * 4;
    const size_t nc = chunks.size();
    bool ok = cudaMalloc(&chunks_dev, sizeof(BChunk) * nc) == cudaSuccess &&
              cudaMalloc(&achunks_dev, sizeof(BChunk) * nc) == cudaSuccess &&
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
    cudaFree(achunks_dev);
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
    cudaFree(amaps);
    cudaFree(ainst);
    cudaFree(apart);
    cudaFree(dots);
    if (fork) cudaEventDestroy(fork);
  }
  unsigned nchunks() const { return (unsigned)chunks.size(); }
};

// The batch's operator through the TMA-staged kernel when every instance
// suits the copy engine (nx % 4 == 0, cell offsets on 16-byte boundaries) and
// the cp.async sweep is not requested; the instances keep the z-runs of the
// batch's CG sweep, so an instance's tiling does not depend on the batch it
// is in once its run length is given.  Otherwise w.tma stays false.
int setup_apply_tma(const tpfa_batch* batch, const float* coef, BWork& w) {
  using namespace tpfa;
  if (batch->sweep_sel == 1 || !w.vec4 || reinterpret_cast<uintptr_t>(coef) % 16 != 0)
    return TPFA_OK;
  for (const Grid& g : batch->g)
    if (!tma_apply_ok(g, false)) return TPFA_OK;
  // maps per instance: coefficients, z, P slots (with halo); r, M^-1, Q slots
  // (own cells, for the fused dot products)
  const int N = w.ninst, per = 4 + 2 * w.m;
  std::vector<const float*> own(2 + w.m);
  const std::vector<int> zr = batch_tma_zc_request(batch);
  std::vector<CUtensorMap> maps((size_t)per * N);
  std::vector<TmaInst> inst(N);
  std::vector<const float*> in(1 + w.m);
  int64_t blocks = 0;
  for (int i = 0; i < N; ++i) {
    const TmaPlan p = plan_tma(batch->g[i], 0, zr[i], batch->num_sms, false, false, true);
    const int64_t o = batch->off[i];
    in[0] = w.z + o;
    for (int k = 0; k < w.m; ++k) in[1 + k] = w.P + (size_t)k * w.stride + o;
    own[0] = w.r + o;
    own[1] = w.dinv + o;
    for (int k = 0; k < w.m; ++k) own[2 + k] = w.Q + (size_t)k * w.stride + o;
    if (!make_apply_maps(batch->g[i], p, reinterpret_cast<const float4*>(coef) + o, in.data(),
                         1 + w.m, &maps[(size_t)per * i]) ||
        !make_own_maps(batch->g[i], p, own.data(), 2 + w.m, &maps[(size_t)per * i + 2 + w.m]))
      return TPFA_ECUDA;
    TmaInst& I = inst[i];
    I.g = batch->g[i];
    I.zc = p.zc;
    I.nbx = (int)p.nbx;
    I.nby = (int)p.nby;
    I.id = i;
    I.off = o;
    I.bstart = blocks;
    I.nblocks = p.nblocks;
    blocks += p.nblocks;
  }
  if (blocks > 0x7fffffff) return TPFA_OK;
  if (cudaMalloc(&w.amaps, sizeof(CUtensorMap) * maps.size()) != cudaSuccess ||
      cudaMalloc(&w.ainst, sizeof(TmaInst) * N) != cudaSuccess ||
      cudaMalloc(&w.apart, sizeof(double) * blocks * (3 + 2 * kApplyMaxDirs)) != cudaSuccess ||
      cudaMalloc(&w.dots, sizeof(double) * kApplyDotsStride * N) != cudaSuccess) {
    cudaGetLastError();
    return TPFA_ENOMEM;
  }
  for (int i = 0; i < N; ++i) inst[i].maps = w.amaps + (size_t)per * i;
  if (cudaMemcpyAsync(w.amaps, maps.data(), sizeof(CUtensorMap) * maps.size(),
                      cudaMemcpyHostToDevice, w.s) != cudaSuccess ||
      cudaMemcpyAsync(w.ainst, inst.data(), sizeof(TmaInst) * N, cudaMemcpyHostToDevice, w.s) !=
          cudaSuccess ||
      cudaStreamSynchronize(w.s) != cudaSuccess)
    return TPFA_ECUDA;
  w.ainst_all = inst;
  w.nainst = N;
  w.own0 = 2 + w.m;
  w.tma = true;
  w.ablocks = blocks;
  return TPFA_OK;
}

// The launch lists of the per-iteration passes for the instances whose host
// flags (w.hflags) hold kAct: their chunks, and their operator blocks
// numbered consecutively.  The copies are ordered on the stream before the
// passes that read the lists.
int compact_active(BWork& w) {
  using namespace tpfa;
  std::vector<int> act;
  for (int i = 0; i < w.ninst; ++i)
    if (w.hflags[i] & kAct) act.push_back(i);
  if (act == w.aset && w.nach > 0) return TPFA_OK;
  w.aset = act;
  w.achunks.clear();
  for (int i : act)
    for (int c = w.cfirst[i]; c < w.cfirst[i] + w.ccount[i]; ++c) w.achunks.push_back(w.chunks[c]);
  w.nach = (unsigned)w.achunks.size();
  if (w.nach > 0 && cudaMemcpyAsync(w.achunks_dev, w.achunks.data(), sizeof(BChunk) * w.nach,
                                    cudaMemcpyHostToDevice, w.s) != cudaSuccess)
    return TPFA_ECUDA;
  if (w.tma) {
    std::vector<TmaInst> t;
    int64_t b = 0;
    for (int i : act) {
      TmaInst I = w.ainst_all[i];
      I.bstart = b;
      b += I.nblocks;
      t.push_back(I);
    }
    w.nainst = (int)t.size();
    w.ablocks = b;
    if (!t.empty() && cudaMemcpyAsync(w.ainst, t.data(), sizeof(TmaInst) * t.size(),
                                      cudaMemcpyHostToDevice, w.s) != cudaSuccess)
      return TPFA_ECUDA;
  }
  return TPFA_OK;
}

// Operator q = A (input) of the instances with (flags & need) == need, p'q per
// instance into pap; input `which`: 0 = z, 1 + k = P slot k.
bool batch_apply(const tpfa_batch* batch, BWork& w, const float4* cf4, int which, float* out,
                 double* pap, int need) {
  using namespace tpfa;
  if (w.tma) {
    if (w.nainst == 0) return true;  // nothing iterates
    return launch_apply_tma_batch(w.ainst, w.nainst, w.ablocks, which, out, pap, w.flags, need,
                                  w.apart, batch->counters, w.s) == cudaSuccess;
  }
  const float* in = which == 0 ? w.z : w.P + (size_t)(which - 1) * w.stride;
  return launch_apply_batch(batch->inst_dev, w.ninst, batch->sweep_blocks, cf4, in, out, pap,
                            w.flags, need, batch->partials, batch->counters, w.s) == cudaSuccess;
}

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
    const int L = N.levels;
    launch_restrict_levels(L, w.nb, w.s, w.r, N.rl[L], N.dims[0], N.dims[1], N.dims[2], ns, N.soff,
                           N.pdims[0], N.pdims[1], N.pdims[2]);
    rc = tpfa_unet_forward_samples(N.net, ns, N.rl[L], N.lnkc, N.ul[L], w.s);
    if (rc) return rc;
    launch_prolong_levels(L, w.nb, w.s, N.ul[L], w.z, N.dims[0], N.dims[1], N.dims[2], ns, N.soff,
                          N.pdims[0], N.pdims[1], N.pdims[2], w.vec4 != 0);
    w.launches += 17;
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
        ch.id = (int)w.chunks.size();
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
    if (ok) {
      rc = setup_apply_tma(batch, coef, w);
      if (rc) return rc;
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
      {
        const int L = B.levels;
        const size_t bytes = (size_t)B.ncoarse * ns * 4;
        ok = ok && cudaMalloc(&B.rl[L], bytes) == cudaSuccess &&
             cudaMalloc(&B.ul[L], bytes) == cudaSuccess &&
             cudaMemsetAsync(B.rl[L], 0, bytes, s) == cudaSuccess;
      }
      ok = ok && cudaMalloc(&B.lnkc, (size_t)B.ncoarse * ns * 4) == cudaSuccess &&
           cudaMalloc(&B.lnk_all, (size_t)B.ncoarse * ns * 4) == cudaSuccess &&
           cudaMemsetAsync(B.lnk_all, 0, (size_t)B.ncoarse * ns * 4, s) == cudaSuccess &&
           cudaMalloc(&B.coff, sizeof(int64_t) * ns) == cudaSuccess;
      if (!ok) break;
      // ln K on the network's grid (mean over each 2^levels block), member
      // after member
      if (B.levels == 0)
        gather_kernel<<<w.nb, kT, 0, s>>>(lnk, B.soff, B.lnk_all, nf, ns, 0);
      else
        launch_restrict_levels(B.levels, w.nb, s, lnk, B.lnk_all, B.dims[0], B.dims[1], B.dims[2],
                               ns, B.soff, B.pdims[0], B.pdims[1], B.pdims[2]);
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
      rc = compact_active(w);
      if (rc) break;
      bool first = true;
      while (running && rc == TPFA_OK) {
        bool any_blend = false, any_plain = false;  // instances with / without the network
        for (int i = 0; i < N; ++i) {
          any_blend = any_blend || blend[i];
          any_plain = any_plain || ((w.hflags[i] & kAct) && !blend[i]);
        }
        Dirs qd, pd;
        int qmap[kMaxDirs];
        for (int j = 0; j < gstored; ++j) {
          const size_t slot = (size_t)((head - 1 - j + w.m) % w.m);
          qd.v[j] = w.Q + slot * w.stride;
          pd.v[j] = w.P + slot * w.stride;
          qmap[j] = (int)slot;
        }
        // the TMA-staged operator A u also forms the dot products of the blend
        // instances (A u itself is not stored; r, M^-1 and the q_j come in
        // through its producer); the dots pass then covers the others only
        const bool fused = any_blend && w.tma && gstored <= kApplyMaxDirs;
        if (any_blend) {
          rc = batch_network_term(bn, w);
          if (rc) break;
          const bool ok =
              fused ? launch_apply_dots_tma_batch(w.ainst, w.nainst, w.ablocks, 0, w.flags,
                                                  kAct | kNet, w.own0, qmap, gstored, w.uau,
                                                  w.dots, w.apart, batch->counters,
                                                  s) == cudaSuccess
                    : batch_apply(batch, w, cf4, 0, w.au, w.uau, kAct | kNet);
          if (!ok) {
            rc = TPFA_ECUDA;
            break;
          }
          ++w.launches;
        }
        float* p = w.P + (size_t)head * w.stride;
        float* q = w.Q + (size_t)head * w.stride;
        if (!fused || any_plain) {
          launch_bdots(gstored, w.nach, s, w.achunks_dev, w.flags, w.r, w.dinv, w.z, w.au, qd,
                       w.vec4, w.part, fused ? 1 : 0);
          ++w.launches;
        }
        bfinish_dots_kernel<<<N, kT, 0, s>>>(w.cfirst_dev, w.ccount_dev, w.flags, w.part, gstored,
                                             w.uau, w.sc, head, w.m, fused ? w.dots : nullptr);
        launch_bdir(gstored, w.nach, s, w.achunks_dev, w.flags, w.sc, w.r, w.dinv, w.z, pd, p,
                    w.vec4, w.part);
        if (!batch_apply(batch, w, cf4, 1 + head, q, w.pq, kAct)) {
          rc = TPFA_ECUDA;
          break;
        }
        bfinish_alpha_kernel<<<N, kT, 0, s>>>(w.cfirst_dev, w.ccount_dev, w.flags, w.part, w.pq,
                                              w.sc, head, w.m);
        bupdate_kernel<<<w.nach, kT, 0, s>>>(w.achunks_dev, w.flags, w.sc, w.e, w.r, p, q,
                                             w.vec4, w.part);
        bfinish_rr_kernel<<<N, kT, 0, s>>>(w.cfirst_dev, w.ccount_dev, w.flags, w.part, w.sc,
                                           w.hist, pending);
        w.launches += 6;
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
        // the networks run on the members that still iterate with them, the
        // passes on the instances that still iterate
        rc = update_active(bn, blend, batch->off, w);
        if (rc) break;
        rc = compact_active(w);
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
