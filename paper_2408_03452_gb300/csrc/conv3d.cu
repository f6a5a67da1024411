// 3x3x3 convolutions of BF16 channels-last volumes on the tcgen05 tensor
// cores (implicit GEMM, FP32 accumulation in tensor memory).
//
// Forward (and input gradient).  An output tile is 128 consecutive voxel
// indices of the haloed layout (halo voxels inside the range are computed
// and discarded).  For one z-offset dz the three rows dy = -1, 0, 1 of 130
// voxels (the tile plus one voxel either side) are copied to shared memory
// as "row groups" in the K-major core-matrix layout [CIN/8][130][8 channels],
// i.e. 16 bytes per voxel and channel block.  With M-direction stride 128
// bytes per 8 voxels, tap (dy, dx) of the GEMM operand A[m][ci] =
// x[s0 + m + off][ci] is the row group of dy started dx voxels later -- a
// descriptor offset of 16 dx bytes, no data movement.  Each (dz, dy, dx, 16
// channel) step is one tcgen05.mma with M = 128, N = COUT, K = 16 against
// the weights of that tap, which sit in shared memory for the whole
// persistent CTA.  The dz row-group triples are double-buffered: the copy
// of the next one runs while the tensor core works on the current one.
// Epilogue: bias, ReLU or a ReLU-derivative mask, BF16 rounding, halo skip.
// The input gradient of a convolution is the same operation with the taps
// flipped and the weight matrices transposed.
//
// Weight gradient.  dw[t][co][ci] = sum_v dy[v][co] x[v + off_t][ci] is a
// GEMM with rows (t, ci) -- 128/CIN taps per 128-row tile -- columns co and
// the voxels as the reduction.  Chunks of 64 voxels of x (shifted per tap)
// and of dy are transposed 8x8 at a time with movmatrix into K-major tiles;
// CTAs split the voxel range, write FP32 partial tiles, and a second kernel
// adds the partials in a fixed order.
#include <cuda_bf16.h>

#include "net_internal.cuh"
#include "tc_common.cuh"
#include "tpfa_internal.cuh"

namespace tpfa {
namespace net {

// Set (never cleared by a kernel) when a bounded tensor-core wait gave up.
__device__ int g_tc_timeout;

namespace {

constexpr uint32_t kWaitLimit = 1u << 22;  // mbarrier polls before giving up
constexpr int kRG = 130;                   // voxels per staged row group

__device__ __forceinline__ void cp16z(void* dst, const void* src, bool ok) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(tc::smem_addr(dst)),
               "l"(src), "r"(ok ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_commit_group() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait_groups() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ uint32_t movmatrix_trans(uint32_t a) {
  uint32_t d;
  asm volatile("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;" : "=r"(d) : "r"(a));
  return d;
}

__device__ __forceinline__ bool bf16_positive(uint32_t h) {
  return (h & 0x8000u) == 0 && (h & 0x7fffu) != 0;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&v);
}

// stages of the row-group ring: as deep as shared memory allows several CTAs
// per SM for the small layers; the 64-channel layers hold 110 KB of weights
template <int CIN, int COUT>
constexpr int fwd_stages() {
  return (CIN == 16) ? 4 : (CIN == 32 && COUT == 16) ? 3 : 2;
}

template <int CIN, int COUT>
struct FwdCfg {
  static constexpr int kS = fwd_stages<CIN, COUT>();
  static constexpr int kWTap = COUT * CIN * 2;  // bytes of one tap's weight matrix
  static constexpr int kWBytes = 27 * kWTap;
  static constexpr int kRGBytes = kRG * CIN * 2;
  static constexpr int kStage = 3 * kRGBytes;
  static constexpr int kSmem = kWBytes + kS * kStage;
  static constexpr uint32_t kCols = COUT < 32 ? 32 : COUT;
  static_assert(CIN % 16 == 0 && COUT % 16 == 0 && COUT <= 256, "shape");
  static_assert(kSmem <= 227 * 1024, "shared memory");
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(128)
conv_fwd_kernel(const uint16_t* __restrict__ x, const uint16_t* __restrict__ w,
                const float* __restrict__ bias, const uint16_t* __restrict__ mask,
                uint16_t* __restrict__ y, Vol g, int flags, int ntiles) {
  using Cfg = FwdCfg<CIN, COUT>;
  constexpr int kc = CIN / 8;
  constexpr int S = Cfg::kS;
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) uint64_t bars[S];
  __shared__ uint32_t tbase;
  unsigned char* sW = sm;
  unsigned char* sS = sm + Cfg::kWBytes;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  for (int i = tid; i < 27 * COUT * kc; i += 128) {
    const int c = i % kc, r = (i / kc) % COUT, t = i / (kc * COUT);
    const uint4 v = *reinterpret_cast<const uint4*>(w + ((size_t)t * COUT + r) * CIN + c * 8);
    *reinterpret_cast<uint4*>(sW + t * Cfg::kWTap + tc::kmajor_off(r, c * 8, CIN)) = v;
  }
  if (tid == 0)
    for (int b = 0; b < S; ++b) tc::mbar_init(&bars[b], 1);
  if (warp == 0) tc::tmem_alloc(&tbase, Cfg::kCols);
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t acc = tbase;

  const int my_tiles = (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const int njobs = 3 * my_tiles;  // job = (tile, dz)

  // copies of job j into buffer j % S; every call commits one group (empty
  // past the last job) so that wait_group counts stay uniform
  auto load_job = [&](int j) {
    if (j < njobs) {
      const int tile = blockIdx.x + (j / 3) * gridDim.x;
      const int dz = j % 3 - 1;
      const int base = g.g0 + tile * 128 + dz * g.pp - g.wp - 1;
      unsigned char* st = sS + (j % S) * Cfg::kStage;
      for (int i = tid; i < 3 * kRG * kc; i += 128) {
        const int c = i % kc, v = (i / kc) % kRG, gi = i / (kc * kRG);
        const int row = base + gi * g.wp + v;
        const bool ok = row >= 0 && row < g.vp;
        cp16z(st + gi * Cfg::kRGBytes + c * (kRG * 16) + v * 16,
              x + (size_t)(ok ? row : 0) * CIN + c * 8, ok);
      }
    }
    cp_commit_group();
  };

  bool abort = false;
  for (int j = 0; j < S - 1; ++j) load_job(j);
  for (int j = 0; j < njobs; ++j) {
    const int buf = j % S;
    cp_wait_groups<S - 2>();  // job j's group is complete
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      const int dzi = j % 3;
      const uint32_t st = tc::smem_addr(sS + buf * Cfg::kStage);
      const uint32_t wb = tc::smem_addr(sW);
      constexpr uint32_t idesc = tc::idesc_bf16_f32(128, COUT);
#pragma unroll 1
      for (int gi = 0; gi < 3; ++gi) {
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          const int t = dzi * 9 + gi * 3 + dx;
#pragma unroll
          for (int ks = 0; ks < CIN / 16; ++ks) {
            const uint64_t ad = tc::smem_desc(st + gi * Cfg::kRGBytes + dx * 16 + ks * 2 * kRG * 16,
                                              kRG * 16, 128);
            const uint64_t bd = tc::smem_desc(wb + t * Cfg::kWTap + ks * 256, 128, kc * 128);
            tc::mma_bf16(acc, ad, bd, idesc, (dzi | gi | dx | ks) != 0);
          }
        }
      }
      tc::mma_commit(&bars[buf]);
    }
    // job j+S-1 reuses the buffer of job j-1: wait for that job's MMAs
    bool ok = true;
    if (j >= 1 && j + S - 1 < njobs)
      ok = tc::mbar_wait(&bars[(j - 1) % S], ((j - 1) / S) & 1, kWaitLimit);
    if (__syncthreads_or(!ok)) {
      abort = true;
      break;
    }
    load_job(j + S - 1);
    if (j % 3 == 2) {
      const bool done = tc::mbar_wait(&bars[buf], (j / S) & 1, kWaitLimit);
      if (__syncthreads_or(!done)) {
        abort = true;
        break;
      }
      tc::fence_after();
      const int tile = blockIdx.x + (j / 3) * gridDim.x;
      const int idx = g.g0 + tile * 128 + warp * 32 + lane;
      const bool in = vol_interior(g, idx);
#pragma unroll
      for (int c0 = 0; c0 < COUT; c0 += 8) {
        float v[8];
        tc::tmem_ld8(acc + ((uint32_t)(warp * 32) << 16) + c0, v);
        if (in) {
          uint4 mk = make_uint4(0, 0, 0, 0);
          if (flags & kConvMask) mk = *reinterpret_cast<const uint4*>(mask + (size_t)idx * COUT + c0);
          const uint32_t mw[4] = {mk.x, mk.y, mk.z, mk.w};
          uint32_t o[4];
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            float a = v[2 * h], b = v[2 * h + 1];
            if (bias) {
              a += bias[c0 + 2 * h];
              b += bias[c0 + 2 * h + 1];
            }
            if (flags & kConvRelu) {
              a = fmaxf(a, 0.f);
              b = fmaxf(b, 0.f);
            }
            if (flags & kConvMask) {
              if (!bf16_positive(mw[h] & 0xffffu)) a = 0.f;
              if (!bf16_positive(mw[h] >> 16)) b = 0.f;
            }
            o[h] = pack_bf16(a, b);
          }
          *reinterpret_cast<uint4*>(y + (size_t)idx * COUT + c0) = make_uint4(o[0], o[1], o[2], o[3]);
        }
      }
      tc::fence_before();
    }
  }
  cp_wait_all();
  if (abort && tid == 0) atomicOr(&g_tc_timeout, 1);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(acc, Cfg::kCols);
}

// ---- z-marching forward kernel ---------------------------------------------
// A work unit is one 128-voxel segment of a padded plane (offset bi * 128)
// followed through zc consecutive interior planes of one sample.  Output k of
// the unit needs the row-group triples of planes k-1, k, k+1; triple j of the
// unit goes to ring slot j % ST and is loaded once, ST - 3 outputs ahead of its
// first use, instead of three times.  Two TMEM accumulators alternate between
// outputs so that the epilogue of output k-1 runs while the tensor core works
// on output k.
template <int CIN, int COUT>
constexpr int zm_stages() {
  return (CIN == 32 && COUT == 64) ? 4 : (CIN == 16) ? 7 : 5;
}

template <int CIN, int COUT>
struct ZmCfg {
  static constexpr int kST = zm_stages<CIN, COUT>();
  static constexpr int kWTap = COUT * CIN * 2;
  static constexpr int kWBytes = 27 * kWTap;
  static constexpr int kRGBytes = kRG * CIN * 2;
  static constexpr int kTriple = 3 * kRGBytes;
  static constexpr int kSmem = kWBytes + kST * kTriple;
  static constexpr uint32_t kCols = 2 * COUT < 32 ? 32 : 2 * COUT;  // two accumulators
  static_assert(kSmem <= 227 * 1024, "shared memory");
};

struct ZmGrid {
  int nb;   // 128-voxel segments per padded plane
  int zc;   // interior planes per unit
  int nzc;  // units per sample along z
  int units;
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(128)
conv_fwd_zm_kernel(const uint16_t* __restrict__ x, const uint16_t* __restrict__ w,
                   const float* __restrict__ bias, const uint16_t* __restrict__ mask,
                   uint16_t* __restrict__ y, Vol g, int flags, ZmGrid zg) {
  using Cfg = ZmCfg<CIN, COUT>;
  constexpr int ST = Cfg::kST;
  constexpr int kc = CIN / 8;
  constexpr int kChunks = 3 * kRG * kc;            // 16-byte copies per triple
  constexpr int kPer = (kChunks + 127) / 128;      // per thread
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t tbase;
  __shared__ float sbias[COUT];
  unsigned char* sW = sm;
  unsigned char* sR = sm + Cfg::kWBytes;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  for (int i = tid; i < 27 * COUT * kc; i += 128) {
    const int c = i % kc, r = (i / kc) % COUT, t = i / (kc * COUT);
    const uint4 v = *reinterpret_cast<const uint4*>(w + ((size_t)t * COUT + r) * CIN + c * 8);
    *reinterpret_cast<uint4*>(sW + t * Cfg::kWTap + tc::kmajor_off(r, c * 8, CIN)) = v;
  }
  if (tid < COUT) sbias[tid] = bias ? bias[tid] : 0.f;
  if (tid == 0) {
    tc::mbar_init(&bars[0], 1);
    tc::mbar_init(&bars[1], 1);
  }
  if (warp == 0) tc::tmem_alloc(&tbase, Cfg::kCols);
  // this thread's copies of a triple: row offset from the triple's first row,
  // and byte offset inside the ring slot
  int roff[kPer], coff[kPer];
  uint32_t soff[kPer];
#pragma unroll
  for (int m = 0; m < kPer; ++m) {
    const int i = tid + 128 * m;
    const int c = i % kc, v = (i / kc) % kRG, gi = i / (kc * kRG);
    roff[m] = gi * g.wp + v;
    coff[m] = c * 8;
    soff[m] = (uint32_t)(gi * Cfg::kRGBytes + c * (kRG * 16) + v * 16);
  }
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t acc0 = tbase;
  // descriptors of ring slot 0 (A) and of the weights (B); a byte offset d
  // inside shared memory adds d >> 4 to the start-address field
  const uint64_t adesc0 = tc::smem_desc(tc::smem_addr(sR), kRG * 16, 128);
  const uint64_t bdesc0 = tc::smem_desc(tc::smem_addr(sW), 128, kc * 128);

  bool abort = false;
  int o = 0;  // outputs issued by this CTA (accumulator and barrier phase)
  for (int u = blockIdx.x; u < zg.units && !abort; u += gridDim.x) {
    const int bi = u % zg.nb, cz = u / zg.nb;
    const int sidx = cz / zg.nzc;
    const int z0 = (cz % zg.nzc) * zg.zc;
    const int nout = min(zg.zc, g.nz - z0);
    const int kp0 = sidx * g.dp + 1 + z0;  // padded plane of output 0
    const int seg = bi * 128;              // offset of the segment in its plane
    const int ntrip = nout + 2;            // triples: planes kp0-1 .. kp0+nout
    // this thread's output voxel in the plane: interior in x and y (every
    // plane of a unit is interior in z)
    const int poff = seg + warp * 32 + lane;
    const int px = poff % g.wp, py = poff / g.wp;
    const bool in_xy = poff < g.pp && px >= 1 && px <= g.nx && py >= 1 && py <= g.ny;
    auto load_triple = [&](int j) {
      if (j < ntrip) {
        const int base = seg + (kp0 - 1 + j) * g.pp - g.wp - 1;
        unsigned char* st = sR + (j % ST) * Cfg::kTriple;
#pragma unroll
        for (int m = 0; m < kPer; ++m) {
          if (kChunks % 128 == 0 || tid + 128 * m < kChunks) {
            const int row = base + roff[m];
            const bool ok = row >= 0 && row < g.vp;
            cp16z(st + soff[m], x + (size_t)(ok ? row : 0) * CIN + coff[m], ok);
          }
        }
      }
      cp_commit_group();
    };
    for (int j = 0; j < ST; ++j) load_triple(j);

    auto epilogue = [&](int k, int ok_) {
      const size_t idx = (size_t)(kp0 + k) * g.pp + poff;
      const uint32_t acc = acc0 + (uint32_t)((ok_ & 1) * COUT);
      float va[COUT];
      tc::tmem_ld_cols<COUT>(acc + ((uint32_t)(warp * 32) << 16), va);
#pragma unroll
      for (int c0 = 0; c0 < COUT; c0 += 8) {
        const float* v = va + c0;
        if (in_xy) {
          uint4 mk = make_uint4(0, 0, 0, 0);
          if (flags & kConvMask) mk = *reinterpret_cast<const uint4*>(mask + idx * COUT + c0);
          const uint32_t mw[4] = {mk.x, mk.y, mk.z, mk.w};
          uint32_t ov[4];
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            float a = v[2 * h] + sbias[c0 + 2 * h], b = v[2 * h + 1] + sbias[c0 + 2 * h + 1];
            if (flags & kConvRelu) {
              a = fmaxf(a, 0.f);
              b = fmaxf(b, 0.f);
            }
            if (flags & kConvMask) {
              if (!bf16_positive(mw[h] & 0xffffu)) a = 0.f;
              if (!bf16_positive(mw[h] >> 16)) b = 0.f;
            }
            ov[h] = pack_bf16(a, b);
          }
          *reinterpret_cast<uint4*>(y + idx * COUT + c0) = make_uint4(ov[0], ov[1], ov[2], ov[3]);
        }
      }
    };

    for (int k = 0; k < nout; ++k, ++o) {
      cp_wait_groups<ST - 4>();  // triples k .. k+2 are complete
      tc::fence_proxy_async();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after();
        const uint32_t acc = acc0 + (uint32_t)((o & 1) * COUT);
        constexpr uint32_t idesc = tc::idesc_bf16_f32(128, COUT);
        uint64_t slot[3];
#pragma unroll
        for (int dz = 0; dz < 3; ++dz)
          slot[dz] = adesc0 + (uint64_t)(((k + dz) % ST) * (Cfg::kTriple >> 4));
#pragma unroll
        for (int dz = 0; dz < 3; ++dz)
#pragma unroll
          for (int gi = 0; gi < 3; ++gi)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx)
#pragma unroll
              for (int ks = 0; ks < CIN / 16; ++ks) {
                const int t = dz * 9 + gi * 3 + dx;
                const uint64_t ad =
                    slot[dz] + (uint64_t)((gi * Cfg::kRGBytes + dx * 16 + ks * 2 * kRG * 16) >> 4);
                const uint64_t bd = bdesc0 + (uint64_t)((t * Cfg::kWTap + ks * 256) >> 4);
                tc::mma_bf16(acc, ad, bd, idesc, (dz | gi | dx | ks) != 0);
              }
        tc::mma_commit(&bars[o & 1]);
      }
      if (k >= 1) {
        // output k-1 done: its triple k-1 is free and its accumulator is final
        const bool ok = tc::mbar_wait(&bars[(o - 1) & 1], ((o - 1) >> 1) & 1, kWaitLimit);
        if (__syncthreads_or(!ok)) {
          abort = true;
          break;
        }
        load_triple(k - 1 + ST);
        tc::fence_after();
        epilogue(k - 1, o - 1);
        tc::fence_before();
      } else {
        cp_commit_group();
      }
    }
    if (abort) break;
    // last output of the unit
    {
      const bool ok = tc::mbar_wait(&bars[(o - 1) & 1], ((o - 1) >> 1) & 1, kWaitLimit);
      if (__syncthreads_or(!ok)) {
        abort = true;
        break;
      }
      tc::fence_after();
      epilogue(nout - 1, o - 1);
      tc::fence_before();
    }
    cp_wait_all();
    __syncthreads();  // ring slots are rewritten by the next unit
  }
  cp_wait_all();
  if (abort && tid == 0) atomicOr(&g_tc_timeout, 1);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(acc0, Cfg::kCols);
}

// ---- z-marching forward kernel with the z-taps folded into N ---------------
// Same work units and row-group triples as the z-marching kernel, but the loop
// runs over input planes instead of output planes.  Triple j (planes
// kp0-2+j .. in the unit's numbering) feeds outputs j-2, j-1 and j through the
// taps dz = 2, 1, 0, and for one (dy, dx) row-group offset the three tap
// matrices sit side by side in shared memory, so one tcgen05.mma with
// N = 3 COUT computes all three contributions from one read of the A operand
// (the staged input rows): 9 MMAs of N = 48 per output plane for 16 -> 16
// instead of 27 of N = 16, a third of the operand traffic from shared memory.
// The accumulators of consecutive outputs are consecutive COUT-column slots of
// a TMEM ring of R slots; an output range that wraps around the ring is split
// into two MMAs, and an output's first contribution (triple j = k, first
// (dy, dx, k16) step) is its own MMA with accumulation off.  Output k is final
// after triple k+2: its epilogue runs while the tensor core works on triple
// k+3.
template <int CIN, int COUT>
struct ZfCfg {
  static constexpr int kST = zm_stages<CIN, COUT>();
  static constexpr int kWTap = COUT * CIN * 2;
  static constexpr int kWBytes = 27 * kWTap;
  static constexpr int kRGBytes = kRG * CIN * 2;
  static constexpr int kTriple = 3 * kRGBytes;
  static constexpr int kSmem = kWBytes + kST * kTriple;
  static constexpr int kR = 256 / COUT;  // accumulator slots: 256 TMEM columns
  static constexpr uint32_t kCols = 256;
  static_assert(kSmem <= 227 * 1024, "shared memory");
  static_assert(kR >= 4, "the ring must hold the three outputs in work and one in its epilogue");
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(128)
conv_fwd_zf_kernel(const uint16_t* __restrict__ x, const uint16_t* __restrict__ w,
                   const float* __restrict__ bias, const uint16_t* __restrict__ mask,
                   uint16_t* __restrict__ y, Vol g, int flags, ZmGrid zg) {
  using Cfg = ZfCfg<CIN, COUT>;
  constexpr int ST = Cfg::kST;
  constexpr int R = Cfg::kR;
  constexpr int kc = CIN / 8;
  constexpr int kChunks = 3 * kRG * kc;            // 16-byte copies per triple
  constexpr int kPer = (kChunks + 127) / 128;      // per thread
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t tbase;
  __shared__ float sbias[COUT];
  unsigned char* sW = sm;
  unsigned char* sR = sm + Cfg::kWBytes;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // tap t = dz * 9 + dy * 3 + dx goes to tile (dy * 3 + dx) * 3 + (2 - dz): the
  // taps of one (dy, dx) are consecutive K-major tiles in the order dz = 2, 1, 0,
  // i.e. one B operand of N = 3 COUT rows
  for (int i = tid; i < 27 * COUT * kc; i += 128) {
    const int c = i % kc, r = (i / kc) % COUT, t = i / (kc * COUT);
    const int tt = (t % 9) * 3 + (2 - t / 9);
    const uint4 v = *reinterpret_cast<const uint4*>(w + ((size_t)t * COUT + r) * CIN + c * 8);
    *reinterpret_cast<uint4*>(sW + tt * Cfg::kWTap + tc::kmajor_off(r, c * 8, CIN)) = v;
  }
  if (tid < COUT) sbias[tid] = bias ? bias[tid] : 0.f;
  if (tid == 0) {
    tc::mbar_init(&bars[0], 1);
    tc::mbar_init(&bars[1], 1);
  }
  if (warp == 0) tc::tmem_alloc(&tbase, Cfg::kCols);
  int roff[kPer], coff[kPer];
  uint32_t soff[kPer];
#pragma unroll
  for (int m = 0; m < kPer; ++m) {
    const int i = tid + 128 * m;
    const int c = i % kc, v = (i / kc) % kRG, gi = i / (kc * kRG);
    roff[m] = gi * g.wp + v;
    coff[m] = c * 8;
    soff[m] = (uint32_t)(gi * Cfg::kRGBytes + c * (kRG * 16) + v * 16);
  }
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t acc0 = tbase;
  const uint64_t adesc0 = tc::smem_desc(tc::smem_addr(sR), kRG * 16, 128);
  const uint64_t bdesc0 = tc::smem_desc(tc::smem_addr(sW), 128, kc * 128);

  bool abort = false;
  int tg = 0;     // triples issued by this CTA (barrier phase)
  int obase = 0;  // outputs of earlier units (accumulator ring position)
  for (int u = blockIdx.x; u < zg.units && !abort; u += gridDim.x) {
    const int bi = u % zg.nb, cz = u / zg.nb;
    const int sidx = cz / zg.nzc;
    const int z0 = (cz % zg.nzc) * zg.zc;
    const int nout = min(zg.zc, g.nz - z0);
    const int kp0 = sidx * g.dp + 1 + z0;  // padded plane of output 0
    const int seg = bi * 128;
    const int ntrip = nout + 2;            // triples: planes kp0-1 .. kp0+nout
    const int poff = seg + warp * 32 + lane;
    const int px = poff % g.wp, py = poff / g.wp;
    const bool in_xy = poff < g.pp && px >= 1 && px <= g.nx && py >= 1 && py <= g.ny;
    auto load_triple = [&](int j) {
      if (j < ntrip) {
        const int base = seg + (kp0 - 1 + j) * g.pp - g.wp - 1;
        unsigned char* st = sR + (j % ST) * Cfg::kTriple;
#pragma unroll
        for (int m = 0; m < kPer; ++m) {
          if (kChunks % 128 == 0 || tid + 128 * m < kChunks) {
            const int row = base + roff[m];
            const bool ok = row >= 0 && row < g.vp;
            cp16z(st + soff[m], x + (size_t)(ok ? row : 0) * CIN + coff[m], ok);
          }
        }
      }
      cp_commit_group();
    };
    for (int j = 0; j < ST; ++j) load_triple(j);

    auto epilogue = [&](int k) {
      const size_t idx = (size_t)(kp0 + k) * g.pp + poff;
      const uint32_t acc = acc0 + (uint32_t)(((obase + k) % R) * COUT);
      float va[COUT];
      tc::tmem_ld_cols<COUT>(acc + ((uint32_t)(warp * 32) << 16), va);
#pragma unroll
      for (int c0 = 0; c0 < COUT; c0 += 8) {
        const float* v = va + c0;
        if (in_xy) {
          uint4 mk = make_uint4(0, 0, 0, 0);
          if (flags & kConvMask) mk = *reinterpret_cast<const uint4*>(mask + idx * COUT + c0);
          const uint32_t mw[4] = {mk.x, mk.y, mk.z, mk.w};
          uint32_t ov[4];
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            float a = v[2 * h] + sbias[c0 + 2 * h], b = v[2 * h + 1] + sbias[c0 + 2 * h + 1];
            if (flags & kConvRelu) {
              a = fmaxf(a, 0.f);
              b = fmaxf(b, 0.f);
            }
            if (flags & kConvMask) {
              if (!bf16_positive(mw[h] & 0xffffu)) a = 0.f;
              if (!bf16_positive(mw[h] >> 16)) b = 0.f;
            }
            ov[h] = pack_bf16(a, b);
          }
          *reinterpret_cast<uint4*>(y + idx * COUT + c0) = make_uint4(ov[0], ov[1], ov[2], ov[3]);
        }
      }
    };

    for (int j = 0; j < ntrip; ++j, ++tg) {
      cp_wait_groups<ST - 2>();  // triple j is complete
      tc::fence_proxy_async();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after();
        const int klo = max(0, j - 2), khi = min(nout - 1, j);
        const uint64_t slot = adesc0 + (uint64_t)((j % ST) * (Cfg::kTriple >> 4));
        // outputs ka..kb of this triple, one (dy, dx, k16) step: B tiles
        // consecutive from the tile of output ka, D slots consecutive modulo R
        auto mma_range = [&](int ka, int kb, uint64_t ad, int tile0, int ks, bool accum) {
          int k = ka;
          while (k <= kb) {
            const int sl = (obase + k) % R;
            const int n = min(kb - k + 1, R - sl);
            const uint64_t bd =
                bdesc0 + (uint64_t)(((tile0 + (k - ka)) * Cfg::kWTap + ks * 256) >> 4);
            tc::mma_bf16(acc0 + (uint32_t)(sl * COUT), ad, bd, tc::idesc_bf16_f32(128, n * COUT),
                         accum);
            k += n;
          }
        };
#pragma unroll 1
        for (int gi = 0; gi < 3; ++gi)
#pragma unroll
          for (int dx = 0; dx < 3; ++dx)
#pragma unroll
            for (int ks = 0; ks < CIN / 16; ++ks) {
              const uint64_t ad =
                  slot + (uint64_t)((gi * Cfg::kRGBytes + dx * 16 + ks * 2 * kRG * 16) >> 4);
              // tile of output ka: (dy, dx) group, index 2 - dz with dz = j - ka
              const int grp = (gi * 3 + dx) * 3 + 2 - j;
              const bool first = (gi | dx | ks) == 0;
              if (first && khi == j) {  // output j starts here: accumulation off for it
                if (klo < j) mma_range(klo, j - 1, ad, grp + klo, ks, true);
                mma_range(j, j, ad, grp + j, ks, false);
              } else {
                mma_range(klo, khi, ad, grp + klo, ks, true);
              }
            }
        tc::mma_commit(&bars[tg & 1]);
      }
      if (j >= 1) {
        // triple j-1's MMAs are done: its ring slot is free, and output j-3 is final
        const bool ok = tc::mbar_wait(&bars[(tg - 1) & 1], ((tg - 1) >> 1) & 1, kWaitLimit);
        if (__syncthreads_or(!ok)) {
          abort = true;
          break;
        }
        load_triple(j - 1 + ST);
        if (j >= 3) {
          tc::fence_after();
          epilogue(j - 3);
          tc::fence_before();
        }
      } else {
        cp_commit_group();
      }
    }
    if (abort) break;
    {  // the last output of the unit
      const bool ok = tc::mbar_wait(&bars[(tg - 1) & 1], ((tg - 1) >> 1) & 1, kWaitLimit);
      if (__syncthreads_or(!ok)) {
        abort = true;
        break;
      }
      tc::fence_after();
      epilogue(nout - 1);
      tc::fence_before();
    }
    obase += nout;
    cp_wait_all();
    __syncthreads();  // ring slots are rewritten by the next unit
  }
  cp_wait_all();
  if (abort && tid == 0) atomicOr(&g_tc_timeout, 1);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(acc0, Cfg::kCols);
}

// ---- the folded z-marching kernel with warp-specialised roles -------------
// Same work units, row-group triples, folded MMAs (N = 3 cout) and TMEM ring
// of accumulators as conv_fwd_zf_kernel, but the three kinds of work no
// longer wait for each other at a block barrier:
//   warp 4 copies triples into a ring of ST slots (cp.async); once the next
//          triple's copies are issued, each lane waits for its copies of the
//          previous one, fences them to the async proxy and arrives on that
//          slot's "full" mbarrier;
//   warp 5 (one thread) issues the MMAs of a triple once it is full and the
//          slot of the output it starts is free, and commits to the triple's
//          "empty" barrier and to the "full" barrier of the output the triple
//          completes;
//   warps 0-3 (the four TMEM lane quarters) drain finished accumulators:
//          load, release the slot ("empty"), then bias / ReLU / mask, BF16
//          rounding and the stores.
// Every wait is bounded; a wait that runs out raises a shared abort flag that
// every role checks, and the kernel records the timeout like the others.
template <int CIN, int COUT>
struct WsCfg {
  static constexpr int kST = zm_stages<CIN, COUT>();
  static constexpr int kWTap = COUT * CIN * 2;
  static constexpr int kWBytes = 27 * kWTap;
  static constexpr int kRGBytes = kRG * CIN * 2;
  static constexpr int kTriple = 3 * kRGBytes;
  static constexpr int kSmem = kWBytes + kST * kTriple;
  static constexpr int kR = 256 / COUT;
  static constexpr uint32_t kCols = 256;
  static_assert(kSmem <= 227 * 1024, "shared memory");
  static_assert(kR >= 4, "accumulator ring");
};

__device__ __forceinline__ void mbar_arrive1(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_addr(bar)) : "memory");
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(192)
conv_fwd_ws_kernel(const uint16_t* __restrict__ x, const uint16_t* __restrict__ w,
                   const float* __restrict__ bias, const uint16_t* __restrict__ mask,
                   uint16_t* __restrict__ y, Vol g, int flags, ZmGrid zg) {
  using Cfg = WsCfg<CIN, COUT>;
  constexpr int ST = Cfg::kST;
  constexpr int R = Cfg::kR;
  constexpr int kc = CIN / 8;
  constexpr int kChunks = 3 * kRG * kc;  // 16-byte copies per triple
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) uint64_t tfull[ST], tempty[ST], afull[R], aempty[R], done_bar;
  __shared__ uint32_t tbase;
  __shared__ float sbias[COUT];
  __shared__ volatile int s_abort;
  unsigned char* sW = sm;
  unsigned char* sR = sm + Cfg::kWBytes;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // weights in the folded order (see conv_fwd_zf_kernel)
  for (int i = tid; i < 27 * COUT * kc; i += 192) {
    const int c = i % kc, r = (i / kc) % COUT, t = i / (kc * COUT);
    const int tt = (t % 9) * 3 + (2 - t / 9);
    const uint4 v = *reinterpret_cast<const uint4*>(w + ((size_t)t * COUT + r) * CIN + c * 8);
    *reinterpret_cast<uint4*>(sW + tt * Cfg::kWTap + tc::kmajor_off(r, c * 8, CIN)) = v;
  }
  if (tid < COUT) sbias[tid] = bias ? bias[tid] : 0.f;
  if (tid == 0) {
    for (int i = 0; i < ST; ++i) {
      tc::mbar_init(&tfull[i], 32);
      tc::mbar_init(&tempty[i], 1);
    }
    for (int i = 0; i < R; ++i) {
      tc::mbar_init(&afull[i], 1);
      tc::mbar_init(&aempty[i], 4);
    }
    tc::mbar_init(&done_bar, 1);
    s_abort = 0;
  }
  if (warp == 5) tc::tmem_alloc(&tbase, Cfg::kCols);
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t acc0 = tbase;

  auto wait = [&](uint64_t* bar, uint32_t parity) -> bool {
    if (s_abort) return false;
    if (tc::mbar_wait(bar, parity, kWaitLimit)) return true;
    s_abort = 1;
    return false;
  };

  if (warp == 4) {
    // ---- copy warp -----------------------------------------------------------
    // A triple is handed to the tensor core once the copies of the next one
    // are issued: each lane waits for its own copies of the triple, makes
    // them visible to the async proxy (the MMAs read shared memory through
    // it), then arrives on the triple's "full" barrier.
    int tg = 0, pend = -1;  // pend: slot of the triple whose arrival is due
    auto hand_over = [&](bool last) {
      if (pend < 0) return;
      if (last) cp_wait_all();
      else cp_wait_groups<1>();
      tc::fence_proxy_async();
      mbar_arrive1(&tfull[pend]);
      pend = -1;
    };
    for (int u = blockIdx.x; u < zg.units && !s_abort; u += gridDim.x) {
      const int bi = u % zg.nb, cz = u / zg.nb;
      const int sidx = cz / zg.nzc;
      const int z0 = (cz % zg.nzc) * zg.zc;
      const int nout = min(zg.zc, g.nz - z0);
      const int kp0 = sidx * g.dp + 1 + z0;
      const int seg = bi * 128;
      for (int j = 0; j < nout + 2; ++j, ++tg) {
        const int s = tg % ST;
        if (tg >= ST && !wait(&tempty[s], ((tg / ST) - 1) & 1)) break;
        const int base = seg + (kp0 - 1 + j) * g.pp - g.wp - 1;
        unsigned char* st = sR + s * Cfg::kTriple;
        for (int i = lane; i < kChunks; i += 32) {
          const int c = i % kc, v = (i / kc) % kRG, gi = i / (kc * kRG);
          const int row = base + gi * g.wp + v;
          const bool ok = row >= 0 && row < g.vp;
          cp16z(st + gi * Cfg::kRGBytes + c * (kRG * 16) + v * 16,
                x + (size_t)(ok ? row : 0) * CIN + c * 8, ok);
        }
        cp_commit_group();
        hand_over(false);  // the previous triple
        pend = s;
      }
    }
    hand_over(true);
    cp_wait_all();
  } else if (warp == 5) {
    // ---- MMA thread --------------------------------------------------------
    if (lane == 0) {
      const uint64_t adesc0 = tc::smem_desc(tc::smem_addr(sR), kRG * 16, 128);
      const uint64_t bdesc0 = tc::smem_desc(tc::smem_addr(sW), 128, kc * 128);
      int tg = 0, obase = 0;
      bool stop = false;
      for (int u = blockIdx.x; u < zg.units && !stop; u += gridDim.x) {
        const int cz = u / zg.nb;
        const int z0 = (cz % zg.nzc) * zg.zc;
        const int nout = min(zg.zc, g.nz - z0);
        for (int j = 0; j < nout + 2; ++j, ++tg) {
          const int s = tg % ST;
          if (!wait(&tfull[s], (tg / ST) & 1)) { stop = true; break; }
          const int klo = max(0, j - 2), khi = min(nout - 1, j);
          if (khi == j) {  // output j starts here: its accumulator slot must be free
            const int oc = obase + j;
            if (oc >= R && !wait(&aempty[oc % R], ((oc / R) - 1) & 1)) { stop = true; break; }
          }
          tc::fence_after();
          const uint64_t slot = adesc0 + (uint64_t)(s * (Cfg::kTriple >> 4));
          auto mma_range = [&](int ka, int kb, uint64_t ad, int tile0, int ks, bool accum) {
            int k = ka;
            while (k <= kb) {
              const int sl = (obase + k) % R;
              const int n = min(kb - k + 1, R - sl);
              const uint64_t bd =
                  bdesc0 + (uint64_t)(((tile0 + (k - ka)) * Cfg::kWTap + ks * 256) >> 4);
              tc::mma_bf16(acc0 + (uint32_t)(sl * COUT), ad, bd,
                           tc::idesc_bf16_f32(128, n * COUT), accum);
              k += n;
            }
          };
#pragma unroll 1
          for (int gi = 0; gi < 3; ++gi)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx)
#pragma unroll
              for (int ks = 0; ks < CIN / 16; ++ks) {
                const uint64_t ad =
                    slot + (uint64_t)((gi * Cfg::kRGBytes + dx * 16 + ks * 2 * kRG * 16) >> 4);
                const int grp = (gi * 3 + dx) * 3 + 2 - j;
                if ((gi | dx | ks) == 0 && khi == j) {
                  if (klo < j) mma_range(klo, j - 1, ad, grp + klo, ks, true);
                  mma_range(j, j, ad, grp + j, ks, false);
                } else {
                  mma_range(klo, khi, ad, grp + klo, ks, true);
                }
              }
          tc::mma_commit(&tempty[s]);
          if (j >= 2) tc::mma_commit(&afull[(obase + j - 2) % R]);  // output j-2 is final
        }
        obase += nout;
      }
      // every MMA issued must be complete before the TMEM is released
      tc::mma_commit(&done_bar);
      if (!tc::mbar_wait(&done_bar, 0, kWaitLimit)) s_abort = 1;
    }
  } else {
    // ---- epilogue warps 0-3: TMEM lanes 32 warp .. 32 warp + 31 -------------
    int obase = 0;
    for (int u = blockIdx.x; u < zg.units && !s_abort; u += gridDim.x) {
      const int bi = u % zg.nb, cz = u / zg.nb;
      const int sidx = cz / zg.nzc;
      const int z0 = (cz % zg.nzc) * zg.zc;
      const int nout = min(zg.zc, g.nz - z0);
      const int kp0 = sidx * g.dp + 1 + z0;
      const int poff = bi * 128 + warp * 32 + lane;
      const int px = poff % g.wp, py = poff / g.wp;
      const bool in_xy = poff < g.pp && px >= 1 && px <= g.nx && py >= 1 && py <= g.ny;
      bool stop = false;
      for (int k = 0; k < nout; ++k) {
        const int oc = obase + k;
        const int sl = oc % R;
        if (!wait(&afull[sl], (oc / R) & 1)) { stop = true; break; }
        tc::fence_after();
        float va[COUT];
        tc::tmem_ld_cols<COUT>(acc0 + ((uint32_t)(warp * 32) << 16) + (uint32_t)(sl * COUT), va);
        tc::fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive1(&aempty[sl]);
        if (in_xy) {
          const size_t idx = (size_t)(kp0 + k) * g.pp + poff;
#pragma unroll
          for (int c0 = 0; c0 < COUT; c0 += 8) {
            const float* v = va + c0;
            uint4 mk = make_uint4(0, 0, 0, 0);
            if (flags & kConvMask) mk = *reinterpret_cast<const uint4*>(mask + idx * COUT + c0);
            const uint32_t mw[4] = {mk.x, mk.y, mk.z, mk.w};
            uint32_t ov[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              float a = v[2 * h] + sbias[c0 + 2 * h], b = v[2 * h + 1] + sbias[c0 + 2 * h + 1];
              if (flags & kConvRelu) {
                a = fmaxf(a, 0.f);
                b = fmaxf(b, 0.f);
              }
              if (flags & kConvMask) {
                if (!bf16_positive(mw[h] & 0xffffu)) a = 0.f;
                if (!bf16_positive(mw[h] >> 16)) b = 0.f;
              }
              ov[h] = pack_bf16(a, b);
            }
            *reinterpret_cast<uint4*>(y + idx * COUT + c0) = make_uint4(ov[0], ov[1], ov[2], ov[3]);
          }
        }
      }
      if (stop) break;
      obase += nout;
    }
  }
  tc::fence_before();
  __syncthreads();
  if (s_abort && tid == 0) atomicOr(&g_tc_timeout, 1);
  if (warp == 5) tc::tmem_dealloc(acc0, Cfg::kCols);
}

template <int CIN, int COUT>
struct WgCfg {
  static constexpr int kTaps = 128 / CIN;                    // taps per 128-row tile
  static constexpr int kMTiles = (27 + kTaps - 1) / kTaps;
  static constexpr int kKV = 64;                             // voxels per reduction chunk
  static constexpr int kABytes = 128 * kKV * 2;
  static constexpr int kBBytes = COUT * kKV * 2;
  static constexpr int kStage = kABytes + kBBytes;
  static constexpr int kSmem = 2 * kStage;
  static constexpr uint32_t kCols = COUT < 32 ? 32 : COUT;
  static_assert(128 % CIN == 0, "CIN must divide 128");
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(128)
conv_wgrad_kernel(const uint16_t* __restrict__ x, const uint16_t* __restrict__ dy,
                  float* __restrict__ ws, Vol g, int nchunks) {
  using Cfg = WgCfg<CIN, COUT>;
  constexpr int kKV = Cfg::kKV;
  constexpr int kAB = Cfg::kTaps * (CIN / 8) * (kKV / 8);  // 8x8 blocks of A per chunk
  constexpr int kBB = (COUT / 8) * (kKV / 8);              // 8x8 blocks of B per chunk
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mt = blockIdx.x, split = blockIdx.y, nsplit = gridDim.y;
  const int my = (nchunks - split + nsplit - 1) / nsplit;

  if (tid == 0) {
    tc::mbar_init(&bars[0], 1);
    tc::mbar_init(&bars[1], 1);
  }
  if (warp == 0) tc::tmem_alloc(&tbase, Cfg::kCols);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t acc = tbase;
  bool abort = false;

  for (int i = 0; i < my; ++i) {
    const int buf = i & 1;
    if (i >= 2) {
      const bool ok = tc::mbar_wait(&bars[buf], ((i - 2) >> 1) & 1, kWaitLimit);
      if (__syncthreads_or(!ok)) {
        abort = true;
        break;
      }
    }
    const int v0 = g.g0 + (split + i * nsplit) * kKV;
    unsigned char* sA = sm + buf * Cfg::kStage;
    unsigned char* sB = sA + Cfg::kABytes;
    for (int b = warp; b < kAB + kBB; b += 4) {
      uint32_t val = 0;
      if (b < kAB) {
        const int vb = b % 8, cb = (b / 8) % (CIN / 8), tl = b / (8 * (CIN / 8));
        const int t = mt * Cfg::kTaps + tl;
        if (t < 27) {
          const int off = (t / 9 - 1) * g.pp + ((t / 3) % 3 - 1) * g.wp + (t % 3 - 1);
          const int v = v0 + vb * 8 + (lane >> 2) + off;
          if (v >= 0 && v < g.vp)
            val = *reinterpret_cast<const uint32_t*>(x + (size_t)v * CIN + cb * 8 + 2 * (lane & 3));
        }
        val = movmatrix_trans(val);
        *reinterpret_cast<uint32_t*>(
            sA + tc::kmajor_off(tl * CIN + cb * 8 + (lane >> 2), vb * 8 + 2 * (lane & 3), kKV)) = val;
      } else {
        const int bb = b - kAB, vb = bb % 8, cb = bb / 8;
        const int v = v0 + vb * 8 + (lane >> 2);
        if (v < g.g1)
          val = *reinterpret_cast<const uint32_t*>(dy + (size_t)v * COUT + cb * 8 + 2 * (lane & 3));
        val = movmatrix_trans(val);
        *reinterpret_cast<uint32_t*>(
            sB + tc::kmajor_off(cb * 8 + (lane >> 2), vb * 8 + 2 * (lane & 3), kKV)) = val;
      }
    }
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      constexpr uint32_t idesc = tc::idesc_bf16_f32(128, COUT);
      const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sB);
#pragma unroll
      for (int ks = 0; ks < kKV / 16; ++ks)
        tc::mma_bf16(acc, tc::smem_desc(a0 + ks * 256, 128, (kKV / 8) * 128),
                     tc::smem_desc(b0 + ks * 256, 128, (kKV / 8) * 128), idesc, (i | ks) != 0);
      tc::mma_commit(&bars[buf]);
    }
  }
  if (!abort && my > 0) {
    const bool ok = tc::mbar_wait(&bars[(my - 1) & 1], ((my - 1) >> 1) & 1, kWaitLimit);
    if (__syncthreads_or(!ok)) abort = true;
  }
  tc::fence_after();
  float* out = ws + ((size_t)(split * gridDim.x + mt) * 128 + warp * 32 + lane) * COUT;
  if (!abort && my > 0) {
#pragma unroll
    for (int c0 = 0; c0 < COUT; c0 += 8) {
      float v[8];
      tc::tmem_ld8(acc + ((uint32_t)(warp * 32) << 16) + c0, v);
      *reinterpret_cast<float4*>(out + c0) = make_float4(v[0], v[1], v[2], v[3]);
      *reinterpret_cast<float4*>(out + c0 + 4) = make_float4(v[4], v[5], v[6], v[7]);
    }
  } else {
    for (int c = 0; c < COUT; ++c) out[c] = 0.f;
    if (abort && tid == 0) atomicOr(&g_tc_timeout, 1);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(acc, Cfg::kCols);
}

template <int CIN, int COUT>
__global__ void wgrad_reduce_kernel(const float* __restrict__ ws, float* __restrict__ dw,
                                    int nsplit, int accumulate) {
  using Cfg = WgCfg<CIN, COUT>;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 27 * COUT * CIN) return;
  const int ci = i % CIN, co = (i / CIN) % COUT, t = i / (CIN * COUT);
  const int mt = t / Cfg::kTaps, row = (t % Cfg::kTaps) * CIN + ci;
  double s = 0.0;
  for (int sp = 0; sp < nsplit; ++sp)
    s += ws[((size_t)(sp * Cfg::kMTiles + mt) * 128 + row) * COUT + co];
  dw[i] = accumulate ? (float)(dw[i] + s) : (float)s;
}

// CTAs per SM from the shared-memory and tensor-memory budgets (the occupancy
// calculator does not see TMEM), with the carveout set to all shared memory
int ctas_per_sm(const void* fn, int smem, uint32_t tmem_cols, int* nsm) {
  int dev = 0, per_sm_smem = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&per_sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  int b = per_sm_smem / (smem + 1024);  // 1 KB reserved per CTA
  const int bt = (int)(512 / tmem_cols);
  if (b > bt) b = bt;
  if (b > 8) b = 8;
  return b < 1 ? 1 : b;
}

template <int CIN, int COUT>
int fwd_grid(int ntiles) {
  static int per_sm = -1, nsm = 0;
  if (per_sm < 0)
    per_sm = ctas_per_sm((const void*)conv_fwd_kernel<CIN, COUT>, FwdCfg<CIN, COUT>::kSmem,
                         FwdCfg<CIN, COUT>::kCols, &nsm);
  const int cap = per_sm * nsm;
  return ntiles < cap ? ntiles : cap;
}

template <int CIN, int COUT>
cudaError_t fwd_launch(const uint16_t* x, const uint16_t* w, const float* bias,
                       const uint16_t* mask, uint16_t* y, const Vol& g, int flags,
                       cudaStream_t s) {
  const int ntiles = (g.g1 - g.g0 + 127) / 128;
  if (ntiles <= 0) return cudaSuccess;
  const int grid = fwd_grid<CIN, COUT>(ntiles);
  conv_fwd_kernel<CIN, COUT><<<grid, 128, FwdCfg<CIN, COUT>::kSmem, s>>>(x, w, bias, mask, y, g,
                                                                        flags, ntiles);
  return cudaGetLastError();
}

template <int CIN, int COUT>
cudaError_t zm_launch(const uint16_t* x, const uint16_t* w, const float* bias,
                      const uint16_t* mask, uint16_t* y, const Vol& g, int flags,
                      cudaStream_t s) {
  static int per_sm = -1, nsm = 0;
  if (per_sm < 0)
    per_sm = ctas_per_sm((const void*)conv_fwd_zm_kernel<CIN, COUT>, ZmCfg<CIN, COUT>::kSmem,
                         ZmCfg<CIN, COUT>::kCols, &nsm);
  const int ctas = per_sm * nsm;
  ZmGrid zg;
  zg.nb = (g.pp + 127) / 128;
  zg.zc = g.nz;
  // shorter z runs until there are at least two units per resident CTA
  while (zg.zc > 4 && (long long)zg.nb * g.ns * ((g.nz + zg.zc - 1) / zg.zc) < 2LL * ctas)
    zg.zc = (zg.zc + 1) / 2;
  zg.nzc = (g.nz + zg.zc - 1) / zg.zc;
  zg.units = zg.nb * g.ns * zg.nzc;
  const int grid = zg.units < ctas ? zg.units : ctas;
  conv_fwd_zm_kernel<CIN, COUT><<<grid, 128, ZmCfg<CIN, COUT>::kSmem, s>>>(x, w, bias, mask, y,
                                                                           g, flags, zg);
  return cudaGetLastError();
}

template <int CIN, int COUT>
cudaError_t zf_launch(const uint16_t* x, const uint16_t* w, const float* bias,
                      const uint16_t* mask, uint16_t* y, const Vol& g, int flags,
                      cudaStream_t s) {
  static int per_sm = -1, nsm = 0;
  if (per_sm < 0)
    per_sm = ctas_per_sm((const void*)conv_fwd_zf_kernel<CIN, COUT>, ZfCfg<CIN, COUT>::kSmem,
                         ZfCfg<CIN, COUT>::kCols, &nsm);
  const int ctas = per_sm * nsm;
  ZmGrid zg;
  zg.nb = (g.pp + 127) / 128;
  zg.zc = g.nz;
  // shorter z runs until there are at least two units per resident CTA
  while (zg.zc > 4 && (long long)zg.nb * g.ns * ((g.nz + zg.zc - 1) / zg.zc) < 2LL * ctas)
    zg.zc = (zg.zc + 1) / 2;
  zg.nzc = (g.nz + zg.zc - 1) / zg.zc;
  zg.units = zg.nb * g.ns * zg.nzc;
  const int grid = zg.units < ctas ? zg.units : ctas;
  conv_fwd_zf_kernel<CIN, COUT><<<grid, 128, ZfCfg<CIN, COUT>::kSmem, s>>>(x, w, bias, mask, y,
                                                                           g, flags, zg);
  return cudaGetLastError();
}

template <int CIN, int COUT>
cudaError_t ws_launch(const uint16_t* x, const uint16_t* w, const float* bias,
                      const uint16_t* mask, uint16_t* y, const Vol& g, int flags,
                      cudaStream_t s) {
  static int per_sm = -1, nsm = 0;
  if (per_sm < 0)
    per_sm = ctas_per_sm((const void*)conv_fwd_ws_kernel<CIN, COUT>, WsCfg<CIN, COUT>::kSmem,
                         WsCfg<CIN, COUT>::kCols, &nsm);
  const int ctas = per_sm * nsm;
  ZmGrid zg;
  zg.nb = (g.pp + 127) / 128;
  zg.zc = g.nz;
  while (zg.zc > 4 && (long long)zg.nb * g.ns * ((g.nz + zg.zc - 1) / zg.zc) < 2LL * ctas)
    zg.zc = (zg.zc + 1) / 2;
  zg.nzc = (g.nz + zg.zc - 1) / zg.zc;
  zg.units = zg.nb * g.ns * zg.nzc;
  const int grid = zg.units < ctas ? zg.units : ctas;
  conv_fwd_ws_kernel<CIN, COUT><<<grid, 192, WsCfg<CIN, COUT>::kSmem, s>>>(x, w, bias, mask, y,
                                                                           g, flags, zg);
  return cudaGetLastError();
}

int wgrad_splits(int mtiles, int nchunks) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int ns = (2 * nsm + mtiles - 1) / mtiles;
  if (ns > nchunks) ns = nchunks;
  return ns < 1 ? 1 : ns;
}

template <int CIN, int COUT>
cudaError_t wgrad_launch(const uint16_t* x, const uint16_t* dy, float* dw, float* ws,
                         const Vol& g, int accumulate, cudaStream_t s) {
  using Cfg = WgCfg<CIN, COUT>;
  const int nchunks = (g.g1 - g.g0 + Cfg::kKV - 1) / Cfg::kKV;
  const int nsplit = wgrad_splits(Cfg::kMTiles, nchunks);
  if (nchunks > 0) {
    cudaFuncSetAttribute(conv_wgrad_kernel<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         Cfg::kSmem);
    conv_wgrad_kernel<CIN, COUT>
        <<<dim3(Cfg::kMTiles, nsplit), 128, Cfg::kSmem, s>>>(x, dy, ws, g, nchunks);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int n = 27 * COUT * CIN;
  wgrad_reduce_kernel<CIN, COUT><<<(n + 255) / 256, 256, 0, s>>>(ws, dw, nchunks > 0 ? nsplit : 0,
                                                                  accumulate);
  return cudaGetLastError();
}

}  // namespace

bool vol_ok(int nx, int ny, int nz, int ns) {
  if (nx < 1 || ny < 1 || nz < 1 || ns < 1) return false;
  const double v = (double)(nx + 2) * (ny + 2) * (nz + 2) * ns;
  return v + 4.0 * (nx + 2) * (ny + 2) < 2147483647.0 / 2;
}

bool conv_shape_ok(int cin, int cout) {
  return (cin == 16 && (cout == 16 || cout == 32)) || (cin == 32 && (cout == 16 || cout == 64)) ||
         (cin == 64 && cout == 32);
}

#define TPFA_CONV_SHAPES(X) X(16, 16) X(16, 32) X(32, 16) X(32, 64) X(64, 32)

// 0: tile kernel, 1: z-marching kernel, 2: z-marching kernel with the z-taps
// folded into N, 4: the folded kernel with warp-specialised roles (1, 2 and 4
// where their ring fits), 3: per layer shape the fastest as measured on GB300
// (default: 1 for 32 -> 16, 4 otherwise)
static int g_conv_kernel = 3;

cudaError_t conv_fwd(const uint16_t* x, const uint16_t* w, const float* bias, const uint16_t* mask,
                     uint16_t* y, const Vol& g, int cin, int cout, int flags, cudaStream_t s) {
  const bool ring = !(cin == 64 && cout == 32);
  const int kern = g_conv_kernel != 3 ? g_conv_kernel : (cin == 32 && cout == 16 ? 1 : 4);
  if (ring && kern == 4) {
#define X(CI, CO) \
  if (cin == CI && cout == CO) return ws_launch<CI, CO>(x, w, bias, mask, y, g, flags, s);
    X(16, 16) X(16, 32) X(32, 16) X(32, 64)
#undef X
  }
  if (ring && kern == 2) {
#define X(CI, CO) \
  if (cin == CI && cout == CO) return zf_launch<CI, CO>(x, w, bias, mask, y, g, flags, s);
    X(16, 16) X(16, 32) X(32, 16) X(32, 64)
#undef X
  }
  if (ring && kern == 1) {
#define X(CI, CO) \
  if (cin == CI && cout == CO) return zm_launch<CI, CO>(x, w, bias, mask, y, g, flags, s);
    X(16, 16) X(16, 32) X(32, 16) X(32, 64)
#undef X
  }
#define X(CI, CO) \
  if (cin == CI && cout == CO) return fwd_launch<CI, CO>(x, w, bias, mask, y, g, flags, s);
  TPFA_CONV_SHAPES(X)
#undef X
  return cudaErrorInvalidValue;
}

size_t conv_wgrad_ws_bytes(const Vol& g, int cin, int cout) {
  const int mtiles = (27 + 128 / cin - 1) / (128 / cin);
  const int nchunks = (g.g1 - g.g0 + 63) / 64;
  const int ns = wgrad_splits(mtiles, nchunks < 1 ? 1 : nchunks);
  return (size_t)ns * mtiles * 128 * cout * sizeof(float);
}

cudaError_t conv_wgrad(const uint16_t* x, const uint16_t* dy, float* dw, float* ws, const Vol& g,
                       int cin, int cout, int accumulate, cudaStream_t s) {
#define X(CI, CO) \
  if (cin == CI && cout == CO) return wgrad_launch<CI, CO>(x, dy, dw, ws, g, accumulate, s);
  TPFA_CONV_SHAPES(X)
#undef X
  return cudaErrorInvalidValue;
}

}  // namespace net
}  // namespace tpfa

using tpfa::net::Vol;

static int conv_args_ok(const void* x, const void* y, int nx, int ny, int nz, int ns, int cin,
                        int cout, int* dev) {
  if (!tpfa::net::vol_ok(nx, ny, nz, ns) || !tpfa::net::conv_shape_ok(cin, cout))
    return TPFA_EINVAL;
  if (cudaGetDevice(dev) != cudaSuccess) return TPFA_ECUDA;
  const Vol g = tpfa::net::make_vol(nx, ny, nz, ns);
  if (!tpfa::dev_ok(x, (size_t)g.vp * cin * 2, 16, *dev) ||
      !tpfa::dev_ok(y, (size_t)g.vp * cout * 2, 16, *dev))
    return TPFA_EINVAL;
  return TPFA_OK;
}

extern "C" int tpfa_conv3d_bf16(const uint16_t* x, const uint16_t* w, const float* bias,
                                const uint16_t* mask, uint16_t* y, int nx, int ny, int nz,
                                int ns, int cin, int cout, int flags, void* stream) {
  int dev = -1;
  int rc = conv_args_ok(x, y, nx, ny, nz, ns, cin, cout, &dev);
  if (rc != TPFA_OK) return rc;
  if (flags & ~3) return TPFA_EINVAL;
  const Vol g = tpfa::net::make_vol(nx, ny, nz, ns);
  if (!tpfa::dev_ok(w, (size_t)27 * cin * cout * 2, 16, dev) ||
      !tpfa::opt_dev_ok(bias, (size_t)cout * 4, 4, dev))
    return TPFA_EINVAL;
  if ((flags & tpfa::net::kConvMask) && !tpfa::dev_ok(mask, (size_t)g.vp * cout * 2, 16, dev))
    return TPFA_EINVAL;
  if (x == y) return TPFA_EINVAL;
  return tpfa::net::conv_fwd(x, w, bias, mask, y, g, cin, cout, flags, (cudaStream_t)stream) ==
                 cudaSuccess
             ? TPFA_OK
             : TPFA_ECUDA;
}

extern "C" int tpfa_conv3d_wgrad_bf16(const uint16_t* x, const uint16_t* dy, float* dw, int nx,
                                      int ny, int nz, int ns, int cin, int cout, int accumulate,
                                      void* stream) {
  int dev = -1;
  int rc = conv_args_ok(x, dy, nx, ny, nz, ns, cin, cout, &dev);
  if (rc != TPFA_OK) return rc;
  if (!tpfa::dev_ok(dw, (size_t)27 * cin * cout * 4, 4, dev)) return TPFA_EINVAL;
  const Vol g = tpfa::net::make_vol(nx, ny, nz, ns);
  cudaStream_t s = (cudaStream_t)stream;
  float* ws = nullptr;
  if (cudaMallocAsync((void**)&ws, tpfa::net::conv_wgrad_ws_bytes(g, cin, cout), s) != cudaSuccess)
    return TPFA_ENOMEM;
  cudaError_t e = tpfa::net::conv_wgrad(x, dy, dw, ws, g, cin, cout, accumulate, s);
  cudaFreeAsync(ws, s);
  return e == cudaSuccess ? TPFA_OK : TPFA_ECUDA;
}

// Selects the forward convolution kernel: 0 = 128-voxel tiles with all nine
// row groups per tile, 1 = z-marching ring where it fits, 2 = z-marching ring
// with the z-taps folded into N, 3 = per layer shape (default), 4 = the folded
// ring with warp-specialised roles.
extern "C" int tpfa_conv3d_select(int kernel) {
  if (kernel < 0 || kernel > 4) return TPFA_EINVAL;
  tpfa::net::g_conv_kernel = kernel;
  return TPFA_OK;
}

namespace tpfa {
namespace net {
// One block waits, with the bounded wait of every tensor-core kernel here, for
// an mbarrier phase that no thread completes (one arrival expected, none
// made): the wait gives up after `polls` polls and records the timeout the way
// a stalled tensor-core kernel does.  No tensor memory, no tensor-core work.
__global__ void wait_probe_kernel(uint32_t polls) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) tc::mbar_init(&bar, 1);
  __syncthreads();
  const bool ok = tc::mbar_wait(&bar, 0, polls);
  if (!ok && threadIdx.x == 0) atomicOr(&g_tc_timeout, 1);
}
}  // namespace net
}  // namespace tpfa

// Test hook for the failure path of the bounded waits (see the header).
extern "C" int tpfa_tc_wait_probe(uint32_t polls, void* stream) {
  if (polls < 1 || polls > tpfa::net::kWaitLimit) return TPFA_EINVAL;
  tpfa::net::wait_probe_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(polls);
  return cudaGetLastError() == cudaSuccess ? TPFA_OK : TPFA_ECUDA;
}

// Waits for the stream, then reports (and clears) a tensor-core wait that
// gave up in any kernel of this library since the last call.
extern "C" int tpfa_net_status(void* stream) {
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return TPFA_ECUDA;
  int h = 0;
  if (cudaMemcpyFromSymbol(&h, tpfa::net::g_tc_timeout, sizeof(int)) != cudaSuccess)
    return TPFA_ECUDA;
  if (h) {
    const int zero = 0;
    cudaMemcpyToSymbol(tpfa::net::g_tc_timeout, &zero, sizeof(int));
    return TPFA_EINTERNAL;
  }
  return TPFA_OK;
}
