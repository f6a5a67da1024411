// Fused CG sweep with its planes staged by the tensor memory accelerator.
//
// Computes what the plain FP32-record CG sweep of kernels_cg.cu computes for
// one iteration of Alg. 1 (arXiv 2408.03452, Section II.A):
// r_k = r_{k-1} - alpha q_{k-1}, p_k = r_k + beta p_{k-1},
// x_k = x_{k-1} + alpha p_{k-1}, q_k = A p_k (Eq. 6 / Alg. 2 in the positive
// form (A p)_K = D_K p_K - sum_f T_f p_nbr) and the four dot products r'r,
// p'q, r'q, q'q, with the same per-cell arithmetic in the same order; only the
// grouping of the dot products' partial sums differs (another tiling).
//
// Vector layout: the four CG vectors of a cell are one 16-byte record
// (r, q, p, x) in FP32, and the sweep reads one set of records and writes the
// other (two sets, ping-ponged).  With the coefficient records that makes
// three DRAM streams per sweep (read records, read vectors, write vectors)
// instead of nine: the same 48 bytes per cell, fewer concurrent access
// streams (a plain copy kernel with this access pattern moves 48 B/cell at
// 6.95 TB/s with three streams against 6.29 TB/s with nine on GB300).
//
// Tiling: a block owns 32 consecutive x-columns (X0 = 32 bx) and TY = W * VY
// y-rows, and marches through a run of zc z-planes.  Warp w (of W compute
// warps) owns rows w*VY .. w*VY+VY-1 of the tile; lane l owns column X0 + l,
// so every output row a warp stores is 512 contiguous bytes.  One more warp
// is the producer: for every plane one of its threads issues two
// cp.async.bulk.tensor loads into a ring of S shared-memory stages,
//   vectors   [TY+2 rows][34 records] from (X0-1, Y0-1)  (x-halo and y-halo),
//   coefficients [TY+1 rows][33 records] from (X0-1, Y0-1) (Tx of x-1, Ty of y-1),
// with out-of-grid elements zero-filled by the copy engine.  x-neighbours
// come from warp shuffles (the two x-halo columns are formed by every lane
// from the stage and used by lanes 0 and 31), y-neighbours from the stage,
// z-neighbours from registers carried plane to plane.  Stages are handed
// over by mbarriers: "full" (transaction bytes of the copies) and "empty"
// (one arrival per compute warp).  Every wait is bounded; a wait that runs
// out records a fault in the CG state, which ends the loop with the guard
// status instead of hanging the GPU.
//
// Requirement of the copy engine: global strides that are multiples of 16
// bytes, which 16-byte records always satisfy (tma_sweep_ok checks the
// driver's tensor-map encoder).
#include <cuda.h>
#include <math.h>
#include <string.h>

#include "sweep_common.cuh"
#include "tc_common.cuh"

namespace tpfa {

namespace {

using tc::mbar_init;
using tc::mbar_wait;
using tc::smem_addr;

constexpr int kVecX = 34;      // vector box width: X0-1 .. X0+32
constexpr int kDinvX = 40;     // M^-1 box width (BF16 Jacobi): X0-4 .. X0+35
constexpr uint32_t kWaitLimit = 1u << 22;  // polls of one mbarrier wait before giving up

// Coefficient records staged per plane, by record type and preconditioner.
//   FP32 records (Tx, Ty, Tz, D), 16 bytes: box from (X0-1, Y0-1), 33 wide and
//   TY+1 rows (Tx of x-1 and Ty of y-1 for the own cells); with Jacobi 34 wide
//   and TY+2 rows, so that D of the halo cells is there too.
//   BF16 records (Tx, Ty, Tz, E), 8 bytes: box from (X0-2, Y0-1) (a 16-byte
//   aligned start), 36 wide, TY+1 rows; D = the six faces + E is formed in the
//   stencil, and with Jacobi M^-1 (from dinv_bf16_kernel) comes from its own
//   FP32 box, 40 wide from (X0-4, Y0-1), TY+2 rows.
template <bool B16, bool JAC>
struct Rec {
  static constexpr int kBytes = B16 ? 8 : 16;
  static constexpr int kX = B16 ? 36 : (JAC ? 34 : 33);  // records per box row
  static constexpr int kC0 = B16 ? 2 : 1;                // box column of x = X0
  static constexpr int kRows = (JAC && !B16) ? 2 : 1;    // box rows beyond TY
  static constexpr bool kDinv = B16 && JAC;
};

struct TmaArgs {
  CUtensorMap mv[2], mc, md;  // vector records (two sets), coefficients, M^-1 (BF16 Jacobi)
  const TmaInst* inst;        // batched sweeps: instance table (ninst entries)
  int ninst;
  Grid g;
  int zc;
  int nbx, nby;  // blocks along x and y
  float4* v4[2];
  CgState* st;
  double* partials;
  unsigned int* counter;
  unsigned long long cond;
};

template <int W, int VY, bool B16, bool JAC>
struct TmaLayout {
  using RC = Rec<B16, JAC>;
  static constexpr int TY = W * VY;
  static constexpr int kVecBytes = (TY + 2) * kVecX * 16;
  static constexpr int kRecBytes = (TY + RC::kRows) * RC::kX * RC::kBytes;
  static constexpr int kDinvBytes = RC::kDinv ? (TY + 2) * kDinvX * 4 : 0;
  static constexpr int al(int b) { return (b + 127) / 128 * 128; }
  static constexpr int kV = 0;
  static constexpr int kC = al(kVecBytes);
  static constexpr int kD = kC + al(kRecBytes);
  static constexpr int kStage = kD + al(kDinvBytes);
  static constexpr uint32_t kTx = kVecBytes + kRecBytes + kDinvBytes;  // bytes per stage
};

template <int W, int VY, int S, bool B16, bool JAC>
constexpr int tma_smem_bytes() {
  return S * TmaLayout<W, VY, B16, JAC>::kStage + 2 * S * 8 + 128;  // + barriers, alignment
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void tma_3d(void* dst, const CUtensorMap* m, uint64_t* bar, int x, int y,
                                       int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

// staged record i as (Tx, Ty, Tz, w): w = D (FP32 records) or E (BF16 records)
template <bool B16>
__device__ __forceinline__ float4 srec(const unsigned char* base, int i) {
  if (B16) {
    const uint2 u = reinterpret_cast<const uint2*>(base)[i];
    return make_float4(bf16_lo(u.x), bf16_hi(u.x), bf16_lo(u.y), bf16_hi(u.y));
  }
  return reinterpret_cast<const float4*>(base)[i];
}

// BATCH: one launch sweeps every instance of a batch.  Blocks of an instance
// are contiguous; each block finds its instance in the table and uses that
// instance's grid, tiling, cell offset, tensor maps (in global memory), CG
// state, completion counter and range of partial sums.  The blocks of an
// instance that is not iterating return at once.
template <int W, int VY, int S, bool COND, bool B16, bool JAC, bool BATCH = false>
__global__ void __launch_bounds__((W + 1) * 32)
cg_sweep_tma_kernel(const __grid_constant__ TmaArgs a) {
  static_assert(!BATCH || (!COND && !B16), "batched sweeps: FP32 records, no graph condition");
  using LY = TmaLayout<W, VY, B16, JAC>;
  using RC = Rec<B16, JAC>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * LY::kStage);
  uint64_t* empty = full + S;

  CgState* st = a.st;
  Grid g = a.g;
  int nbx = a.nbx, nby = a.nby, zc = a.zc;
  int64_t lb = blockIdx.x, pstart = 0, pcount = gridDim.x, off = 0;
  unsigned int* counter = a.counter;
  const CUtensorMap *mv0 = &a.mv[0], *mv1 = &a.mv[1], *mc = &a.mc, *md = &a.md;
  if (BATCH) {
    int lo = 0, hi = a.ninst - 1;  // last instance whose first block <= blockIdx.x
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.inst[mid].bstart <= (int64_t)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    const TmaInst& I = a.inst[lo];
    g = I.g; nbx = I.nbx; nby = I.nby; zc = I.zc; off = I.off;
    lb = blockIdx.x - I.bstart; pstart = I.bstart; pcount = I.nblocks;
    st = a.st + lo;
    counter = a.counter + lo;
    mv0 = I.maps; mv1 = I.maps + 1; mc = I.maps + 2; md = I.maps + 3;
  }
  if (*(volatile int*)&st->done != kRunning) {
    if (lb == 0 && threadIdx.x == 0) {
      st->launches += 1;
      if (COND) cudaGraphSetConditional(a.cond, 0u);
    }
    return;
  }
  if (lb == 0 && threadIdx.x == 0) {
    const long long n = st->launches + 1;
    st->launches = n;
    if (COND && n > st->guard_limit) cudaGraphSetConditional(a.cond, 0u);
  }
  const int par = st->parity;
  const float alpha = (float)st->alpha;
  const float beta = (float)st->beta;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int bx = (int)(lb % nbx);
  const int t = (int)(lb / nbx);
  const int by = t % nby;
  const int bz = t / nby;
  const int X0 = 32 * bx, Y0 = LY::TY * by;
  const int64_t z0 = (int64_t)bz * zc;
  const int64_t z1 = min(z0 + (int64_t)zc, g.nz);
  const int L = (int)(z1 - z0) + 2;  // planes z0-1 .. z1

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], W);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  Acc acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  bool fault = false;

  if (warp == W) {
    // ---- producer: one thread issues the copies of every plane -----------
    if (lane == 0) {
      const CUtensorMap* mv = par ? mv1 : mv0;
      int issued = 0;
      for (int j = 0; j < L; ++j) {
        const int s = j % S;
        if (j >= S && !mbar_wait(&empty[s], ((j / S) - 1) & 1, kWaitLimit)) {
          fault = true;
          break;
        }
        const int z = (int)(z0 - 1 + j);
        unsigned char* sb = smem + s * LY::kStage;
        mbar_expect_tx(&full[s], LY::kTx);
        // x coordinates in 4-byte elements, all multiples of 4 (16 bytes)
        tma_3d(sb + LY::kV, mv, &full[s], 4 * (X0 - 1), Y0 - 1, z);
        tma_3d(sb + LY::kC, mc, &full[s], (RC::kBytes / 4) * (X0 - RC::kC0), Y0 - 1, z);
        if (RC::kDinv) tma_3d(sb + LY::kD, md, &full[s], X0 - 4, Y0 - 1, z);
        issued = j + 1;
      }
      // every issued copy must have landed before the block exits: wait for
      // the phases of the last (up to S) issued planes; phases the compute
      // warps already consumed have completed and pass at once
      for (int j = issued - 1; j >= 0 && j >= issued - S; --j)
        if (!mbar_wait(&full[j % S], (j / S) & 1, kWaitLimit)) fault = true;
    }
  } else {
    // ---- compute warps ----------------------------------------------------
    const int jw = warp * VY;           // first tile row of this warp
    const int gx = X0 + lane;
    const bool inx = gx < g.nx;
    unsigned rowok = 0u;  // bit jj: own row jj inside the grid (and this column too)
#pragma unroll
    for (int jj = 0; jj < VY; ++jj)
      if (inx && Y0 + jw + jj < g.ny) rowok |= 1u << jj;
    const int nxi = (int)g.nx;
    // in-plane offset of own row 0; own rows inside the grid stay below
    // nx * ny < 2^31 (checked at context creation)
    const unsigned o0 = (unsigned)(Y0 + jw) * (unsigned)nxi + (unsigned)gx;
    const int hc = lane == 0 ? 0 : 33;  // vector box column of this lane's x-halo cell
    float4* vout = a.v4[par ^ 1] + off;

    // M^-1 of the staged cell at box row r, column c + (X0 - 1) offset of the
    // vector box (Jacobi only)
    auto minv = [&](const unsigned char* sb, int r, int cv) -> float {
      if (RC::kDinv)
        return reinterpret_cast<const float*>(sb + LY::kD)[r * kDinvX + cv + 3];
      return jac_inv(srec<false>(sb + LY::kC, r * RC::kX + cv).w);
    };

    // Form r_k, p_k (and x_k on own rows) of plane j (absolute z = z0 - 1 + j)
    // for rows -1..VY of this lane's column, and p_k of the x-halo cell of the
    // own rows.  With Jacobi p_k = z_k + beta p_{k-1}, z_k = M^-1 r_k.
    auto form = [&](int j, float (&P)[VY + 2], float (&R)[VY], float (&Zd)[VY], float (&H)[VY],
                    float (&E)[VY], float& s0) {
      const unsigned char* sb = smem + (j % S) * LY::kStage;
      const float4* sv = reinterpret_cast<const float4*>(sb + LY::kV);
      const int64_t z = z0 - 1 + j;
      const bool own = z >= z0 && z < z1;
#pragma unroll
      for (int jj = -1; jj <= VY; ++jj) {
        const int r = jw + jj + 1;
        const float4 v = sv[r * kVecX + lane + 1];  // (r, q, p, x)
        const float r_ = fmaf(-alpha, v.y, v.x);      // Alg. 1 line 7 (previous iteration)
        float z_ = r_;
        if (JAC) z_ = r_ * minv(sb, r, lane + 1);     // z = M^-1 r
        const float p_ = fmaf(beta, v.z, z_);         // Alg. 1 line 10
        P[jj + 1] = p_;
        if (jj >= 0 && jj < VY) {
          R[jj] = r_;
          Zd[jj] = z_;
          E[jj] = fmaf(alpha, v.z, v.w);              // Alg. 1 line 6
          const float4 h = sv[r * kVecX + hc];
          float hz = fmaf(-alpha, h.y, h.x);
          if (JAC) hz = hz * minv(sb, r, hc);
          H[jj] = fmaf(beta, h.z, hz);
          if (own && ((rowok >> jj) & 1u)) s0 = fmaf(r_, z_, s0);
        }
      }
    };
    auto wait_full = [&](int j) -> bool {
      return mbar_wait(&full[j % S], (j / S) & 1, kWaitLimit);
    };
    auto release = [&](int j) {
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[j % S]);
    };

    float Pm[VY], P0[VY + 2], R0[VY], Z0[VY], H0[VY], E0[VY], Tzm[VY];
    float s0 = 0.f;
    if (!wait_full(0)) fault = true;
    if (!fault) {  // plane z0 - 1: direction below the first plane, and its Tz
      float Pt[VY + 2], Rt[VY], Zt[VY], Ht[VY], Et[VY];
      form(0, Pt, Rt, Zt, Ht, Et, s0);
#pragma unroll
      for (int jj = 0; jj < VY; ++jj) {
        Pm[jj] = Pt[jj + 1];
        Tzm[jj] = srec<B16>(smem + LY::kC, (jw + jj + 1) * RC::kX + lane + RC::kC0).z;
      }
      release(0);
      if (!wait_full(1)) fault = true;
    }
    if (!fault) form(1, P0, R0, Z0, H0, E0, s0);

    for (int64_t z = z0; z < z1 && !fault; ++z) {
      const int jc = (int)(z - z0) + 1;  // plane z
      const int jf = jc + 1;             // plane z + 1
      if (!wait_full(jf)) { fault = true; break; }
      float Pp[VY + 2], Rp[VY], Zp[VY], Hp[VY], Ep[VY];
      form(jf, Pp, Rp, Zp, Hp, Ep, s0);
      const unsigned char* sb = smem + (jc % S) * LY::kStage;
      float4* vz = vout + g.plane * z;
      float s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
      for (int jj = 0; jj < VY; ++jj) {
        const int r = jw + jj + 1;
        const int ri = r * RC::kX + lane + RC::kC0;
        float4 cf = srec<B16>(sb + LY::kC, ri);
        const float txm = srec<B16>(sb + LY::kC, ri - 1).x;
        const float tym = srec<B16>(sb + LY::kC, ri - RC::kX).y;
        // BF16 records: D = T(-x) + T(+x) + T(-y) + T(+y) + T(-z) + T(+z) + E
        if (B16) cf.w = (((((txm + cf.x) + tym) + cf.y) + Tzm[jj]) + cf.z) + cf.w;
        const float pc = P0[jj + 1];
        float pxm = __shfl_up_sync(kFull, pc, 1);
        float pxp = __shfl_down_sync(kFull, pc, 1);
        if (lane == 0) pxm = H0[jj];
        if (lane == 31) pxp = H0[jj];
        const float q = stencil7(cf, txm, tym, Tzm[jj], pc, pxp, pxm, P0[jj + 2], P0[jj],
                                 Pp[jj + 1], Pm[jj]);
        if ((rowok >> jj) & 1u) {
          vz[o0 + (unsigned)(jj * nxi)] = make_float4(R0[jj], q, pc, E0[jj]);
          s1 = fmaf(pc, q, s1);
          s2 = fmaf(Z0[jj], q, s2);
          if (JAC && B16) s3 = fmaf(q, q * minv(sb, r, lane + 1), s3);
          else if (JAC) s3 = fmaf(q, q * jac_inv(cf.w), s3);
          else s3 = fmaf(q, q, s3);
        }
        Tzm[jj] = cf.z;
        Pm[jj] = pc;
      }
      release(jc);  // plane z is no longer needed
      kadd(acc[0], s0);
      kadd(acc[1], s1);
      kadd(acc[2], s2);
      kadd(acc[3], s3);
      s0 = 0.f;
#pragma unroll
      for (int jj = 0; jj < VY; ++jj) {
        R0[jj] = Rp[jj];
        Z0[jj] = Zp[jj];
        H0[jj] = Hp[jj];
        E0[jj] = Ep[jj];
      }
#pragma unroll
      for (int jj = 0; jj < VY + 2; ++jj) P0[jj] = Pp[jj];
    }
    if (!fault) {
      kadd(acc[0], s0);
      release(L - 1);  // the last plane (z1) was only formed
    }
  }

  if (fault) st->fault = 1;  // the finishing block turns this into the guard status
  double v[4] = {kval(acc[0]), kval(acc[1]), kval(acc[2]), kval(acc[3])};
  block_partial<4>(v, a.partials);
  double tot[4];
  if (last_block_range<4>(a.partials, counter, pstart, pcount, tot) && threadIdx.x == 0)
    cg_finish(st, tot, a.cond, COND);
}

// ---------------------------------------------------------------------------
// Operator application q = A p with p'q (Eq. 6 / Alg. 2 in the positive form),
// TMA-staged: the CG sweep's tiling and pipeline with one FP32 field in place
// of the vector records.  Per plane the producer copies
//   p             [TY+2 rows][40 floats] from (X0-4, Y0-1) (a 16-byte aligned
//                 start; columns X0-1 and X0+32 are the x-halo),
//   coefficients  [TY+1 rows][33 records] from (X0-1, Y0-1)
//                 (BF16 records: 36 from X0-2).
// The per-cell arithmetic is that of the cp.async-staged operator of
// kernels_cg.cu (same operands, same fused multiply-adds in the same order),
// so both give bit-identical q; only the grouping of p'q differs.
constexpr int kPX = 40;  // p box width: X0-4 .. X0+35

// NE: further FP32 fields staged for the own cells only ([TY rows][32 floats]
// from (X0, Y0) per own plane), for the fused dot products
template <int W, int VY, bool B16, int NE = 0>
struct ApplyLayout {
  using RC = Rec<B16, false>;
  static constexpr int TY = W * VY;
  static constexpr int kPBytes = (TY + 2) * kPX * 4;
  static constexpr int kRecBytes = (TY + 1) * RC::kX * RC::kBytes;
  static constexpr int kOwnBytes = TY * 32 * 4;  // one own-cell field
  static constexpr int al(int b) { return (b + 127) / 128 * 128; }
  static constexpr int kP = 0;
  static constexpr int kC = al(kPBytes);
  static constexpr int kE = kC + al(kRecBytes);
  static constexpr int kStage = kE + NE * kOwnBytes;
  static constexpr uint32_t kTx = kPBytes + kRecBytes;  // bytes per stage (halo planes)
  static constexpr uint32_t kTxOwn = kTx + NE * kOwnBytes;  // own planes
};

template <int W, int VY, int S, bool B16, int NE = 0>
constexpr int apply_smem_bytes() {
  return S * ApplyLayout<W, VY, B16, NE>::kStage + 2 * S * 8 + 128;
}

struct ApplyArgs {
  CUtensorMap mp, mc;  // p, coefficient records
  // batched operator: instance table (all instances of the batch or a subset,
  // blocks numbered consecutively through it); an instance's maps are
  // {coefficients, input 0, input 1, ...} and `which` picks the input; only
  // instances with (act[id] & need) == need are applied, the others' cells are
  // left untouched
  const TmaInst* inst;
  int ninst, which;
  const int* act;
  int need;
  Grid g;
  int zc;
  int nbx, nby;
  float* Ap;
  double* pAp;  // one double (per instance when batched), or null
  double* partials;
  unsigned int* counter;
  // Flexible-CG dot products fused into the batched operator (DM >= 0 in the
  // kernel): with u the input, q = A u (not stored) and w = M^-1 r, per
  // instance u'q, u'r, q'w, w'q_j and u'q_j (j < DM) into
  // dots[id * kApplyDotsStride + ...], u'q also into pAp[id].  r, M^-1 and
  // the q_j are staged like p, own cells only, from the instance's maps
  // own0 (r), own0 + 1 (M^-1) and own0 + 2 + qmap[j].
  int own0;
  int qmap[kApplyMaxDirs];
  double* dots;
};

template <int W, int VY, int S, bool B16, bool BATCH, int DM = -1>
__global__ void __launch_bounds__((W + 1) * 32)
apply_tma_kernel(const __grid_constant__ ApplyArgs a) {
  static_assert(!BATCH || !B16, "batched operator: FP32 records");
  static_assert(DM < 0 || (BATCH && DM <= kApplyMaxDirs), "fused dots: batched, few directions");
  constexpr int NE = DM < 0 ? 0 : 2 + DM;       // own-cell fields: r, M^-1, q_j
  constexpr int NV = DM < 0 ? 1 : 3 + 2 * DM;   // reduced values
  using LY = ApplyLayout<W, VY, B16, NE>;
  using RC = Rec<B16, false>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * LY::kStage);
  uint64_t* empty = full + S;

  Grid g = a.g;
  int nbx = a.nbx, nby = a.nby, zc = a.zc;
  int64_t lb = blockIdx.x, pstart = 0, pcount = gridDim.x, off = 0;
  int inst = 0;
  unsigned int* counter = a.counter;
  const CUtensorMap *mp = &a.mp, *mc = &a.mc, *mown = nullptr;
  if (BATCH) {
    int lo = 0, hi = a.ninst - 1;  // last instance whose first block <= blockIdx.x
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.inst[mid].bstart <= (int64_t)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    const TmaInst& I = a.inst[lo];
    // the table may list a subset of the batch: I.id is the batch index
    if ((a.act[I.id] & a.need) != a.need) return;  // every block of the instance returns
    g = I.g; nbx = I.nbx; nby = I.nby; zc = I.zc; off = I.off;
    lb = blockIdx.x - I.bstart; pstart = I.bstart; pcount = I.nblocks;
    inst = I.id;
    counter = a.counter + I.id;
    mc = I.maps;
    mp = I.maps + 1 + a.which;
    mown = I.maps + a.own0;
  }

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int bx = (int)(lb % nbx);
  const int t = (int)(lb / nbx);
  const int by = t % nby;
  const int bz = t / nby;
  const int X0 = 32 * bx, Y0 = LY::TY * by;
  const int64_t z0 = (int64_t)bz * zc;
  const int64_t z1 = min(z0 + (int64_t)zc, g.nz);
  const int L = (int)(z1 - z0) + 2;  // planes z0-1 .. z1

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], W);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  Acc acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = {0.f, 0.f};
  bool fault = false;

  if (warp == W) {
    // ---- producer ---------------------------------------------------------
    if (lane == 0) {
      int issued = 0;
      for (int j = 0; j < L; ++j) {
        const int s = j % S;
        if (j >= S && !mbar_wait(&empty[s], ((j / S) - 1) & 1, kWaitLimit)) {
          fault = true;
          break;
        }
        const int z = (int)(z0 - 1 + j);
        const bool own = NE > 0 && j >= 1 && j <= L - 2;
        unsigned char* sb = smem + s * LY::kStage;
        mbar_expect_tx(&full[s], own ? LY::kTxOwn : LY::kTx);
        // x coordinates in 4-byte elements, multiples of 4 (16 bytes)
        tma_3d(sb + LY::kP, mp, &full[s], X0 - 4, Y0 - 1, z);
        tma_3d(sb + LY::kC, mc, &full[s], (RC::kBytes / 4) * (X0 - RC::kC0), Y0 - 1, z);
        if (own) {
          tma_3d(sb + LY::kE, mown, &full[s], X0, Y0, z);                        // r
          tma_3d(sb + LY::kE + LY::kOwnBytes, mown + 1, &full[s], X0, Y0, z);    // M^-1
#pragma unroll
          for (int q = 0; q < (DM > 0 ? DM : 0); ++q)
            tma_3d(sb + LY::kE + (2 + q) * LY::kOwnBytes, mown + 2 + a.qmap[q], &full[s], X0, Y0,
                   z);
        }
        issued = j + 1;
      }
      // every issued copy lands before the block exits
      for (int j = issued - 1; j >= 0 && j >= issued - S; --j)
        if (!mbar_wait(&full[j % S], (j / S) & 1, kWaitLimit)) fault = true;
    }
  } else {
    // ---- compute warps ----------------------------------------------------
    const int jw = warp * VY;
    const int gx = X0 + lane;
    const bool inx = gx < g.nx;
    unsigned rowok = 0u;
#pragma unroll
    for (int jj = 0; jj < VY; ++jj)
      if (inx && Y0 + jw + jj < g.ny) rowok |= 1u << jj;
    const int nxi = (int)g.nx;
    const unsigned o0 = (unsigned)(Y0 + jw) * (unsigned)nxi + (unsigned)gx;
    const int hc = lane == 0 ? 3 : 36;  // p box column of this lane's x-halo cell
    float* out = a.Ap + off;

    // p of plane j for rows -1..VY of this lane's column, and of the x-halo
    // cell of the own rows
    auto load = [&](int j, float (&P)[VY + 2], float (&H)[VY]) {
      const float* sp = reinterpret_cast<const float*>(smem + (j % S) * LY::kStage + LY::kP);
#pragma unroll
      for (int jj = -1; jj <= VY; ++jj) {
        const int r = jw + jj + 1;
        P[jj + 1] = sp[r * kPX + lane + 4];
        if (jj >= 0 && jj < VY) H[jj] = sp[r * kPX + hc];
      }
    };
    auto wait_full = [&](int j) -> bool {
      return mbar_wait(&full[j % S], (j / S) & 1, kWaitLimit);
    };
    auto release = [&](int j) {
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[j % S]);
    };

    float Pm[VY], P0[VY + 2], H0[VY], Tzm[VY];
    int64_t zdone = z0;  // first plane of the run not yet written
    if (!wait_full(0)) fault = true;
    if (!fault) {  // plane z0 - 1: p below the first plane, and its Tz
      float Pt[VY + 2], Ht[VY];
      load(0, Pt, Ht);
#pragma unroll
      for (int jj = 0; jj < VY; ++jj) {
        Pm[jj] = Pt[jj + 1];
        Tzm[jj] = srec<B16>(smem + LY::kC, (jw + jj + 1) * RC::kX + lane + RC::kC0).z;
      }
      release(0);
      if (!wait_full(1)) fault = true;
    }
    if (!fault) load(1, P0, H0);

    for (int64_t z = z0; z < z1 && !fault; ++z) {
      const int jc = (int)(z - z0) + 1;  // plane z
      const int jf = jc + 1;             // plane z + 1
      if (!wait_full(jf)) { fault = true; break; }
      float Pp[VY + 2], Hp[VY];
      load(jf, Pp, Hp);
      const unsigned char* sb = smem + (jc % S) * LY::kStage;
      float* oz = out + g.plane * z;
      float s1 = 0.f;
      float sd[NV];
#pragma unroll
      for (int k = 0; k < NV; ++k) sd[k] = 0.f;
#pragma unroll
      for (int jj = 0; jj < VY; ++jj) {
        const int ri = (jw + jj + 1) * RC::kX + lane + RC::kC0;
        float4 cf = srec<B16>(sb + LY::kC, ri);
        const float txm = srec<B16>(sb + LY::kC, ri - 1).x;
        const float tym = srec<B16>(sb + LY::kC, ri - RC::kX).y;
        // BF16 records: D = T(-x) + T(+x) + T(-y) + T(+y) + T(-z) + T(+z) + E
        if (B16) cf.w = (((((txm + cf.x) + tym) + cf.y) + Tzm[jj]) + cf.z) + cf.w;
        const float pc = P0[jj + 1];
        float pxm = __shfl_up_sync(kFull, pc, 1);
        float pxp = __shfl_down_sync(kFull, pc, 1);
        if (lane == 0) pxm = H0[jj];
        if (lane == 31) pxp = H0[jj];
        const float q = stencil7(cf, txm, tym, Tzm[jj], pc, pxp, pxm, P0[jj + 2], P0[jj],
                                 Pp[jj + 1], Pm[jj]);
        if ((rowok >> jj) & 1u) {
          if constexpr (DM < 0) {
            oz[o0 + (unsigned)(jj * nxi)] = q;
            s1 = fmaf(pc, q, s1);
          } else {
            // the dot products of the flexible-CG step at this cell (u = pc)
            const float* se = reinterpret_cast<const float*>(sb + LY::kE) + (jw + jj) * 32 + lane;
            const float rv = se[0];
            const float wv = rv * se[LY::kOwnBytes / 4];
            sd[0] = fmaf(pc, q, sd[0]);
            sd[1] = fmaf(pc, rv, sd[1]);
            sd[2] = fmaf(q, wv, sd[2]);
#pragma unroll
            for (int k = 0; k < (DM > 0 ? DM : 0); ++k) {
              const float qv = se[(2 + k) * (LY::kOwnBytes / 4)];
              sd[3 + k] = fmaf(wv, qv, sd[3 + k]);
              sd[3 + DM + k] = fmaf(pc, qv, sd[3 + DM + k]);
            }
          }
        }
        Tzm[jj] = cf.z;
        Pm[jj] = pc;
      }
      release(jc);
      if constexpr (DM < 0) {
        kadd(acc[0], s1);
      } else {
#pragma unroll
        for (int k = 0; k < NV; ++k) kadd(acc[k], sd[k]);
      }
      zdone = z + 1;
#pragma unroll
      for (int jj = 0; jj < VY; ++jj) H0[jj] = Hp[jj];
#pragma unroll
      for (int jj = 0; jj < VY + 2; ++jj) P0[jj] = Pp[jj];
    }
    if (!fault) {
      release(L - 1);  // the last plane (z1) was only read
    } else {
      // a copy that never landed: the cells this warp did not write become
      // NaN, and so do the dot products, so that the failure cannot pass
      // unnoticed
      const float qnan = __int_as_float(0x7fc00000);
      if (DM < 0)
        for (int64_t z = zdone; z < z1; ++z)
#pragma unroll
          for (int jj = 0; jj < VY; ++jj)
            if ((rowok >> jj) & 1u) out[g.plane * z + o0 + (unsigned)(jj * nxi)] = qnan;
#pragma unroll
      for (int k = 0; k < NV; ++k) kadd(acc[k], qnan);
    }
  }

  if (a.pAp != nullptr) {
    double v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = kval(acc[k]);
    block_partial<NV>(v, a.partials);
    double tot[NV];
    if (last_block_range<NV>(a.partials, counter, pstart, pcount, tot) && threadIdx.x == 0) {
      a.pAp[inst] = tot[0];
      if constexpr (DM >= 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) a.dots[(size_t)inst * kApplyDotsStride + k] = tot[k];
      }
    }
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// 16-byte records [nz][ny][nx][4 floats] as a 3-D FP32 tensor of rows of
// 4 nx floats, box (4 bw, bh, 1): one box row is one contiguous request of
// 16 bw bytes (a 4-D view with the record as the innermost dimension would
// make the copy engine issue one 16-byte request per record)
bool encode_rec(CUtensorMap* m, const float4* base, const Grid& g, int bw, int bh) {
  EncodeTiledFn fn = encode_fn();
  if (fn == nullptr) return false;
  const cuuint64_t dim[3] = {4 * (cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
  const cuuint64_t stride[2] = {(cuuint64_t)g.nx * 16, (cuuint64_t)g.plane * 16};
  const cuuint32_t box[3] = {4 * (cuuint32_t)bw, (cuuint32_t)bh, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float4*>(base), dim, stride, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// FP32 field [nz][ny][nx] as a 3-D tensor, box (bw, bh, 1) (needs nx % 4 == 0)
bool encode_f32(CUtensorMap* m, const float* base, const Grid& g, int bw, int bh) {
  EncodeTiledFn fn = encode_fn();
  if (fn == nullptr) return false;
  const cuuint64_t dim[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
  const cuuint64_t stride[2] = {(cuuint64_t)g.nx * 4, (cuuint64_t)g.plane * 4};
  const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dim, stride, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 8-byte BF16 records [nz][ny][nx][4 x bf16] as a 3-D tensor of 32-bit words,
// rows of 2 nx words, box (2 bw, bh, 1) (needs nx % 2 == 0)
bool encode_rec16(CUtensorMap* m, const uint2* base, const Grid& g, int bw, int bh) {
  EncodeTiledFn fn = encode_fn();
  if (fn == nullptr) return false;
  const cuuint64_t dim[3] = {2 * (cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
  const cuuint64_t stride[2] = {(cuuint64_t)g.nx * 8, (cuuint64_t)g.plane * 8};
  const cuuint32_t box[3] = {2 * (cuuint32_t)bw, (cuuint32_t)bh, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, const_cast<uint2*>(base), dim, stride, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int W, int VY, int S, bool COND, bool B16, bool JAC>
cudaError_t launch_tma_t(const TmaArgs& a, int64_t nblocks, cudaStream_t s) {
  constexpr int smem = tma_smem_bytes<W, VY, S, B16, JAC>();
  auto fn = cg_sweep_tma_kernel<W, VY, S, COND, B16, JAC>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  fn<<<(unsigned)nblocks, (W + 1) * 32, smem, s>>>(a);
  return cudaGetLastError();
}

template <int W, int VY, int S, bool B16, bool JAC>
int tma_blocks_per_sm_t() {
  constexpr int smem = tma_smem_bytes<W, VY, S, B16, JAC>();
  auto fn = cg_sweep_tma_kernel<W, VY, S, true, B16, JAC>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, (W + 1) * 32, smem) != cudaSuccess)
    return 0;
  return nb;
}

template <bool B16>
int apply_blocks_per_sm_t() {
  constexpr int smem = apply_smem_bytes<4, 4, 4, B16>();
  auto fn = apply_tma_kernel<4, 4, 4, B16, false>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, 5 * 32, smem) != cudaSuccess)
    return 0;
  return nb;
}

// stages of the operator's ring: 4; 3 with the fused dot products, whose
// stages also hold the own-cell boxes (three blocks per SM instead of two)
template <int DM>
constexpr int apply_stages() {
  return DM < 0 ? 4 : 3;
}

int apply_dots_blocks_per_sm_t() {
  constexpr int smem = apply_smem_bytes<4, 4, apply_stages<2>(), false, 4>();
  auto fn = apply_tma_kernel<4, 4, apply_stages<2>(), false, true, 2>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, 5 * 32, smem) != cudaSuccess)
    return 0;
  return nb;
}

template <bool B16, bool BATCH, int DM = -1>
cudaError_t launch_apply_t(const ApplyArgs& a, int64_t nblocks, cudaStream_t s) {
  constexpr int S = apply_stages<DM>();
  constexpr int smem = apply_smem_bytes<4, 4, S, B16, DM < 0 ? 0 : 2 + DM>();
  auto fn = apply_tma_kernel<4, 4, S, B16, BATCH, DM>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  fn<<<(unsigned)nblocks, 5 * 32, smem, s>>>(a);
  return cudaGetLastError();
}

// (W, VY, S) of each tile choice; the Jacobi and BF16 variants use tile 0
struct TileShape {
  int w, vy, s;
};
constexpr TileShape kTmaTiles[] = {{4, 4, 4}, {4, 4, 3}, {8, 4, 3}, {4, 2, 6}};
constexpr int kNumTmaTiles = (int)(sizeof(kTmaTiles) / sizeof(kTmaTiles[0]));

template <int W, int VY, int S, bool JAC>
cudaError_t launch_tma_batch_t(const TmaArgs& a, int64_t nblocks, cudaStream_t s) {
  constexpr int smem = tma_smem_bytes<W, VY, S, false, JAC>();
  auto fn = cg_sweep_tma_kernel<W, VY, S, false, false, JAC, true>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  fn<<<(unsigned)nblocks, (W + 1) * 32, smem, s>>>(a);
  return cudaGetLastError();
}

template <bool COND>
cudaError_t launch_variant(const TmaArgs& a, const TmaPlan& p, cudaStream_t s) {
  if (p.b16 && p.jac) return launch_tma_t<4, 4, 4, COND, true, true>(a, p.nblocks, s);
  if (p.b16) return launch_tma_t<4, 4, 4, COND, true, false>(a, p.nblocks, s);
  if (p.jac) return launch_tma_t<4, 4, 4, COND, false, true>(a, p.nblocks, s);
  switch (p.tile) {
    case 0: return launch_tma_t<4, 4, 4, COND, false, false>(a, p.nblocks, s);
    case 1: return launch_tma_t<4, 4, 3, COND, false, false>(a, p.nblocks, s);
    case 2: return launch_tma_t<8, 4, 3, COND, false, false>(a, p.nblocks, s);
    case 3: return launch_tma_t<4, 2, 6, COND, false, false>(a, p.nblocks, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool tma_sweep_ok(const Grid& g, bool b16, bool jac) {
  if (g.nx >= (1 << 30) || g.ny >= (1 << 30) || g.nz >= (1 << 30) || encode_fn() == nullptr)
    return false;
  if (b16 && g.nx % 2 != 0) return false;         // 8-byte records: 16-byte row strides
  if (b16 && jac && g.nx % 4 != 0) return false;  // the FP32 M^-1 array: likewise
  return true;
}

int tma_tile_count() { return kNumTmaTiles; }

TmaPlan plan_tma(const Grid& g, int tile, int zc_opt, int num_sms, bool b16, bool jac,
                 bool apply, bool dots) {
  TmaPlan p{};
  if (tile < 0 || tile >= kNumTmaTiles || b16 || jac || apply) tile = 0;
  if (apply) jac = false;
  p.dots = apply && dots && !b16;
  const TileShape ts = kTmaTiles[tile];
  p.tile = tile;
  p.b16 = b16;
  p.jac = jac;
  p.apply = apply;
  p.w = ts.w;
  p.vy = ts.vy;
  p.stages = ts.s;
  p.nbx = (g.nx + 31) / 32;
  p.nby = (g.ny + ts.w * ts.vy - 1) / (ts.w * ts.vy);
  int zc = zc_opt;
  if (zc <= 0) {
    // Measured on GB300 (plain FP32 sweep, 128^3 ... 1024x1024x256): every run
    // costs more than its two halo planes (pipeline fill at its start), so long
    // runs win, and a partial second wave of blocks costs more than a partly
    // idle first one.  Hence: 128-plane runs when they give at least one full
    // wave of resident blocks; otherwise as many runs per column as still fit
    // one wave (e.g. 256^3: 128-plane runs, 256 blocks, 0.133 ms per sweep
    // against 0.145 ms with the 512 blocks of 64-plane runs; 128^3: 15-plane
    // runs, 288 blocks, 0.029 ms against 0.039 ms with 8-plane runs).
    const int64_t cols = p.nbx * p.nby;
    int per_sm = tma_blocks_per_sm(p);
    if (per_sm < 1) per_sm = 1;
    const int64_t slots = (int64_t)num_sms * per_sm;
    const int64_t nz = g.nz;
    if (cols * ((nz + 127) / 128) >= slots) {
      zc = 128;
    } else {
      const int64_t k = slots / cols;  // runs per column (>= 1 here)
      int64_t z = (nz + k - 1) / k;
      const int64_t zmin = nz < 8 ? nz : 8;
      if (z < zmin) z = zmin;
      if (z > 128) z = 128;
      zc = (int)z;
    }
  }
  if (zc > g.nz) zc = (int)g.nz;
  p.zc = zc;
  p.nbz = (g.nz + zc - 1) / zc;
  p.nblocks = p.nbx * p.nby * p.nbz;
  return p;
}

int tma_blocks_per_sm(const TmaPlan& p) {
  // host-side occupancy queries cost microseconds; the answer is fixed per
  // device and kernel, so it is kept (index: device, kernel variant)
  constexpr int kDevs = 64, kVariants = 3 + kNumTmaTiles + 3;
  static int memo[kDevs][kVariants] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    dev = -1;
  }
  const int var = p.dots ? 3 + kNumTmaTiles + 2
                  : p.apply ? 3 + kNumTmaTiles + (p.b16 ? 1 : 0)
                  : (p.b16 && p.jac) ? 0 : p.b16 ? 1 : p.jac ? 2 : 3 + p.tile;
  if (dev >= 0 && dev < kDevs && var >= 0 && var < kVariants && memo[dev][var] > 0)
    return memo[dev][var];
  int nb = 0;
  if (p.dots) nb = apply_dots_blocks_per_sm_t();
  else if (p.apply) nb = p.b16 ? apply_blocks_per_sm_t<true>() : apply_blocks_per_sm_t<false>();
  else if (p.b16 && p.jac) nb = tma_blocks_per_sm_t<4, 4, 4, true, true>();
  else if (p.b16) nb = tma_blocks_per_sm_t<4, 4, 4, true, false>();
  else if (p.jac) nb = tma_blocks_per_sm_t<4, 4, 4, false, true>();
  else {
    switch (p.tile) {
      case 0: nb = tma_blocks_per_sm_t<4, 4, 4, false, false>(); break;
      case 1: nb = tma_blocks_per_sm_t<4, 4, 3, false, false>(); break;
      case 2: nb = tma_blocks_per_sm_t<8, 4, 3, false, false>(); break;
      case 3: nb = tma_blocks_per_sm_t<4, 2, 6, false, false>(); break;
      default: break;
    }
  }
  if (nb == 0) cudaGetLastError();
  else if (dev >= 0 && dev < kDevs && var >= 0 && var < kVariants) memo[dev][var] = nb;
  return nb;
}

bool make_tma_maps(const Grid& g, const TmaPlan& p, const void* coef, const float* dinv,
                   const CgVecs& v, TmaMaps* m) {
  const int ty = p.w * p.vy;
  if (v.v4[0] == nullptr || v.v4[1] == nullptr) return false;
  bool ok = true;
  for (int i = 0; i < 2; ++i) ok = ok && encode_rec(&m->v[i], v.v4[i], g, kVecX, ty + 2);
  if (p.b16 && p.jac) {
    using RC = Rec<true, true>;
    ok = ok && dinv != nullptr;
    ok = ok && encode_rec16(&m->c, static_cast<const uint2*>(coef), g, RC::kX, ty + RC::kRows);
    ok = ok && encode_f32(&m->d, dinv, g, kDinvX, ty + 2);
  } else if (p.b16) {
    using RC = Rec<true, false>;
    ok = ok && encode_rec16(&m->c, static_cast<const uint2*>(coef), g, RC::kX, ty + RC::kRows);
  } else if (p.jac) {
    using RC = Rec<false, true>;
    ok = ok && encode_rec(&m->c, static_cast<const float4*>(coef), g, RC::kX, ty + RC::kRows);
  } else {
    using RC = Rec<false, false>;
    ok = ok && encode_rec(&m->c, static_cast<const float4*>(coef), g, RC::kX, ty + RC::kRows);
  }
  return ok;
}

cudaError_t launch_cg_sweep_tma(const Grid& g, const TmaPlan& p, const TmaMaps& m, CgVecs v,
                                CgState* st, double* partials, unsigned int* counter,
                                unsigned long long cond, int use_cond, cudaStream_t s) {
  TmaArgs a;
  memset(&a, 0, sizeof(a));
  for (int i = 0; i < 2; ++i) {
    a.mv[i] = m.v[i];
    a.v4[i] = v.v4[i];
  }
  a.mc = m.c;
  a.md = m.d;
  a.g = g;
  a.zc = p.zc;
  a.nbx = (int)p.nbx;
  a.nby = (int)p.nby;
  a.st = st;
  a.partials = partials;
  a.counter = counter;
  a.cond = cond;
  return use_cond != 0 ? launch_variant<true>(a, p, s) : launch_variant<false>(a, p, s);
}

bool tma_apply_ok(const Grid& g, bool b16) {
  return tma_sweep_ok(g, b16, false) && g.nx % 4 == 0;  // FP32 rows of p: 16-byte strides
}

bool make_apply_maps(const Grid& g, const TmaPlan& p, const void* coef, const float* const* in,
                     int nin, CUtensorMap* out) {
  const int ty = p.w * p.vy;
  bool ok;
  if (p.b16)
    ok = encode_rec16(&out[0], static_cast<const uint2*>(coef), g, Rec<true, false>::kX, ty + 1);
  else
    ok = encode_rec(&out[0], static_cast<const float4*>(coef), g, Rec<false, false>::kX, ty + 1);
  for (int i = 0; i < nin && ok; ++i) ok = encode_f32(&out[1 + i], in[i], g, kPX, ty + 2);
  return ok;
}

cudaError_t launch_apply_tma(const Grid& g, const TmaPlan& p, const void* coef, const float* pin,
                             float* Ap, double* pAp, double* partials, unsigned int* counter,
                             cudaStream_t s) {
  ApplyArgs a;
  memset(&a, 0, sizeof(a));
  CUtensorMap m[2];
  if (!make_apply_maps(g, p, coef, &pin, 1, m)) return cudaErrorInvalidValue;
  a.mc = m[0];
  a.mp = m[1];
  a.g = g;
  a.zc = p.zc;
  a.nbx = (int)p.nbx;
  a.nby = (int)p.nby;
  a.Ap = Ap;
  a.pAp = pAp;
  a.partials = partials;
  a.counter = counter;
  return p.b16 ? launch_apply_t<true, false>(a, p.nblocks, s)
               : launch_apply_t<false, false>(a, p.nblocks, s);
}

cudaError_t launch_apply_tma_batch(const TmaInst* inst, int ninst, int64_t nblocks, int which,
                                   float* Ap, double* pAp, const int* act, int need,
                                   double* partials, unsigned int* counters, cudaStream_t s) {
  ApplyArgs a;
  memset(&a, 0, sizeof(a));
  a.inst = inst;
  a.ninst = ninst;
  a.which = which;
  a.act = act;
  a.need = need;
  a.Ap = Ap;
  a.pAp = pAp;
  a.partials = partials;
  a.counter = counters;
  return launch_apply_t<false, true>(a, nblocks, s);
}

bool make_own_maps(const Grid& g, const TmaPlan& p, const float* const* in, int nin,
                   CUtensorMap* out) {
  bool ok = true;
  for (int i = 0; i < nin && ok; ++i) ok = encode_f32(&out[i], in[i], g, 32, p.w * p.vy);
  return ok;
}

cudaError_t launch_apply_dots_tma_batch(const TmaInst* inst, int ninst, int64_t nblocks,
                                        int which, const int* act, int need, int own0,
                                        const int* qmap, int ndirs, double* uq, double* dots,
                                        double* partials, unsigned int* counters,
                                        cudaStream_t s) {
  if (ndirs < 0 || ndirs > kApplyMaxDirs) return cudaErrorInvalidValue;
  ApplyArgs a;
  memset(&a, 0, sizeof(a));
  a.inst = inst;
  a.ninst = ninst;
  a.which = which;
  a.act = act;
  a.need = need;
  a.pAp = uq;
  a.partials = partials;
  a.counter = counters;
  a.own0 = own0;
  for (int j = 0; j < ndirs; ++j) a.qmap[j] = qmap[j];
  a.dots = dots;
  switch (ndirs) {
    case 0: return launch_apply_t<false, true, 0>(a, nblocks, s);
    case 1: return launch_apply_t<false, true, 1>(a, nblocks, s);
    case 2: return launch_apply_t<false, true, 2>(a, nblocks, s);
    case 3: return launch_apply_t<false, true, 3>(a, nblocks, s);
    case 4: return launch_apply_t<false, true, 4>(a, nblocks, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_cg_sweep_tma_batch(const TmaInst* inst, int ninst, int64_t nblocks, int tile,
                                      bool jac, CgVecs v, CgState* st, double* partials,
                                      unsigned int* counters, cudaStream_t s) {
  TmaArgs a;
  memset(&a, 0, sizeof(a));
  a.inst = inst;
  a.ninst = ninst;
  a.v4[0] = v.v4[0];
  a.v4[1] = v.v4[1];
  a.st = st;
  a.partials = partials;
  a.counter = counters;
  if (jac) return launch_tma_batch_t<4, 4, 4, true>(a, nblocks, s);
  switch (tile) {
    case 0: return launch_tma_batch_t<4, 4, 4, false>(a, nblocks, s);
    case 1: return launch_tma_batch_t<4, 4, 3, false>(a, nblocks, s);
    case 2: return launch_tma_batch_t<8, 4, 3, false>(a, nblocks, s);
    case 3: return launch_tma_batch_t<4, 2, 6, false>(a, nblocks, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tpfa
