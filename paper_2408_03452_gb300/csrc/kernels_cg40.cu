// Fused CG iteration that recomputes q_{k-1} = A p_{k-1} instead of storing q.
//
// CG (Alg. 1 of arXiv 2408.03452) carries x, r, p and the product q = A p.
// The previous sweep stored p_{k-1}; applying the operator to it again
// (the same fused multiply-adds on the same values, so the result is
// bit-identical to the q_{k-1} that sweep computed) costs arithmetic but no
// DRAM traffic, so this sweep reads r_{k-1}, p_{k-1}, x and the coefficient
// record and writes r_k, p_k, x_k: 40 bytes per cell instead of 48.
//
// Per warp: 32 x-lanes (lanes 2..29 produce output, lanes 0, 1, 30, 31 are a
// two-cell halo), 4 output rows, a run of z-planes.  p_{k-1} is staged for
// rows -2..5, r_{k-1} and the records for rows -1..4, so that q_{k-1}, r_k
// and p_k are formed on rows -1..4 and lanes 1..30, which is the support of
// q_k on the output cells.  Planes are staged through a per-warp cp.async
// ring of S planes: three are read in each step (z, z+1, z+2 of p_{k-1})
// and S-3 are in flight.
#include "sweep_common.cuh"

namespace tpfa {

namespace {

constexpr int kVY40 = 4;     // output rows per warp
constexpr int kTileX40 = 28; // output columns per warp (lanes 2..29)

struct Cg40Args {
  Grid g;
  int64_t nwx, nwy, nwarps;
  int zc;
  const float4* coef;
  CgVecs v;
  CgState* st;
  double* partials;
  unsigned int* counter;
  unsigned long long cond;
};

// One staged plane of one warp, lane-minor (each lane reads its own column):
//   records rows -1..VY (float4), p_{k-1} rows -2..VY+1, r_{k-1} rows -1..VY,
//   x rows 0..VY-1, Ty of row -2.
struct Stage40 {
  static constexpr int kCoef = 0;
  static constexpr int kP = kCoef + (kVY40 + 2) * 32 * 16;
  static constexpr int kR = kP + (kVY40 + 4) * 32 * 4;
  static constexpr int kE = kR + (kVY40 + 2) * 32 * 4;
  static constexpr int kTy2 = kE + kVY40 * 32 * 4;
  static constexpr int kBytes = kTy2 + 32 * 4;
};

template <int S, int W>
constexpr int cg40_smem_bytes() { return W * S * Stage40::kBytes; }

template <int S, int W, bool COND>
__global__ void __launch_bounds__(W * 32)
cg40_kernel(const Cg40Args a) {
  static_assert(S >= 4, "three staged planes are read per step");
  constexpr int VY = kVY40;
  using LY = Stage40;
  extern __shared__ __align__(16) unsigned char smem[];
  const Grid& g = a.g;
  CgState* st = a.st;
  if (*(volatile int*)&st->done != kRunning) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st->launches += 1;
      if (COND) cudaGraphSetConditional(a.cond, 0u);
    }
    return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const long long n = st->launches + 1;
    st->launches = n;
    if (COND && n > st->guard_limit) cudaGraphSetConditional(a.cond, 0u);
  }
  const int par = st->parity;
  const float alpha = (float)st->alpha;
  const float beta = (float)st->beta;
  const float* rin = a.v.r[par];
  const float* pin = a.v.p[par];
  float* rout = a.v.r[par ^ 1];
  float* pout = a.v.p[par ^ 1];
  float* xe = a.v.e;

  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * W + wib;
  unsigned char* wsm = smem + (size_t)wib * S * LY::kBytes;
  Acc acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};

  if (gw < a.nwarps) {  // warp-uniform
    const int64_t wx = gw % a.nwx;
    const int64_t t = gw / a.nwx;
    const int64_t wy = t % a.nwy;
    const int64_t wz = t / a.nwy;
    const int64_t gx = wx * kTileX40 - 2 + lane;
    const bool inx = gx >= 0 && gx < g.nx;
    const bool outl = inx && lane >= 2 && lane <= kTileX40 + 1;
    const int64_t y0 = wy * VY;
    const int64_t z0 = wz * (int64_t)a.zc;
    const int64_t z1 = min(z0 + (int64_t)a.zc, g.nz);
    unsigned rowok = 0u;  // bit jj+2: row y0+jj (jj = -2..VY+1) inside the grid, this column too
#pragma unroll
    for (int jj = -2; jj <= VY + 1; ++jj)
      if (inx && y0 + jj >= 0 && y0 + jj < g.ny) rowok |= 1u << (jj + 2);
    const int nxi = (int)g.nx;
    const int o0 = (int)(gx + g.nx * y0);  // < 2^31: checked at context creation
    const int64_t L = z1 - z0 + 4;         // planes z0-2 .. z1+1

    auto stage = [&](int64_t j) { return wsm + (size_t)(j % S) * LY::kBytes; };

    auto issue = [&](int64_t j) {
      if (j < L) {
        const int64_t z = z0 - 2 + j;
        const bool zok = z >= 0 && z < g.nz;
        const int64_t zo = g.plane * (z < 0 ? 0 : (z >= g.nz ? g.nz - 1 : z));
        const bool own = outl && z >= z0 && z < z1;
        unsigned char* sb = stage(j);
        float4* scf = reinterpret_cast<float4*>(sb + LY::kCoef);
        float* sp = reinterpret_cast<float*>(sb + LY::kP);
        float* sr = reinterpret_cast<float*>(sb + LY::kR);
        float* se = reinterpret_cast<float*>(sb + LY::kE);
        float* sty = reinterpret_cast<float*>(sb + LY::kTy2);
#pragma unroll
        for (int jj = -2; jj <= VY + 1; ++jj) {
          const bool ok = zok && ((rowok >> (jj + 2)) & 1u);
          const int64_t src = zo + (ok ? (int64_t)(o0 + jj * nxi) : 0);
          cp4(sp + (jj + 2) * 32 + lane, pin + src, ok);
          if (jj == -2) cp4(sty + lane, reinterpret_cast<const float*>(a.coef + src) + 1, ok);
          if (jj >= -1 && jj <= VY) {
            cp4(sr + (jj + 1) * 32 + lane, rin + src, ok);
            cp16(scf + (jj + 1) * 32 + lane, a.coef + src, ok);
          }
          if (jj >= 0 && jj < VY) cp4(se + jj * 32 + lane, xe + src, ok && own);
        }
      }
      cp_commit();
    };

    // q_{k-1}, r_k = r_{k-1} - alpha q_{k-1} (Alg. 1 line 7 of the previous
    // iteration) and p_k = r_k + beta p_{k-1} (line 10) on plane j, rows
    // -1..VY.  On this warp's own output cells also x_k = x_{k-1} + alpha
    // p_{k-1} (line 6), store r_k, p_k and accumulate r_k'r_k.
    auto form = [&](int64_t j, float (&P)[VY + 2], float (&R)[VY], float& s0) {
      const int64_t z = z0 - 2 + j;
      const bool own = outl && z >= z0 && z < z1;
      const unsigned char* bm = stage(j - 1);
      const unsigned char* b0 = stage(j);
      const unsigned char* bp = stage(j + 1);
      const float4* cf0 = reinterpret_cast<const float4*>(b0 + LY::kCoef);
      const float4* cfm = reinterpret_cast<const float4*>(bm + LY::kCoef);
      const float* p0 = reinterpret_cast<const float*>(b0 + LY::kP);
      const float* pm = reinterpret_cast<const float*>(bm + LY::kP);
      const float* pp = reinterpret_cast<const float*>(bp + LY::kP);
      const float* r0 = reinterpret_cast<const float*>(b0 + LY::kR);
      const float* e0 = reinterpret_cast<const float*>(b0 + LY::kE);
      const float* ty2 = reinterpret_cast<const float*>(b0 + LY::kTy2);
      const int64_t zo = g.plane * z;
      float tyl = ty2[lane];
#pragma unroll
      for (int jj = -1; jj <= VY; ++jj) {
        const float4 c = cf0[(jj + 1) * 32 + lane];
        const float pc = p0[(jj + 2) * 32 + lane];
        const float pxm = __shfl_up_sync(kFull, pc, 1);
        const float pxp = __shfl_down_sync(kFull, pc, 1);
        const float txm = __shfl_up_sync(kFull, c.x, 1);
        const float q1 = stencil7(c, txm, tyl, cfm[(jj + 1) * 32 + lane].z, pc, pxp, pxm,
                                  p0[(jj + 3) * 32 + lane], p0[(jj + 1) * 32 + lane],
                                  pp[(jj + 2) * 32 + lane], pm[(jj + 2) * 32 + lane]);
        const float r_ = fmaf(-alpha, q1, r0[(jj + 1) * 32 + lane]);
        const float p_ = fmaf(beta, pc, r_);
        if (jj >= 0 && jj < VY) {
          R[jj] = r_;
          if (own && ((rowok >> (jj + 2)) & 1u)) {
            const int64_t id = zo + o0 + jj * nxi;
            xe[id] = fmaf(alpha, pc, e0[jj * 32 + lane]);
            rout[id] = r_;
            pout[id] = p_;
            s0 = fmaf(r_, r_, s0);
          }
        }
        P[jj + 1] = p_;
        tyl = c.y;
      }
    };

    float PkM[VY], Pk0[VY + 2], Rk0[VY], TzM[VY];
    float s0 = 0.f;
#pragma unroll
    for (int i = 0; i < S; ++i) issue(i);
    cp_wait<S - 3>();
    {  // plane z0 - 1: the direction below the first output plane, and its Tz
      float Pt[VY + 2], Rt[VY];
      form(1, Pt, Rt, s0);
      const float4* cf = reinterpret_cast<const float4*>(stage(1) + LY::kCoef);
#pragma unroll
      for (int jj = 0; jj < VY; ++jj) {
        PkM[jj] = Pt[jj + 1];
        TzM[jj] = cf[(jj + 1) * 32 + lane].z;
      }
    }
    issue(S);  // into the stage of plane z0 - 2, read for the last time above
    cp_wait<S - 3>();
    form(2, Pk0, Rk0, s0);

#pragma unroll 1
    for (int64_t z = z0; z < z1; ++z) {
      const int64_t jz = z - z0 + 2;
      issue(jz + S - 1);  // into the stage of plane z - 1, no longer read
      cp_wait<S - 3>();
      float PkP[VY + 2], RkP[VY];
      form(jz + 1, PkP, RkP, s0);
      // q_k = A p_k on the output rows of plane z (Alg. 2)
      const float4* cf = reinterpret_cast<const float4*>(stage(jz) + LY::kCoef);
      float s1 = 0.f, s2 = 0.f, s3 = 0.f;
      float tyl = cf[lane].y;  // record row -1
#pragma unroll
      for (int jj = 0; jj < VY; ++jj) {
        const float4 c = cf[(jj + 1) * 32 + lane];
        const float pc = Pk0[jj + 1];
        const float pxm = __shfl_up_sync(kFull, pc, 1);
        const float pxp = __shfl_down_sync(kFull, pc, 1);
        const float txm = __shfl_up_sync(kFull, c.x, 1);
        const float q = stencil7(c, txm, tyl, TzM[jj], pc, pxp, pxm, Pk0[jj + 2], Pk0[jj],
                                 PkP[jj + 1], PkM[jj]);
        if (outl && ((rowok >> (jj + 2)) & 1u)) {
          s1 = fmaf(pc, q, s1);
          s2 = fmaf(Rk0[jj], q, s2);
          s3 = fmaf(q, q, s3);
        }
        tyl = c.y;
        TzM[jj] = c.z;
        PkM[jj] = pc;
      }
      kadd(acc[0], s0);
      kadd(acc[1], s1);
      kadd(acc[2], s2);
      kadd(acc[3], s3);
      s0 = 0.f;
#pragma unroll
      for (int jj = 0; jj < VY; ++jj) Rk0[jj] = RkP[jj];
#pragma unroll
      for (int jj = 0; jj < VY + 2; ++jj) Pk0[jj] = PkP[jj];
    }
    kadd(acc[0], s0);
    cp_wait<0>();
  }

  double v[4] = {kval(acc[0]), kval(acc[1]), kval(acc[2]), kval(acc[3])};
  block_partial<4>(v, a.partials);
  double tot[4];
  if (last_block_total<4>(a.partials, a.counter, tot) && threadIdx.x == 0)
    cg_finish(a.st, tot, a.cond, COND);
}

// End of an inner solve for this variant: x_{k+1} = x_k + alpha_fin p_k.
// (No q is stored, so the recursive residual is not advanced here; the FP64
// residual that follows is the check.)
__global__ void __launch_bounds__(kElemThreads)
finalize40_kernel(Grid g, CgVecs v, const CgState* st) {
  const float af = (float)st->alpha_fin;
  const float* p = v.p[st->parity];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < g.n; c += stride)
    v.e[c] = fmaf(af, p[c], v.e[c]);
}

template <int S, int W, bool COND>
cudaError_t launch40_t(const Cg40Args& a, int64_t nblocks, cudaStream_t s) {
  constexpr int smem = cg40_smem_bytes<S, W>();
  cudaError_t e = cudaFuncSetAttribute(cg40_kernel<S, W, COND>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  cg40_kernel<S, W, COND><<<(unsigned)nblocks, W * 32, smem, s>>>(a);
  return cudaGetLastError();
}

template <int S, int W>
int blocks_per_sm40_t() {
  constexpr int smem = cg40_smem_bytes<S, W>();
  if (cudaFuncSetAttribute(cg40_kernel<S, W, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           smem) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cg40_kernel<S, W, true>, W * 32, smem) !=
      cudaSuccess)
    return 0;
  return nb;
}

}  // namespace

Sweep plan_sweep40(const Grid& g, int stages, int warps, int zc_opt, int num_sms) {
  Sweep s;
  s.vy = kVY40;
  s.stages = stages;
  s.warps = warps;
  s.nwx = (g.nx + kTileX40 - 1) / kTileX40;
  s.nwy = (g.ny + kVY40 - 1) / kVY40;
  int zc = zc_opt;
  if (zc <= 0) {
    const int64_t target = (int64_t)num_sms * 8 * 4;
    const int64_t cols = s.nwx * s.nwy;
    zc = 128;
    while (zc > 1 && cols * ((g.nz + zc - 1) / zc) < target) zc /= 2;
  }
  if (zc > g.nz) zc = (int)g.nz;
  s.zc = zc;
  s.nwz = (g.nz + zc - 1) / zc;
  s.nwarps = s.nwx * s.nwy * s.nwz;
  s.nblocks = (s.nwarps + warps - 1) / warps;
  return s;
}

bool sweep40_config_ok(int stages, int warps) {
  return (warps == 2 && (stages == 4 || stages == 5 || stages == 6)) ||
         (warps == 4 && (stages == 4 || stages == 5));
}

cudaError_t launch_cg40_sweep(const Grid& g, const Sweep& sw, const float4* coef, CgVecs v,
                              CgState* st, double* partials, unsigned int* counter,
                              unsigned long long cond, int use_cond, cudaStream_t s) {
  Cg40Args a{};
  a.g = g;
  a.nwx = sw.nwx;
  a.nwy = sw.nwy;
  a.nwarps = sw.nwarps;
  a.zc = sw.zc;
  a.coef = coef;
  a.v = v;
  a.st = st;
  a.partials = partials;
  a.counter = counter;
  a.cond = cond;
  const bool c = use_cond != 0;
#define TPFA_CG40(S_, W_) \
  if (sw.stages == S_ && sw.warps == W_) \
    return c ? launch40_t<S_, W_, true>(a, sw.nblocks, s) : launch40_t<S_, W_, false>(a, sw.nblocks, s);
  TPFA_CG40(4, 2)
  TPFA_CG40(5, 2)
  TPFA_CG40(6, 2)
  TPFA_CG40(4, 4)
  TPFA_CG40(5, 4)
#undef TPFA_CG40
  return cudaErrorInvalidValue;
}

int sweep40_blocks_per_sm(int stages, int warps) {
  int nb = 0;
  if (warps == 2 && stages == 4) nb = blocks_per_sm40_t<4, 2>();
  else if (warps == 2 && stages == 5) nb = blocks_per_sm40_t<5, 2>();
  else if (warps == 2 && stages == 6) nb = blocks_per_sm40_t<6, 2>();
  else if (warps == 4 && stages == 4) nb = blocks_per_sm40_t<4, 4>();
  else if (warps == 4 && stages == 5) nb = blocks_per_sm40_t<5, 4>();
  if (nb == 0) cudaGetLastError();
  return nb;
}

cudaError_t launch_finalize40(const Grid& g, CgVecs v, const CgState* st, int nblocks,
                              cudaStream_t s) {
  finalize40_kernel<<<nblocks, kElemThreads, 0, s>>>(g, v, st);
  return cudaGetLastError();
}

}  // namespace tpfa
