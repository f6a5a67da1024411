// Stencil sweeps, fused CG iteration, FP64 residual and refinement kernels.
//
// The operator is the matrix-free TPFA product of Eq. 6 / Alg. 2 (arXiv
// 2408.03452, Section II.A) in its symmetric positive form
//   (A p)_K = D_K p_K - sum_faces T_f p_nbr,
// read from one 16-byte coefficient record per cell (Tx, Ty, Tz, D).
//
// Sweep layout (both the plain operator and the fused CG iteration): each
// warp owns a column block of 32 x-lanes (lanes 1..30 produce output, lanes
// 0 and 31 carry the x-halo), VY consecutive y-rows, and marches through zc
// consecutive z-planes, keeping the z-neighbours in registers.  x-neighbours
// come from warp shuffles, y-neighbours from the warp's own rows plus one
// halo row on each side.  Every plane a warp needs is staged into a
// per-warp shared-memory ring with cp.async (zero-filled outside the grid)
// two planes ahead of the plane being computed; each input array is read
// once per sweep from DRAM, halo rows and columns are L2 hits.  There is no
// block-level barrier inside the march: warps are independent.
//
// Reductions are deterministic: per-thread compensated FP32 sums over a
// fixed cell set, FP64 warp shuffles in a fixed tree, FP64 block sums in a
// fixed order, and a last-block finish that adds the block partials in a
// fixed order (no floating-point atomics).
#include <math.h>

#include "sweep_common.cuh"

namespace tpfa {

namespace {

struct SweepArgs {
  const BatchInst* inst;  // batched sweeps: instance table (ninst entries)
  int ninst;
  Grid g;
  int64_t nwx, nwy, nwarps;
  int zc;
  const float4* coef;     // FP32 records (Tx, Ty, Tz, D)
  const uint2* coef16;    // BF16 records (Tx, Ty, Tz, E), D = sum of the six T + E
  const float* dinv;      // Jacobi with BF16 records: M^-1 per cell (dinv_bf16_kernel)
  // plain operator
  const float* p;
  float* Ap;
  double* pAp;            // batched: one value per instance
  const int* act;         // batched operator: instance i is swept iff (act[i] & need) == need
  int need;
  // fused CG iteration
  CgVecs v;
  CgState* st;
  double* partials;
  unsigned int* counter;
  unsigned long long cond;
};

// Shared-memory stage of one warp for one z-plane: the coefficient records
// of the warp's VY rows, r/q/p (or p alone) of rows -1..VY, x of the VY
// rows, and the word holding Ty of row -1.  Lane-minor, each lane reads only
// its own column.  Records are 16 bytes (FP32) or 8 bytes (BF16).
// With Jacobi preconditioning and FP32 records the stage also holds D of the
// halo rows -1 and VY (the records of the own rows carry theirs); with BF16
// records, which do not store D, it holds M^-1 of every row -1 .. VY.
template <int VY, bool B16, bool JAC = false>
struct StageLayout {
  static constexpr int kRec = B16 ? 8 : 16;
  static constexpr int kCoef = 0;                               // record [VY][32]
  static constexpr int kVec = VY * 32 * kRec;                   // float [3][VY+2][32]
  static constexpr int kE = kVec + 3 * (VY + 2) * 32 * 4;       // float [VY][32]
  static constexpr int kTy = kE + VY * 32 * 4;                  // 32-bit word [32]
  static constexpr int kDh = kTy + 32 * 4;                      // float [2 or VY+2][32] (JAC)
  static constexpr int kDhRows = JAC ? (B16 ? VY + 2 : 2) : 0;
  static constexpr int kBytes = kDh + kDhRows * 32 * 4;
};

template <int VY, int S, bool B16, bool JAC = false>
constexpr int sweep_smem_bytes() { return kSweepWarps * S * StageLayout<VY, B16, JAC>::kBytes; }

// A staged record as (Tx, Ty, Tz, w): w = D for FP32 records, w = E (the
// diagonal beyond the six face terms) for BF16 records.
template <bool B16>
__device__ __forceinline__ float4 rec_at(const unsigned char* base, int i) {
  if (B16) {
    const uint2 u = reinterpret_cast<const uint2*>(base)[i];
    return make_float4(bf16_lo(u.x), bf16_hi(u.x), bf16_lo(u.y), bf16_hi(u.y));
  }
  return reinterpret_cast<const float4*>(base)[i];
}
// Ty from the staged Ty word of row -1
template <bool B16>
__device__ __forceinline__ float ty_word(const unsigned char* base, int lane) {
  const unsigned w = reinterpret_cast<const unsigned*>(base)[lane];
  return B16 ? bf16_hi(w) : __uint_as_float(w);
}

// JAC: Jacobi-preconditioned CG (M = diag(D)).  The preconditioned residual
// z = r / D is formed on the fly, p_k = z_k + beta p_{k-1}, and the four
// dots become r'z, p'q, z'q, q'D^-1 q, which give alpha = r'z / p'q and
// (r - alpha q)' D^-1 (r - alpha q) by the same identity as the plain
// iteration.  With FP32 records no extra vector is read or written; with
// BF16 records M^-1 is read from a per-cell FP32 array (4 B/cell).
// BATCH: one launch sweeps every instance of a batch; each block finds its
// instance in the table (blocks of one instance are contiguous) and uses that
// instance's grid, tiling, cell offset, CG state, completion counter and
// partial sums.  A finished instance's blocks return at once.  Without CG it
// is the plain operator of every instance whose activity flags hold the
// requested bits, with p'Ap per instance.
template <int VY, int S, bool CG, bool COND, bool B16, bool JAC = false, bool BATCH = false>
__global__ void __launch_bounds__(kSweepWarps * 32)
sweep_kernel(const SweepArgs a) {
  static_assert(S >= 3, "the plane pipeline needs at least three stages");
  static_assert(!JAC || CG, "Jacobi preconditioning is for CG sweeps");
  static_assert(!BATCH || (!B16 && !COND), "batched sweeps use FP32 records, no graph condition");
  static_assert(!BATCH || !JAC || CG, "the batched operator has no preconditioner");
  using LY = StageLayout<VY, B16, JAC>;
  extern __shared__ __align__(16) unsigned char smem[];
  Grid g = a.g;
  int64_t nwx = a.nwx, nwy = a.nwy, nwarps = a.nwarps, zcr = a.zc, off = 0;
  int64_t lb = blockIdx.x, pstart = 0, pcount = gridDim.x;
  int inst = 0;
  CgState* st = a.st;
  unsigned int* counter = a.counter;
  if (BATCH) {
    int lo = 0, hi = a.ninst - 1;  // last instance whose first block <= blockIdx.x
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.inst[mid].bstart <= (int64_t)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    const BatchInst& I = a.inst[lo];
    g = I.g; nwx = I.nwx; nwy = I.nwy; nwarps = I.nwarps; zcr = I.zc; off = I.off;
    lb = blockIdx.x - I.bstart; pstart = I.bstart; pcount = I.nblocks;
    inst = lo;
    counter = a.counter + lo;
    if (CG) st = a.st + lo;
    else if ((a.act[lo] & a.need) != a.need) return;  // every block of the instance returns
  }
  const float4* coefp = a.coef != nullptr ? a.coef + off : nullptr;
  float* ep = CG ? a.v.e + off : nullptr;
  float alpha = 0.f, beta = 0.f;
  const float *rin = nullptr, *qin = nullptr, *pin = CG ? nullptr : a.p + off;
  float *rout = nullptr, *qout = nullptr, *pout = nullptr;
  float* apo = CG ? nullptr : a.Ap + off;
  if (CG) {
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
    alpha = (float)st->alpha;
    beta = (float)st->beta;
    rin = a.v.r[par] + off; qin = a.v.q[par] + off; pin = a.v.p[par] + off;
    rout = a.v.r[par ^ 1] + off; qout = a.v.q[par ^ 1] + off; pout = a.v.p[par ^ 1] + off;
  }

  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int64_t gw = lb * kSweepWarps + wib;
  unsigned char* wsm = smem + (size_t)wib * S * LY::kBytes;
  Acc acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};

  if (gw < nwarps) {  // warp-uniform
    const int64_t wx = gw % nwx;
    const int64_t t = gw / nwx;
    const int64_t wy = t % nwy;
    const int64_t wz = t / nwy;
    const int64_t gx = wx * kTileX - 1 + lane;
    const bool inx = gx >= 0 && gx < g.nx;
    const bool outl = inx && lane >= 1 && lane <= kTileX;
    const int64_t y0 = wy * VY;
    const int64_t z0 = wz * zcr;
    const int64_t z1 = min(z0 + zcr, g.nz);
    unsigned rowok = 0u;  // bit jj+1: row y0+jj inside the grid (and this lane's column too)
#pragma unroll
    for (int jj = -1; jj <= VY; ++jj)
      if (inx && y0 + jj >= 0 && y0 + jj < g.ny) rowok |= 1u << (jj + 1);
    // in-plane offset of (gx, y0) (fits 32 bits: nx*ny + 2nx < 2^31 is
    // checked at context creation); row jj at + jj*nx, plane z at + z*nx*ny
    const int nxi = (int)g.nx;
    const int o0 = (int)(gx + g.nx * y0);
    const int64_t L = z1 - z0 + 2;  // planes z0-1 .. z1

    // Issue the asynchronous copies of plane j (absolute z = z0 - 1 + j)
    // into stage j % S; out-of-grid cells are zero-filled.  Always commits
    // one group so that group counts stay uniform.
    auto issue = [&](int64_t j) {
      if (j < L) {
        const int64_t z = z0 - 1 + j;
        const bool zok = z >= 0 && z < g.nz;
        const int64_t zo = g.plane * (z < 0 ? 0 : (z >= g.nz ? g.nz - 1 : z));
        const bool own = outl && z >= z0 && z < z1;
        unsigned char* sb = wsm + (size_t)(j % S) * LY::kBytes;
        unsigned char* scf = sb + LY::kCoef;
        float* sv = reinterpret_cast<float*>(sb + LY::kVec);
        float* se = reinterpret_cast<float*>(sb + LY::kE);
        float* sty = reinterpret_cast<float*>(sb + LY::kTy);
#pragma unroll
        for (int jj = -1; jj <= VY; ++jj) {
          const bool ok = zok && ((rowok >> (jj + 1)) & 1u);
          const int64_t src = zo + (ok ? (int64_t)(o0 + jj * nxi) : 0);
          if (CG) {
            cp4(sv + (0 * (VY + 2) + jj + 1) * 32 + lane, rin + src, ok);
            cp4(sv + (1 * (VY + 2) + jj + 1) * 32 + lane, qin + src, ok);
            cp4(sv + (2 * (VY + 2) + jj + 1) * 32 + lane, pin + src, ok);
          } else {
            cp4(sv + (2 * (VY + 2) + jj + 1) * 32 + lane, pin + src, ok);
          }
          if (jj == -1) {
            if (B16) cp4(sty + lane, a.coef16 + src, ok);  // word 0 = Tx | Ty << 16
            else cp4(sty + lane, reinterpret_cast<const float*>(coefp + src) + 1, ok);
          }
          if (JAC && !B16 && (jj == -1 || jj == VY))
            cp4(reinterpret_cast<float*>(sb + LY::kDh) + (jj == -1 ? 0 : 32) + lane,
                reinterpret_cast<const float*>(coefp + src) + 3, ok);
          if (JAC && B16)
            cp4(reinterpret_cast<float*>(sb + LY::kDh) + (jj + 1) * 32 + lane, a.dinv + src, ok);
          if (jj >= 0 && jj < VY) {
            if (B16) cp8(reinterpret_cast<uint2*>(scf) + jj * 32 + lane, a.coef16 + src, ok);
            else cp16(reinterpret_cast<float4*>(scf) + jj * 32 + lane, coefp + src, ok);
            if (CG) cp4(se + jj * 32 + lane, ep + src, ok && own);
          }
        }
      }
      cp_commit();
    };

    // Form r_k and p_k on plane j from its stage (rows -1 .. VY).  For this
    // warp's own output cells also write r_k, p_k and the x update
    // x_k = x_{k-1} + alpha p_{k-1}, and accumulate r_k'r_k.
    auto form = [&](int64_t j, float (&P)[VY + 2], float (&R)[VY], float& s0) {
      const int64_t z = z0 - 1 + j;
      const bool own = outl && z >= z0 && z < z1;
      const unsigned char* sb = wsm + (size_t)(j % S) * LY::kBytes;
      const float* sv = reinterpret_cast<const float*>(sb + LY::kVec);
      const float* se = reinterpret_cast<const float*>(sb + LY::kE);
      const int64_t zo = g.plane * z;
#pragma unroll
      for (int jj = -1; jj <= VY; ++jj) {
        const float p0 = sv[(2 * (VY + 2) + jj + 1) * 32 + lane];
        float p_ = p0, r_ = 0.f;
        if (CG) {
          const float r0 = sv[(0 * (VY + 2) + jj + 1) * 32 + lane];
          const float q0 = sv[(1 * (VY + 2) + jj + 1) * 32 + lane];
          r_ = fmaf(-alpha, q0, r0);  // Alg. 1 line 7 (previous iteration)
          float z_ = r_;
          if (JAC && B16) {
            z_ = r_ * reinterpret_cast<const float*>(sb + LY::kDh)[(jj + 1) * 32 + lane];
          } else if (JAC) {
            const float D = (jj == -1 || jj == VY)
                ? reinterpret_cast<const float*>(sb + LY::kDh)[(jj == -1 ? 0 : 32) + lane]
                : rec_at<false>(sb + LY::kCoef, jj * 32 + lane).w;
            z_ = r_ * jac_inv(D);  // z = M^-1 r
          }
          p_ = fmaf(beta, p0, z_);    // Alg. 1 line 10
          if (jj >= 0 && jj < VY && own && ((rowok >> (jj + 1)) & 1u)) {
            const int64_t id = zo + o0 + jj * nxi;
            ep[id] = fmaf(alpha, p0, se[jj * 32 + lane]);  // Alg. 1 line 6
            rout[id] = r_;
            pout[id] = p_;
            s0 = fmaf(r_, z_, s0);
          }
          r_ = z_;  // the direction dots below use z (= r without preconditioning)
        }
        P[jj + 1] = p_;
        if (jj >= 0 && jj < VY) R[jj] = r_;
      }
    };

    float Pm[VY], P0[VY + 2], R0[VY], Tzm[VY];
    float s0 = 0.f;
#pragma unroll
    for (int i = 0; i < S - 1; ++i) issue(i);
    cp_wait<S - 2>();
    {  // plane z0 - 1: direction below the first plane, and its Tz
      float Pt[VY + 2], Rt[VY];
      form(0, Pt, Rt, s0);
#pragma unroll
      for (int jj = 0; jj < VY; ++jj) {
        Pm[jj] = Pt[jj + 1];
        Tzm[jj] = rec_at<B16>(wsm + LY::kCoef, jj * 32 + lane).z;
      }
    }
    issue(S - 1);
    cp_wait<S - 2>();
    form(1, P0, R0, s0);

#pragma unroll 1
    for (int64_t z = z0; z < z1; ++z) {
      const int64_t jf = z - z0 + 2;  // plane z + 1
      issue(jf + S - 2);              // reuses the stage of plane z - 1
      cp_wait<S - 2>();
      float Pp[VY + 2], Rp[VY];
      form(jf, Pp, Rp, s0);
      const unsigned char* sb = wsm + (size_t)((jf - 1) % S) * LY::kBytes;  // plane z
      const int64_t zo = g.plane * z;
      float s1 = 0.f, s2 = 0.f, s3 = 0.f, tyl = ty_word<B16>(sb + LY::kTy, lane);
#pragma unroll
      for (int jj = 0; jj < VY; ++jj) {
        float4 cf = rec_at<B16>(sb + LY::kCoef, jj * 32 + lane);
        const float pc = P0[jj + 1];
        const float pxm = __shfl_up_sync(kFull, pc, 1);
        const float pxp = __shfl_down_sync(kFull, pc, 1);
        const float txm = __shfl_up_sync(kFull, cf.x, 1);
        // BF16 records: D = T(-x) + T(+x) + T(-y) + T(+y) + T(-z) + T(+z) + E
        if (B16) cf.w = (((((txm + cf.x) + tyl) + cf.y) + Tzm[jj]) + cf.z) + cf.w;
        const float q = stencil7(cf, txm, tyl, Tzm[jj], pc, pxp, pxm, P0[jj + 2], P0[jj],
                                 Pp[jj + 1], Pm[jj]);
        if (outl && ((rowok >> (jj + 1)) & 1u)) {
          const int64_t id = zo + o0 + jj * nxi;
          if (CG) {
            qout[id] = q;
            s1 = fmaf(pc, q, s1);
            s2 = fmaf(R0[jj], q, s2);
            if (JAC && B16)
              s3 = fmaf(q, q * reinterpret_cast<const float*>(sb + LY::kDh)[(jj + 1) * 32 + lane], s3);
            else if (JAC) s3 = fmaf(q, q * jac_inv(cf.w), s3);
            else s3 = fmaf(q, q, s3);
          } else {
            apo[id] = q;
            s1 = fmaf(pc, q, s1);
          }
        }
        tyl = cf.y;
        Tzm[jj] = cf.z;
        Pm[jj] = pc;
      }
      kadd(acc[1], s1);
      if (CG) {
        kadd(acc[0], s0);
        kadd(acc[2], s2);
        kadd(acc[3], s3);
        s0 = 0.f;
#pragma unroll
        for (int jj = 0; jj < VY; ++jj) R0[jj] = Rp[jj];
      }
#pragma unroll
      for (int jj = 0; jj < VY + 2; ++jj) P0[jj] = Pp[jj];
    }
    if (CG) kadd(acc[0], s0);
    cp_wait<0>();  // drain the (empty) trailing groups before the warp leaves
  }

  if (CG) {
    double v[4] = {kval(acc[0]), kval(acc[1]), kval(acc[2]), kval(acc[3])};
    block_partial<4>(v, a.partials);
    double tot[4];
    if (last_block_range<4>(a.partials, counter, pstart, pcount, tot) && threadIdx.x == 0)
      cg_finish(st, tot, a.cond, COND);
  } else if (a.pAp != nullptr) {
    double v[1] = {kval(acc[1])};
    block_partial<1>(v, a.partials);
    double tot[1];
    if (last_block_range<1>(a.partials, counter, pstart, pcount, tot) && threadIdx.x == 0)
      a.pAp[inst] = tot[0];
  }
}

// ---------------------------------------------------------------------------
// FP64 residual r = b - A x (one thread per cell, grid-stride, fixed grid).
__global__ void __launch_bounds__(kElemThreads)
residual64_kernel(Grid g, const double2* __restrict__ coef64, const double* __restrict__ b,
                  const double* __restrict__ x, double* __restrict__ r, double* norms,
                  CgState* st, double* partials, unsigned int* counter) {
  double rr = 0.0, bb = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < g.n; c += stride) {
    const int64_t i = c % g.nx, j = (c / g.nx) % g.ny, k = c / g.plane;
    const double2 c01 = __ldg(coef64 + 2 * c), c23 = __ldg(coef64 + 2 * c + 1);
    const double xc = __ldg(x + c);
    double s = c23.y * xc;
    if (i + 1 < g.nx) s = fma(-c01.x, __ldg(x + c + 1), s);
    if (i > 0) s = fma(-__ldg(&coef64[2 * (c - 1)].x), __ldg(x + c - 1), s);
    if (j + 1 < g.ny) s = fma(-c01.y, __ldg(x + c + g.nx), s);
    if (j > 0) s = fma(-__ldg(&coef64[2 * (c - g.nx)].y), __ldg(x + c - g.nx), s);
    if (k + 1 < g.nz) s = fma(-c23.x, __ldg(x + c + g.plane), s);
    if (k > 0) s = fma(-__ldg(&coef64[2 * (c - g.plane) + 1].x), __ldg(x + c - g.plane), s);
    const double bc = __ldg(b + c);
    const double rc = bc - s;
    r[c] = rc;
    rr = fma(rc, rc, rr);
    bb = fma(bc, bc, bb);
  }
  double v[2] = {rr, bb};
  block_partial<2>(v, partials);
  double tot[2];
  if (last_block_total<2>(partials, counter, tot) && threadIdx.x == 0) {
    if (norms != nullptr) { norms[0] = tot[0]; norms[1] = tot[1]; }
    if (st != nullptr) { st->rr64 = tot[0]; st->bb64 = tot[1]; }
  }
}

// Start of an inner solve: r32 = scale * r64 with scale = 1/||r64||, zero
// correction and directions, reset the scalars.
__global__ void __launch_bounds__(kElemThreads)
prepare_kernel(Grid g, const double* __restrict__ r64, CgVecs v, CgState* st, double rtol2,
               long long maxit) {
  const double rr = st->rr64;
  const double scale = rr > 0.0 ? 1.0 / sqrt(rr) : 1.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < g.n; c += stride) {
    if (v.v4[0] != nullptr) {  // interleaved records (r, q, p, x)
      v.v4[0][c] = make_float4((float)(scale * r64[c]), 0.f, 0.f, 0.f);
    } else {
      v.r[0][c] = (float)(scale * r64[c]);
      v.p[0][c] = 0.f;
      v.q[0][c] = 0.f;
      v.e[c] = 0.f;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->alpha = 0.0; st->beta = 0.0; st->rho = 0.0; st->rho0 = 0.0; st->rho_est = 0.0;
    st->alpha_fin = 0.0;
    st->rtol2 = rtol2;
    st->scale = scale;
    st->iter = 0; st->maxit = maxit; st->launches = 0;
    st->guard_limit = 2 * maxit + 64;
    st->parity = 0; st->done = kRunning; st->fault = 0;
  }
}

// End of an inner solve: apply the last step alpha_fin (x += alpha p,
// r -= alpha q) and recompute r'r from the stored residual.  If the
// estimate that stopped the loop was too optimistic, arm a restart of the
// loop with the exact CG continuation (alpha = 0, beta = r+'r+ / r'r).
__global__ void __launch_bounds__(kElemThreads)
finalize_kernel(Grid g, CgVecs v, CgState* st, double* partials, unsigned int* counter,
                const float4* jac, const float* dinv) {
  const int par = st->parity;
  const float af = (float)st->alpha_fin;
  float* r = v.r[par];
  const float* p = v.p[par];
  const float* q = v.q[par];
  float4* v4 = v.v4[par];
  Acc acc = {0.f, 0.f};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < g.n; c += stride) {
    float rn;
    if (v4 != nullptr) {  // interleaved records (r, q, p, x)
      float4 t = v4[c];
      t.w = fmaf(af, t.z, t.w);
      rn = fmaf(-af, t.y, t.x);
      t.x = rn;
      v4[c] = t;
    } else {
      v.e[c] = fmaf(af, p[c], v.e[c]);
      rn = fmaf(-af, q[c], r[c]);
      r[c] = rn;
    }
    if (dinv != nullptr) {  // preconditioned norm r' M^-1 r (BF16 records)
      kadd(acc, rn * (rn * dinv[c]));
    } else if (jac != nullptr) {  // preconditioned norm r' D^-1 r
      kadd(acc, rn * (rn * jac_inv(jac[c].w)));
    } else {
      kadd(acc, rn * rn);
    }
  }
  double vv[1] = {kval(acc)};
  block_partial<1>(vv, partials);
  double tot[1];
  if (last_block_total<1>(partials, counter, tot) && threadIdx.x == 0) {
    const double rho1 = tot[0];
    const int done = st->done;
    if (done == kConvEst || done == kMaxit) {
      const double rho_prev = st->rho;
      st->rho = rho1;
      st->alpha_fin = 0.0;
      if (done == kConvEst && rho1 > st->rtol2 * st->rho0 && st->iter < st->maxit &&
          isfinite(rho1) && rho_prev > 0.0) {
        st->alpha = 0.0;
        st->beta = rho1 / rho_prev;
        st->done = kRunning;
      }
    }
  }
}

// M^-1 = jac_inv(D) per cell for Jacobi with BF16 records, where D is the
// diagonal the BF16 sweep forms: the six rounded face values and E added in
// the sweep's order (zero for faces on the outer boundary), so that the
// preconditioner is one fixed function of the operator the sweep applies.
__global__ void __launch_bounds__(kElemThreads)
dinv_bf16_kernel(Grid g, const uint2* __restrict__ coef16, float* __restrict__ dinv) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < g.n; c += stride) {
    const int64_t i = c % g.nx, j = (c / g.nx) % g.ny, k = c / g.plane;
    const uint2 u = __ldg(coef16 + c);
    const float txm = i > 0 ? bf16_lo(__ldg(&coef16[c - 1].x)) : 0.f;
    const float tym = j > 0 ? bf16_hi(__ldg(&coef16[c - g.nx].x)) : 0.f;
    const float tzm = k > 0 ? bf16_lo(__ldg(&coef16[c - g.plane].y)) : 0.f;
    const float D = (((((txm + bf16_lo(u.x)) + tym) + bf16_hi(u.x)) + tzm) + bf16_lo(u.y)) +
                    bf16_hi(u.y);
    dinv[c] = jac_inv(D);
  }
}

// x64 += e / scale (e: the correction array, or the x component of the
// current interleaved record set).
__global__ void __launch_bounds__(kElemThreads)
correct_kernel(Grid g, CgVecs v, double* __restrict__ x, const CgState* st) {
  const double inv = 1.0 / st->scale;
  const float4* v4 = v.v4[st->parity];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < g.n; c += stride)
    x[c] = fma((double)(v4 != nullptr ? v4[c].w : v.e[c]), inv, x[c]);
}

}  // namespace

// ---------------------------------------------------------------------------

bool sweep_config_ok(int vy, int stages) {
  return (vy == 4 && (stages == 3 || stages == 4)) || (vy == 8 && stages == 3);
}

int elem_blocks(const Grid& g, int num_sms) {
  const int64_t need = (g.n + kElemThreads - 1) / kElemThreads;
  const int64_t cap = (int64_t)num_sms * 8;
  return (int)(need < cap ? (need > 0 ? need : 1) : cap);
}

static SweepArgs sweep_args(const Grid& g, const Sweep& sw, const float4* coef) {
  SweepArgs a{};
  a.g = g;
  a.nwx = sw.nwx;
  a.nwy = sw.nwy;
  a.nwarps = sw.nwarps;
  a.zc = sw.zc;
  a.coef = coef;
  return a;
}

template <int VY, int S, bool CG, bool COND, bool B16, bool JAC = false, bool BATCH = false>
static cudaError_t launch_t(const SweepArgs& a, const Sweep& sw, cudaStream_t s) {
  constexpr int smem = sweep_smem_bytes<VY, S, B16, JAC>();
  cudaError_t e = cudaFuncSetAttribute(sweep_kernel<VY, S, CG, COND, B16, JAC, BATCH>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  sweep_kernel<VY, S, CG, COND, B16, JAC, BATCH>
      <<<(unsigned)sw.nblocks, kSweepWarps * 32, smem, s>>>(a);
  return cudaGetLastError();
}

template <int VY, int S, bool B16>
static cudaError_t launch_vs(const SweepArgs& a, const Sweep& sw, bool cg, bool cond,
                             cudaStream_t s) {
  if (!cg) return launch_t<VY, S, false, false, B16>(a, sw, s);
  if (cond) return launch_t<VY, S, true, true, B16>(a, sw, s);
  return launch_t<VY, S, true, false, B16>(a, sw, s);
}

static cudaError_t launch_sweep(const SweepArgs& a, const Sweep& sw, bool cg, bool cond,
                                cudaStream_t s) {
  const bool b16 = a.coef16 != nullptr;
  if (b16) {
    if (sw.vy == 4 && sw.stages == 3) return launch_vs<4, 3, true>(a, sw, cg, cond, s);
    if (sw.vy == 4 && sw.stages == 4) return launch_vs<4, 4, true>(a, sw, cg, cond, s);
    return cudaErrorInvalidValue;
  }
  if (sw.vy == 4 && sw.stages == 3) return launch_vs<4, 3, false>(a, sw, cg, cond, s);
  if (sw.vy == 4 && sw.stages == 4) return launch_vs<4, 4, false>(a, sw, cg, cond, s);
  if (sw.vy == 8 && sw.stages == 3) return launch_vs<8, 3, false>(a, sw, cg, cond, s);
  return cudaErrorInvalidValue;
}

static SweepArgs sweep_args_rec(const Grid& g, const Sweep& sw, const void* coef, bool b16) {
  SweepArgs a = sweep_args(g, sw, b16 ? nullptr : static_cast<const float4*>(coef));
  a.coef16 = b16 ? static_cast<const uint2*>(coef) : nullptr;
  return a;
}

cudaError_t launch_apply(const Grid& g, const Sweep& sw, const void* coef, bool b16,
                         const float* p, float* Ap, double* pAp, double* partials,
                         unsigned int* counter, cudaStream_t s) {
  SweepArgs a = sweep_args_rec(g, sw, coef, b16);
  a.p = p;
  a.Ap = Ap;
  a.pAp = pAp;
  a.partials = partials;
  a.counter = counter;
  return launch_sweep(a, sw, false, false, s);
}

template <int S, bool B16>
static cudaError_t launch_jac(const SweepArgs& a, const Sweep& sw, bool cond, cudaStream_t s) {
  return cond ? launch_t<4, S, true, true, B16, true>(a, sw, s)
              : launch_t<4, S, true, false, B16, true>(a, sw, s);
}

cudaError_t launch_cg_sweep_jacobi(const Grid& g, const Sweep& sw, const void* coef, bool b16,
                                   const float* dinv, CgVecs v, CgState* st, double* partials,
                                   unsigned int* counter, unsigned long long cond, int use_cond,
                                   cudaStream_t s) {
  SweepArgs a = sweep_args_rec(g, sw, coef, b16);
  a.dinv = dinv;
  a.v = v;
  a.st = st;
  a.partials = partials;
  a.counter = counter;
  a.cond = cond;
  const bool c = use_cond != 0;
  if (b16 && dinv == nullptr) return cudaErrorInvalidValue;
  if (sw.vy == 4 && sw.stages == 3) return b16 ? launch_jac<3, true>(a, sw, c, s) : launch_jac<3, false>(a, sw, c, s);
  if (sw.vy == 4 && sw.stages == 4) return b16 ? launch_jac<4, true>(a, sw, c, s) : launch_jac<4, false>(a, sw, c, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_dinv_bf16(const Grid& g, const uint2* coef16, float* dinv, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  dinv_bf16_kernel<<<elem_blocks(g, sms), kElemThreads, 0, s>>>(g, coef16, dinv);
  return cudaGetLastError();
}

// Condition of the batched while loop: continue while any instance runs
// (one block; a single thread sets the condition).
__global__ void batch_cond_kernel(const CgState* st, int ninst, unsigned long long cond,
                                  long long* sweeps, long long limit) {
  __shared__ int running;
  if (threadIdx.x == 0) running = 0;
  __syncthreads();
  int r = 0;
  for (int i = threadIdx.x; i < ninst; i += blockDim.x) r += st[i].done == kRunning ? 1 : 0;
  if (r) atomicAdd(&running, r);
  __syncthreads();
  if (threadIdx.x == 0) {
    const long long n = *sweeps + 1;
    *sweeps = n;
    cudaGraphSetConditional(cond, (running > 0 && n <= limit) ? 1u : 0u);
  }
}

cudaError_t launch_cg_sweep_batch(const BatchInst* inst, int ninst, int64_t nblocks,
                                  const float4* coef, CgVecs v, CgState* st, double* partials,
                                  unsigned int* counters, bool jac, cudaStream_t s) {
  SweepArgs a{};
  a.inst = inst;
  a.ninst = ninst;
  a.coef = coef;
  a.v = v;
  a.st = st;
  a.partials = partials;
  a.counter = counters;
  Sweep sw{};
  sw.nblocks = nblocks;
  if (jac) return launch_t<4, 4, true, false, false, true, true>(a, sw, s);
  return launch_t<4, 4, true, false, false, false, true>(a, sw, s);
}

cudaError_t launch_apply_batch(const BatchInst* inst, int ninst, int64_t nblocks,
                               const float4* coef, const float* p, float* Ap, double* pAp,
                               const int* act, int need, double* partials,
                               unsigned int* counters, cudaStream_t s) {
  SweepArgs a{};
  a.inst = inst;
  a.ninst = ninst;
  a.coef = coef;
  a.p = p;
  a.Ap = Ap;
  a.pAp = pAp;
  a.act = act;
  a.need = need;
  a.partials = partials;
  a.counter = counters;
  Sweep sw{};
  sw.nblocks = nblocks;
  return launch_t<4, 4, false, false, false, false, true>(a, sw, s);
}

cudaError_t launch_batch_cond(const CgState* st, int ninst, unsigned long long cond,
                              long long* sweeps, long long limit, cudaStream_t s) {
  batch_cond_kernel<<<1, 128, 0, s>>>(st, ninst, cond, sweeps, limit);
  return cudaGetLastError();
}

cudaError_t launch_cg_sweep(const Grid& g, const Sweep& sw, const void* coef, bool b16,
                            CgVecs v, CgState* st, double* partials, unsigned int* counter,
                            unsigned long long cond, int use_cond, cudaStream_t s) {
  SweepArgs a = sweep_args_rec(g, sw, coef, b16);
  a.v = v;
  a.st = st;
  a.partials = partials;
  a.counter = counter;
  a.cond = cond;
  return launch_sweep(a, sw, true, use_cond != 0, s);
}

template <int VY, int S>
static int blocks_per_sm_t() {
  constexpr int smem = sweep_smem_bytes<VY, S, false>();
  if (cudaFuncSetAttribute(sweep_kernel<VY, S, true, true, false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<VY, S, true, true, false>,
                                                    kSweepWarps * 32, smem) != cudaSuccess)
    return 0;
  return nb;
}

int sweep_blocks_per_sm(int vy, int stages) {
  int nb = 0;
  if (vy == 4 && stages == 3) nb = blocks_per_sm_t<4, 3>();
  else if (vy == 4 && stages == 4) nb = blocks_per_sm_t<4, 4>();
  else if (vy == 8 && stages == 3) nb = blocks_per_sm_t<8, 3>();
  if (nb == 0) cudaGetLastError();
  return nb;
}

cudaError_t launch_residual64(const Grid& g, const double* coef64, const double* b,
                              const double* x, double* r, double* norms, CgState* st,
                              double* partials, unsigned int* counter, int nblocks,
                              cudaStream_t s) {
  residual64_kernel<<<nblocks, kElemThreads, 0, s>>>(g, reinterpret_cast<const double2*>(coef64),
                                                      b, x, r, norms, st, partials, counter);
  return cudaGetLastError();
}

cudaError_t launch_prepare(const Grid& g, const double* r64, CgVecs v, CgState* st, double rtol,
                           long long maxit, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  prepare_kernel<<<elem_blocks(g, sms), kElemThreads, 0, s>>>(g, r64, v, st, rtol * rtol, maxit);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const Grid& g, CgVecs v, CgState* st, double* partials,
                            unsigned int* counter, int nblocks, const float4* jac,
                            const float* dinv, cudaStream_t s) {
  finalize_kernel<<<nblocks, kElemThreads, 0, s>>>(g, v, st, partials, counter, jac, dinv);
  return cudaGetLastError();
}

cudaError_t launch_correct(const Grid& g, const CgVecs& v, double* x, const CgState* st,
                           cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  correct_kernel<<<elem_blocks(g, sms), kElemThreads, 0, s>>>(g, v, x, st);
  return cudaGetLastError();
}

}  // namespace tpfa
