// Host-side tiling of the cp.async-staged stencil sweeps (plain C++, no CUDA
// dependency, so that the planning rules can be checked on a machine without
// a GPU).
#pragma once

#include <stdint.h>

namespace tpfa {

constexpr int kTileX = 30;       // output columns per warp (lanes 1..30; lanes 0, 31 are halo)
constexpr int kSweepWarps = 4;   // warps per block in the stencil sweeps
// reduction workspace of tpfa_apply_noalloc: one partial sum per block
constexpr int kNoAllocMaxBlocks = 16384;

struct Grid {
  int64_t nx, ny, nz;
  int64_t plane;  // nx * ny
  int64_t n;      // nx * ny * nz
};

// Warp tiling of the z-marching stencil sweeps.
struct Sweep {
  int vy;           // rows per warp (4 or 8)
  int stages;       // shared-memory plane stages per warp
  int warps;        // warps per block
  int zc;           // planes per warp
  int64_t nwx, nwy, nwz;
  int64_t nwarps;
  int64_t nblocks;  // blocks of `warps` warps
};

// zc_opt > 0 fixes the z-run length; zc_opt <= 0 picks the longest run (at
// most 128 planes; each run re-reads two halo planes) that still gives about
// four warps per SM: on 128^3 and 256^3 grids the sweep is 20% faster with
// these runs (32 and 128 planes) than with the shorter ones that would give
// several waves of resident warps.
inline Sweep plan_sweep(const Grid& g, int vy, int stages, int zc_opt, int num_sms) {
  Sweep s;
  s.vy = vy;
  s.stages = stages;
  s.warps = kSweepWarps;
  s.nwx = (g.nx + kTileX - 1) / kTileX;
  s.nwy = (g.ny + vy - 1) / vy;
  int zc = zc_opt;
  if (zc <= 0) {
    const int64_t target = (int64_t)num_sms * 4;
    const int64_t cols = s.nwx * s.nwy;
    zc = 128;
    while (zc > 1 && cols * ((g.nz + zc - 1) / zc) < target) zc /= 2;
  }
  if (zc > g.nz) zc = (int)g.nz;
  s.zc = zc;
  s.nwz = (g.nz + zc - 1) / zc;
  s.nwarps = s.nwx * s.nwy * s.nwz;
  s.nblocks = (s.nwarps + kSweepWarps - 1) / kSweepWarps;
  return s;
}

// Tiling of tpfa_apply_noalloc: tpfa_apply's, with z-runs doubled (up to the
// whole column) until the block count fits the fixed workspace.  Returns
// false for grids whose single-run tiling still needs more blocks.
inline bool plan_noalloc(const Grid& g, int num_sms, Sweep* out) {
  Sweep sw = plan_sweep(g, 4, 4, 0, num_sms);
  while (sw.nblocks > kNoAllocMaxBlocks && sw.zc < g.nz)
    sw = plan_sweep(g, 4, 4, (int)(2 * (int64_t)sw.zc < g.nz ? 2 * sw.zc : g.nz), num_sms);
  *out = sw;
  return sw.nblocks <= kNoAllocMaxBlocks;
}

}  // namespace tpfa
