// Internal declarations of the learned-preconditioner kernels (3D U-Net on
// BF16 channels-last volumes).
//
// Volume layout ("haloed channels-last"): ns samples of nz x ny x nx cells,
// each sample surrounded by a one-cell zero halo, channels innermost:
//   element (s, z, y, x, c) at  (((s*(nz+2) + z+1)*(ny+2) + y+1)*(nx+2) + x+1)*C + c.
// The halo is zeroed when the buffer is created and no kernel writes it, so
// a 3x3x3 tap of a border cell reads zero (zero padding) and the samples of
// a batch never see each other.  Every 3x3x3 tap is then a constant offset
// in the flat voxel index:  off(dz, dy, dx) = dz*P + dy*W + dx  with
// W = nx+2, P = (nx+2)(ny+2).  Tap index t = 9(dz+1) + 3(dy+1) + (dx+1).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tpfa {
namespace net {

struct Vol {
  int nx, ny, nz, ns;
  int wp, hp, dp;  // padded extents
  int pp;          // padded plane (voxels)
  int sp;          // padded sample (voxels)
  int vp;          // all samples (voxels)
  int g0, g1;      // [first interior voxel, last interior voxel + 1)
};

inline Vol make_vol(int nx, int ny, int nz, int ns) {
  Vol v;
  v.nx = nx; v.ny = ny; v.nz = nz; v.ns = ns;
  v.wp = nx + 2; v.hp = ny + 2; v.dp = nz + 2;
  v.pp = v.wp * v.hp;
  v.sp = v.pp * v.dp;
  v.vp = v.sp * ns;
  v.g0 = v.pp + v.wp + 1;
  v.g1 = (ns - 1) * v.sp + nz * v.pp + ny * v.wp + nx + 1;
  return v;
}

// true when the extents give a layout whose voxel indices fit in int
bool vol_ok(int nx, int ny, int nz, int ns);

__device__ __forceinline__ bool vol_interior(const Vol& g, int idx) {
  if (idx < g.g0 || idx >= g.g1) return false;
  const int x = idx % g.wp;
  const int t = idx / g.wp;
  const int y = t % g.hp;
  const int z = (t / g.hp) % g.dp;
  return x >= 1 && x <= g.nx && y >= 1 && y <= g.ny && z >= 1 && z <= g.nz;
}

enum ConvFlags : int { kConvRelu = 1, kConvMask = 2 };

// y = epilogue(conv3x3x3(x; w) + bias): see tpfa_conv3d_bf16.
cudaError_t conv_fwd(const uint16_t* x, const uint16_t* w, const float* bias, const uint16_t* mask,
                     uint16_t* y, const Vol& g, int cin, int cout, int flags, cudaStream_t s);
// workspace bytes conv_wgrad needs for this shape
size_t conv_wgrad_ws_bytes(const Vol& g, int cin, int cout);
// dw[t][co][ci] (+)= sum_v dy[v][co] x[v + off_t][ci]
cudaError_t conv_wgrad(const uint16_t* x, const uint16_t* dy, float* dw, float* ws,
                       const Vol& g, int cin, int cout, int accumulate, cudaStream_t s);
bool conv_shape_ok(int cin, int cout);

}  // namespace net
}  // namespace tpfa
