// Lattice constants and index helpers of the CUDA path.
//
// D3Q19 velocities are the columns of the matrix M of Sec. 2.1 (rest vector
// last), weights from Eq. d3q19_weight_function (c_s^2 = 1/3).  D3Q7 for the
// dissolved reactant (an addition of this library): +x, -x, +y, -y, +z, -z,
// rest, weights 1/8 and 1/4, c_s^2 = 1/4.
#pragma once
#include <cstdint>

namespace cglbm {

constexpr int Q = 19;
constexpr int Q7 = 7;
constexpr int NPOP = 2 * Q + Q7;   // f^r[19], f^p[19], g[7]

__device__ constexpr int CX[Q] = {1, -1, 0, 0, 0, 0, 1, 1, 1, 1, -1, -1, -1, -1, 0, 0, 0, 0, 0};
__device__ constexpr int CY[Q] = {0, 0, 1, -1, 0, 0, 1, -1, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0};
__device__ constexpr int CZ[Q] = {0, 0, 0, 0, 1, -1, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, 1, -1, 0};
__device__ constexpr int OPP[Q] = {1, 0, 3, 2, 5, 4, 11, 10, 13, 12, 7, 6, 9, 8, 17, 16, 15, 14, 18};
constexpr float W1 = 1.0f / 18.0f;
constexpr float W2 = 1.0f / 36.0f;
constexpr float W0 = 1.0f / 3.0f;
__device__ constexpr float W[Q] = {W1, W1, W1, W1, W1, W1, W2, W2, W2, W2, W2, W2,
                        W2, W2, W2, W2, W2, W2, W0};
// 1/|c_i| for the recolouring cosine, 0 for the rest vector
constexpr float RSQRT2 = 0.70710678118654752f;
__device__ constexpr float INVNORM[Q] = {1, 1, 1, 1, 1, 1, RSQRT2, RSQRT2, RSQRT2, RSQRT2, RSQRT2, RSQRT2,
                              RSQRT2, RSQRT2, RSQRT2, RSQRT2, RSQRT2, RSQRT2, 0};
// D3Q7 shares the first six D3Q19 directions and the rest vector
__device__ constexpr int GDIR[Q7] = {0, 1, 2, 3, 4, 5, 18};
__device__ constexpr int GOPP[Q7] = {1, 0, 3, 2, 5, 4, 6};
__device__ constexpr float W7[Q7] = {0.125f, 0.125f, 0.125f, 0.125f, 0.125f, 0.125f, 0.25f};

// per-node static bits (uint32 "link" word)
constexpr uint32_t BIT_SOLID = 1u << 19;      // s(x) = 1
constexpr uint32_t BIT_WALL = 1u << 20;       // fluid node with a solid D3Q19 neighbour
constexpr uint32_t BIT_REACTIVE = 1u << 21;   // r(x) = 1
constexpr uint32_t BIT_SOLID_BND = 1u << 22;  // solid node with a fluid D3Q19 neighbour
constexpr uint32_t BIT_NS_OK = 1u << 23;      // solid normal defined
constexpr int NN_SHIFT = 24;                  // NN(x) in bits 24..26
constexpr uint32_t LINK_MASK = (1u << 19) - 1;  // bit i: x - c_i is solid (bounce back)

constexpr float GRAD_EPS = 1e-5f;   // |grad rho^N| below this: n = 0, H = 0 (above FP32 noise)
constexpr float SIN2_EPS = 1e-6f;   // sin^2(theta') below this: no wetting rotation

struct Lattice {
  int nx, ny, nz, bc_z;
  long long n;        // nx * ny * nz
  long long plane;    // nx * ny
  long long pstride;  // plane * (nz + 2): one population of one buffer (with ghost planes)
};

// population p at stored plane zp (z + 1; 0 and nz + 1 are the column ghosts)
__device__ __forceinline__ long long pidx(const Lattice &L, int p, int zp, int y, int x) {
  return (long long)p * L.pstride + (long long)zp * L.plane + (long long)y * L.nx + x;
}

__device__ __forceinline__ long long nidx(const Lattice &L, int x, int y, int z) {
  return ((long long)z * L.ny + y) * L.nx + x;
}

// coordinates x + d for d = -1, 0, +1 (index d + 1); x and y periodic; z periodic
// or clamped into [0, nz - 1] (column mode: zero-gradient stencil extension)
struct Stencil {
  int xs[3], ys[3], zs[3];
  __device__ __forceinline__ void init(const Lattice &L, int x, int y, int z) {
    xs[0] = x > 0 ? x - 1 : L.nx - 1;
    xs[1] = x;
    xs[2] = x + 1 < L.nx ? x + 1 : 0;
    ys[0] = y > 0 ? y - 1 : L.ny - 1;
    ys[1] = y;
    ys[2] = y + 1 < L.ny ? y + 1 : 0;
    zs[1] = z;
    if (L.bc_z == 0) {
      zs[0] = z > 0 ? z - 1 : L.nz - 1;
      zs[2] = z + 1 < L.nz ? z + 1 : 0;
    } else {
      zs[0] = z > 0 ? z - 1 : 0;
      zs[2] = z + 1 < L.nz ? z + 1 : L.nz - 1;
    }
  }
  // node index of x + c_i
  __device__ __forceinline__ long long nb(const Lattice &L, int cx, int cy, int cz) const {
    return ((long long)zs[cz + 1] * L.ny + ys[cy + 1]) * L.nx + xs[cx + 1];
  }
};

// 32-bit offsets (within one population array) of the pull sources x - c:
// own offset + dx[1 - cx] + dy[1 - cy] + dz[1 - cz].  x and y periodic; z
// periodic or (column mode) the ghost planes 0 / nz + 1.  One population array
// of one buffer holds pstride < 2^32 / 45 floats (checked at create).
struct PullOffsets {
  unsigned own;
  int dx[3], dy[3], dz[3];
  __device__ __forceinline__ void init(const Lattice &L, int x, int y, int z) {
    const int plane = (int)L.plane;
    own = (unsigned)((z + 1) * plane + y * L.nx + x);
    dx[1] = dy[1] = dz[1] = 0;
    dx[0] = x > 0 ? -1 : L.nx - 1;            // x - 1
    dx[2] = x + 1 < L.nx ? 1 : 1 - L.nx;      // x + 1
    dy[0] = y > 0 ? -L.nx : (L.ny - 1) * L.nx;
    dy[2] = y + 1 < L.ny ? L.nx : (1 - L.ny) * L.nx;
    if (L.bc_z == 0) {
      dz[0] = z > 0 ? -plane : (L.nz - 1) * plane;
      dz[2] = z + 1 < L.nz ? plane : (1 - L.nz) * plane;
    } else {
      dz[0] = -plane;   // plane 0 is the inlet ghost when z = 0
      dz[2] = plane;    // plane nz + 1 is the outlet ghost when z = nz - 1
    }
  }
  // offset of the pull source of velocity (cx, cy, cz)
  __device__ __forceinline__ unsigned src(int cx, int cy, int cz) const {
    return own + (unsigned)(dx[1 - cx] + dy[1 - cy] + dz[1 - cz]);
  }
};

// 32-bit node-index offsets of the stencil neighbours x + c (periodic x, y; z
// periodic or clamped), for fields indexed by node: own + dx[cx+1] + dy[cy+1] + dz[cz+1]
struct StencilOffsets {
  unsigned own;
  int dx[3], dy[3], dz[3];
  __device__ __forceinline__ void init(const Lattice &L, int x, int y, int z) {
    const int plane = (int)L.plane;
    own = (unsigned)(z * plane + y * L.nx + x);
    dx[1] = dy[1] = dz[1] = 0;
    dx[0] = x > 0 ? -1 : L.nx - 1;
    dx[2] = x + 1 < L.nx ? 1 : 1 - L.nx;
    dy[0] = y > 0 ? -L.nx : (L.ny - 1) * L.nx;
    dy[2] = y + 1 < L.ny ? L.nx : (1 - L.ny) * L.nx;
    if (L.bc_z == 0) {
      dz[0] = z > 0 ? -plane : (L.nz - 1) * plane;
      dz[2] = z + 1 < L.nz ? plane : (1 - L.nz) * plane;
    } else {
      dz[0] = z > 0 ? -plane : 0;
      dz[2] = z + 1 < L.nz ? plane : 0;
    }
  }
  __device__ __forceinline__ unsigned nb(int cx, int cy, int cz) const {
    return own + (unsigned)(dx[cx + 1] + dy[cy + 1] + dz[cz + 1]);
  }
};

// stored-plane index of the pull source z - cz: periodic wrap, or the ghost
// planes 0 / nz + 1 in column mode
__device__ __forceinline__ void pull_planes(const Lattice &L, int z, int zp_src[3]) {
  // zp_src[k] is the stored plane of z + (k - 1)
  zp_src[1] = z + 1;
  if (L.bc_z == 0) {
    zp_src[0] = (z > 0 ? z - 1 : L.nz - 1) + 1;
    zp_src[2] = (z + 1 < L.nz ? z + 1 : 0) + 1;
  } else {
    zp_src[0] = z;       // z - 1 + 1 (0 = inlet ghost when z = 0)
    zp_src[2] = z + 2;   // z + 1 + 1 (nz + 1 = outlet ghost when z = nz - 1)
  }
}

}  // namespace cglbm
