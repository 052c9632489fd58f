// CUDA kernels of one colour-gradient LB time step (sm_103a, FP32 storage and
// arithmetic, FP64 reductions).
//
// Per step, in order (one launch each):
//   k_density       pull rho^r, rho^p -> colour function rho^N       (Eq. color_function)
//   k_color_solid   rho^N at solid nodes next to the fluid           (Eq. color_lattice_weighted_average)
//   k_normal        gradient, n = +grad/|grad|, wetting              (Eq. finite_difference_scheme,
//                                                                     Eq. realigned_normal_vectors)
//   k_normal_solid  n at solid nodes next to the fluid (weighted average of fluid n, renormalised)
//   k_main          pull all 45 populations, curvature, CSF/EDM force, central-moment collision,
//                   recolouring, reaction, D3Q7 transport; store; outlet ghost; FP64 sum of delta
// plus k_geom (once), k_init, k_ghost_init and k_observables.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "lattice.cuh"

namespace cglbm {

struct StepParams {
  float omega_cm;     // 1 - 1/tau (Eq. post_collision_moments)
  float half_sigma;   // sigma / 2 (Eq. continuum_surface_force)
  float beta;
  float ax, ay, az;
  float inv_tau_g;    // 1 / (D / c_s^2 + 1/2), c_s^2 = 1/4 on D3Q7
  float k_rate, xi, rho_out;
  int reaction_mode;  // 0: C-mode reaction + D3Q7 transport; 1: paper mode
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
// c_i . (a, b, c) with only the nonzero components of c_i (+-1) entering: a product
// with a zero component cannot be folded away (0 * x is not 0 for every x), so the
// hot loops spell the sum out per direction.
__device__ __forceinline__ float cdot(int i, float a, float b, float c) {
  float s = 0.f;
  bool any = false;
  if (CX[i]) {
    s = CX[i] > 0 ? a : -a;
    any = true;
  }
  if (CY[i]) {
    s = any ? (CY[i] > 0 ? s + b : s - b) : (CY[i] > 0 ? b : -b);
    any = true;
  }
  if (CZ[i]) s = any ? (CZ[i] > 0 ? s + c : s - c) : (CZ[i] > 0 ? c : -c);
  return s;
}

__device__ __forceinline__ float feq19(int i, float rho, float vx, float vy, float vz, float vv) {
  const float cu = CX[i] * vx + CY[i] * vy + CZ[i] * vz;
  return W[i] * rho * (1.0f + 3.0f * cu + 4.5f * cu * cu - 1.5f * vv);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum of NV doubles into global accumulators (one atomic per value per block)
template <int NV>
__device__ __forceinline__ void block_accumulate(double (&v)[NV], double *acc) {
  __shared__ double red[32][NV];
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthreads = blockDim.x * blockDim.y * blockDim.z;
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) red[warp][k] = v[k];
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = (nthreads + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = lane < nw ? red[lane][k] : 0.0;
      s = warp_sum(s);
      if (lane == 0 && s != 0.0) atomicAdd(acc + k, s);
    }
  }
}

// Closed-form T^{-1} k* of Appendix A, Eq. back_transformation_vector, one row
// per population; rows 6..17 share one pattern per coordinate plane.
__device__ __forceinline__ void back_transform(float ux, float uy, float uz, float k5, float k6,
                                               float k7, float k8, float k9, float (&bt)[Q]) {
  const float ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
  {  // rows 0, 1: c = (+-1, 0, 0)
    const float A = ux2 - uy2 - uz2 + 1.0f;
    const float P = k5 * (1.0f / 3.0f) + k6 * (1.0f / 6.0f);
    const float R = uy * k7 + uz * k8;
    bt[0] = (A + ux) * P - (2.0f * ux + 1.0f) * R;
    bt[1] = (A - ux) * P - (2.0f * ux - 1.0f) * R;
  }
  {  // rows 2, 3: c = (0, +-1, 0)
    const float B = ux2 - uy2 + uz2 - 1.0f;
    const float P = (k5 - k6) * (1.0f / 6.0f);
    const float R = ux * k7 + uz * k9;
    bt[2] = (B - uy) * P - (2.0f * uy + 1.0f) * R;
    bt[3] = (B + uy) * P - (2.0f * uy - 1.0f) * R;
  }
  {  // rows 4, 5: c = (0, 0, +-1)
    const float Cc = ux2 + uy2 - uz2 - 1.0f;
    const float P = k5 * (1.0f / 6.0f) + k6 * (1.0f / 3.0f);
    const float R = ux * k8 + uy * k9;
    bt[4] = (Cc - uz) * P - (2.0f * uz + 1.0f) * R;
    bt[5] = (Cc + uz) * P - (2.0f * uz - 1.0f) * R;
  }
  constexpr float T12 = 1.0f / 12.0f;
  // rows c = (a, b, 0): 6 (1,1), 7 (1,-1), 10 (-1,1), 11 (-1,-1)
  {
    const float uxuy12 = 12.0f * ux * uy;
    const int ia[4] = {6, 7, 10, 11};
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int i = ia[m];
      const float a = (float)CX[i], b = (float)CY[i];
      const float c5 = -ux2 - a * ux + 2.0f * uy2 + 2.0f * b * uy;
      const float c6 = ux2 + a * ux + uy2 + b * uy;
      const float c7 = uxuy12 + 6.0f * b * ux + 6.0f * a * uy + 3.0f * a * b;
      bt[i] = (c5 * k5 + c6 * k6 + c7 * k7) * T12;
    }
  }
  // rows c = (a, 0, b): 8 (1,1), 9 (1,-1), 12 (-1,1), 13 (-1,-1)
  {
    const float uxuz12 = 12.0f * ux * uz;
    const int ia[4] = {8, 9, 12, 13};
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int i = ia[m];
      const float a = (float)CX[i], b = (float)CZ[i];
      const float c5 = -ux2 - a * ux + 2.0f * uz2 + 2.0f * b * uz;
      const float c6 = -2.0f * ux2 - 2.0f * a * ux + uz2 + b * uz;
      const float c8 = uxuz12 + 6.0f * b * ux + 6.0f * a * uz + 3.0f * a * b;
      bt[i] = (c5 * k5 + c6 * k6 + c8 * k8) * T12;
    }
  }
  // rows c = (0, a, b): 14 (1,1), 15 (1,-1), 16 (-1,1), 17 (-1,-1)
  {
    const float uyuz12 = 12.0f * uy * uz;
    const int ia[4] = {14, 15, 16, 17};
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int i = ia[m];
      const float a = (float)CY[i], b = (float)CZ[i];
      const float c5 = -uy2 - a * uy - uz2 - b * uz;
      const float c6 = -2.0f * uy2 - 2.0f * a * uy + uz2 + b * uz;
      const float c9 = uyuz12 + 6.0f * b * uy + 6.0f * a * uz + 3.0f * a * b;
      bt[i] = (c5 * k5 + c6 * k6 + c9 * k9) * T12;
    }
  }
  bt[18] = (-2.0f * ux2 + uy2 + uz2) * k5 * (1.0f / 3.0f) + (-ux2 - uy2 + 2.0f * uz2) * k6 * (1.0f / 3.0f) +
           4.0f * (ux * uy * k7 + ux * uz * k8 + uy * uz * k9);
}

// Outlet ghost plane (column mode) from the post-collision populations of a
// fluid node of plane nz - 1: non-equilibrium extrapolation to rho_out, split
// by the node's colour ratio; g copied.  Writes the populations with c_z = -1.
__device__ __forceinline__ void write_outlet_ghost(const Lattice &L, float *__restrict__ f, int x, int y,
                                                   const float (&fr)[Q], const float (&fp)[Q],
                                                   float g5, float rho_out) {
  float rho = 0.f, rr = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float m = fr[i] + fp[i];
    rho += m;
    rr += fr[i];
    jx += CX[i] * m;
    jy += CY[i] * m;
    jz += CZ[i] * m;
  }
  const float inv = 1.0f / rho;
  const float vx = jx * inv, vy = jy * inv, vz = jz * inv;
  const float vv = vx * vx + vy * vy + vz * vz;
  const float psi = rr * inv;
  const int zp = L.nz + 1;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (CZ[i] != -1) continue;
    const float corr = feq19(i, rho_out - rho, vx, vy, vz, vv);
    f[pidx(L, i, zp, y, x)] = fr[i] + psi * corr;
    f[pidx(L, Q + i, zp, y, x)] = fp[i] + (1.0f - psi) * corr;
  }
  f[pidx(L, 2 * Q + 5, zp, y, x)] = g5;
}

// ---------------------------------------------------------------------------
// one-time geometry: link bits, NN, r, wall / boundary flags, solid normal
// ---------------------------------------------------------------------------
__device__ __forceinline__ float omega8(int e2) {
  // Eq. eigth_order_weight_function
  switch (e2) {
    case 1: return 4.0f / 45.0f;
    case 2: return 1.0f / 21.0f;
    case 3: return 2.0f / 105.0f;
    case 4: return 5.0f / 504.0f;
    case 5: return 1.0f / 315.0f;
    case 6: return 1.0f / 630.0f;
    case 8: return 1.0f / 5040.0f;
    default: return 0.0f;
  }
}

__device__ __forceinline__ bool solid_at(const Lattice &L, const uint8_t *__restrict__ solid, int x, int y,
                                         int z) {
  x = ((x % L.nx) + L.nx) % L.nx;
  y = ((y % L.ny) + L.ny) % L.ny;
  if (L.bc_z == 0)
    z = ((z % L.nz) + L.nz) % L.nz;
  else
    z = z < 0 ? 0 : (z >= L.nz ? L.nz - 1 : z);
  return solid[nidx(L, x, y, z)] != 0;
}

// ns[node].w of a wall node holds its contact angle theta in radians: the
// uniform value theta_rad, or the D3Q19-weighted mean of a per-solid-node field
// (k_wall_theta).  k_geom writes the uniform value.
// It runs in blocks of kGeomBX x kGeomBY nodes of one z-plane (node_block()): the block
// first stages the mask of its nodes and of everything within kGeomH nodes of them (the
// reach of the solid-normal stencil) in shared memory, with solid_at's periodic and
// clamped-ghost rules applied once per staged byte, so the 18- and 92-point stencils
// below read shared memory only.
constexpr int kGeomBX = 32, kGeomBY = 4, kGeomH = 2;
constexpr int kGeomTX = kGeomBX + 2 * kGeomH, kGeomTY = kGeomBY + 2 * kGeomH, kGeomTZ = 1 + 2 * kGeomH;

__global__ void __launch_bounds__(kGeomBX * kGeomBY) k_geom(Lattice L, const uint8_t *__restrict__ solid,
                                                            const uint8_t *__restrict__ reactive, float theta_rad,
                                                            uint32_t *__restrict__ link, float4 *__restrict__ ns) {
  __shared__ uint8_t tile[kGeomTZ][kGeomTY][kGeomTX];
  const int x0 = blockIdx.x * kGeomBX, y0 = blockIdx.y * kGeomBY, z = blockIdx.z;
  for (int q = threadIdx.y * kGeomBX + threadIdx.x; q < kGeomTZ * kGeomTY * kGeomTX; q += kGeomBX * kGeomBY) {
    const int tx = q % kGeomTX, ty = (q / kGeomTX) % kGeomTY, tz = q / (kGeomTX * kGeomTY);
    (&tile[0][0][0])[q] = solid_at(L, solid, x0 + tx - kGeomH, y0 + ty - kGeomH, z + tz - kGeomH) ? 1 : 0;
  }
  __syncthreads();
  const int x = x0 + (int)threadIdx.x;
  const int y = y0 + (int)threadIdx.y;
  if (x >= L.nx || y >= L.ny) return;
  // the mask at (x + dx, y + dy, z + dz), |d| <= kGeomH, by solid_at's rules
  auto sol = [&](int dx, int dy, int dz) {
    return tile[dz + kGeomH][(int)threadIdx.y + dy + kGeomH][(int)threadIdx.x + dx + kGeomH] != 0;
  };
  const long long node = nidx(L, x, y, z);
  uint32_t bits = 0;
  float4 nsv = make_float4(0.f, 0.f, 0.f, 0.f);
  if (solid[node]) {
    // solid node: bit i set if x + c_i is fluid (stencil rules), used by the
    // solid-colour and solid-normal averages
    bits = BIT_SOLID;
    for (int i = 0; i < Q - 1; ++i)
      if (!sol(CX[i], CY[i], CZ[i])) bits |= BIT_SOLID_BND | (1u << i);
  } else {
    // bounce-back links: the pull source x - c_i is solid (column ghosts are fluid)
    for (int i = 0; i < Q - 1; ++i) {
      const int sz = z - CZ[i];
      if (L.bc_z == 1 && (sz < 0 || sz >= L.nz)) continue;
      if (sol(-CX[i], -CY[i], -CZ[i])) bits |= 1u << i;
    }
    bool wall = false;
    for (int i = 0; i < Q - 1; ++i) wall |= sol(CX[i], CY[i], CZ[i]);
    // Eq. nearest_solid_neighbors
    int nn = 0;
    for (int i = 0; i < 6; ++i) nn += sol(CX[i], CY[i], CZ[i]) ? 1 : 0;
    bits |= (uint32_t)nn << NN_SHIFT;
    const bool r = reactive ? (reactive[node] != 0) : (nn >= 1);
    if (r) bits |= BIT_REACTIVE;
    if (wall) {
      bits |= BIT_WALL;
      // Eq. normal_vector_solid over the 92 vectors with |e|^2 in {1,..,6,8}
      float sx = 0.f, sy = 0.f, sz = 0.f;
      for (int ez = -2; ez <= 2; ++ez)
        for (int ey = -2; ey <= 2; ++ey)
          for (int ex = -2; ex <= 2; ++ex) {
            const float w = omega8(ex * ex + ey * ey + ez * ez);
            if (w == 0.f) continue;
            if (sol(ex, ey, ez)) {
              sx += w * ex;
              sy += w * ey;
              sz += w * ez;
            }
          }
      const float m = sqrtf(sx * sx + sy * sy + sz * sz);
      if (m > 0.f) {
        bits |= BIT_NS_OK;
        nsv = make_float4(sx / m, sy / m, sz / m, theta_rad);
      }
    }
  }
  link[node] = bits;
  ns[node] = nsv;
}

// Contact angle of every wall node from a per-node field theta_deg (degrees, read
// at solid nodes): the D3Q19-weighted mean over the solid neighbours x + c_i of
// the geometry stencil (a spatially varying wettability; the paper's is uniform).
// theta_deg null: the uniform value theta_rad.
__global__ void k_wall_theta(Lattice L, const uint32_t *__restrict__ link, const float *__restrict__ theta_deg,
                             float theta_rad, float4 *__restrict__ ns) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= L.nx || y >= L.ny) return;
  const long long node = nidx(L, x, y, z);
  const uint32_t lk = link[node];
  if ((lk & BIT_SOLID) || !(lk & BIT_WALL) || !(lk & BIT_NS_OK)) return;
  float th = theta_rad;
  if (theta_deg) {
    float num = 0.f, den = 0.f;
    for (int i = 0; i < Q - 1; ++i) {
      const int xx = ((x + CX[i]) % L.nx + L.nx) % L.nx, yy = ((y + CY[i]) % L.ny + L.ny) % L.ny;
      int zz = z + CZ[i];
      zz = L.bc_z == 0 ? (zz + L.nz) % L.nz : (zz < 0 ? 0 : (zz >= L.nz ? L.nz - 1 : zz));
      const long long nb = nidx(L, xx, yy, zz);
      if (link[nb] & BIT_SOLID) {
        num += W[i] * theta_deg[nb];
        den += W[i];
      }
    }
    th = num / den * 0.017453292519943295f;
  }
  ns[node].w = th;
}

// ---------------------------------------------------------------------------
// start state
// ---------------------------------------------------------------------------
// f^k = f^eq(rho^k, u), g = g^eq(C, u); fields may be null (uniform defaults)
__global__ void k_init(Lattice L, const uint32_t *__restrict__ link, const float *__restrict__ rho_r,
                       const float *__restrict__ rho_p, const float *__restrict__ conc,
                       const float *__restrict__ u, float rr0, float rp0, float c0, float *__restrict__ fa,
                       float *__restrict__ fb) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= L.nx || y >= L.ny) return;
  const long long node = nidx(L, x, y, z);
  const bool fluid = !(link[node] & BIT_SOLID);
  const float rr = fluid ? (rho_r ? rho_r[node] : rr0) : 0.f;
  const float rp = fluid ? (rho_p ? rho_p[node] : rp0) : 0.f;
  const float cc = fluid ? (conc ? conc[node] : c0) : 0.f;
  const float ux = (fluid && u) ? u[node] : 0.f;
  const float uy = (fluid && u) ? u[L.n + node] : 0.f;
  const float uz = (fluid && u) ? u[2 * L.n + node] : 0.f;
  const float uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float a = feq19(i, rr, ux, uy, uz, uu), b = feq19(i, rp, ux, uy, uz, uu);
    fa[pidx(L, i, z + 1, y, x)] = a;
    fb[pidx(L, i, z + 1, y, x)] = a;
    fa[pidx(L, Q + i, z + 1, y, x)] = b;
    fb[pidx(L, Q + i, z + 1, y, x)] = b;
  }
#pragma unroll
  for (int j = 0; j < Q7; ++j) {
    const int d = GDIR[j];
    const float gv = W7[j] * cc * (1.0f + 4.0f * (CX[d] * ux + CY[d] * uy + CZ[d] * uz));
    fa[pidx(L, 2 * Q + j, z + 1, y, x)] = gv;
    fb[pidx(L, 2 * Q + j, z + 1, y, x)] = gv;
  }
}

// Column ghost planes of both buffers: constant inlet (z = -1): f^r = f^eq(1, u_in z),
// f^p = 0, g = g^eq(c_in, u_in z); outlet (z = nz) from plane nz - 1 of buffer fa
// (the current state), resting reactant equilibrium above solid nodes.
__global__ void k_ghost_init(Lattice L, const uint32_t *__restrict__ link, float u_in, float c_in,
                             float rho_out, float *__restrict__ fa, float *__restrict__ fb) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= L.nx || y >= L.ny) return;
  const float uu = u_in * u_in;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (CZ[i] != 1) continue;
    const float v = feq19(i, 1.0f, 0.f, 0.f, u_in, uu);
    fa[pidx(L, i, 0, y, x)] = v;
    fb[pidx(L, i, 0, y, x)] = v;
    fa[pidx(L, Q + i, 0, y, x)] = 0.f;
    fb[pidx(L, Q + i, 0, y, x)] = 0.f;
  }
  const float g4 = W7[4] * c_in * (1.0f + 4.0f * u_in);
  fa[pidx(L, 2 * Q + 4, 0, y, x)] = g4;
  fb[pidx(L, 2 * Q + 4, 0, y, x)] = g4;
  const int z = L.nz - 1;
  const long long node = nidx(L, x, y, z);
  if (link[node] & BIT_SOLID) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (CZ[i] != -1) continue;
      const float v = W[i] * rho_out;
      fa[pidx(L, i, L.nz + 1, y, x)] = v;
      fb[pidx(L, i, L.nz + 1, y, x)] = v;
      fa[pidx(L, Q + i, L.nz + 1, y, x)] = 0.f;
      fb[pidx(L, Q + i, L.nz + 1, y, x)] = 0.f;
    }
    fa[pidx(L, 2 * Q + 5, L.nz + 1, y, x)] = 0.f;
    fb[pidx(L, 2 * Q + 5, L.nz + 1, y, x)] = 0.f;
  } else {
    float fr[Q], fp[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      fr[i] = fa[pidx(L, i, z + 1, y, x)];
      fp[i] = fa[pidx(L, Q + i, z + 1, y, x)];
    }
    write_outlet_ghost(L, fa, x, y, fr, fp, fa[pidx(L, 2 * Q + 5, z + 1, y, x)], rho_out);
  }
}

// ---------------------------------------------------------------------------
// a1 + a2: colour function from the pulled populations
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_density(Lattice L, const float *__restrict__ f,
                                                 const uint32_t *__restrict__ link, float *__restrict__ rhoN) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  const bool inside = x < L.nx && y < L.ny;
  const unsigned node = inside ? (unsigned)nidx(L, x, y, z) : 0u;
  const uint32_t lk = inside ? link[node] : BIT_SOLID;
  const bool fluid = !(lk & BIT_SOLID);
  // a warp with any fluid node writes every node of its row segment (solid: 0)
  // so that the stores cover whole sectors
  if (!__any_sync(0xffffffffu, fluid) || !inside) return;
  if (!fluid) {
    rhoN[node] = 0.f;
    return;
  }
  PullOffsets O;
  O.init(L, x, y, z);
  const unsigned ps = (unsigned)L.pstride;
  float rr = 0.f, rp = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    // halfway bounce-back: f_i(x) = f*_opp(i)(x) when x - c_i is solid
    const bool bb = (lk >> i) & 1u;
    const unsigned off = bb ? O.own : O.src(CX[i], CY[i], CZ[i]);
    const unsigned pr = bb ? (unsigned)OPP[i] : (unsigned)i;
    rr += f[pr * ps + off];
    rp += f[(pr + Q) * ps + off];
  }
  rhoN[node] = (rr - rp) / (rr + rp);
}

// a3: Eq. color_lattice_weighted_average at solid nodes next to the fluid.
// list holds packed x | y << 10 | z << 20; a solid node's link word marks in
// bit i whether x + c_i is fluid.
__global__ void k_color_solid(Lattice L, const uint32_t *__restrict__ list, long long count,
                              const uint32_t *__restrict__ link, float *__restrict__ rhoN) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const uint32_t pk = list[t];
  const int x = (int)(pk & 1023u), y = (int)((pk >> 10) & 1023u), z = (int)((pk >> 20) & 2047u);
  StencilOffsets S;
  S.init(L, x, y, z);
  const uint32_t lk = link[S.own];
  float num = 0.f, den = 0.f;
#pragma unroll
  for (int i = 0; i < Q - 1; ++i) {
    if ((lk >> i) & 1u) {
      num += W[i] * rhoN[S.nb(CX[i], CY[i], CZ[i])];
      den += W[i];
    }
  }
  rhoN[S.own] = den > 0.f ? num / den : 0.f;
}

// a4 + a5 from the gradient (gx, gy, gz): n = +grad/|grad| (reading of
// Eq. color_gradient_normal), then at wall nodes n_+ or n_- of
// Eq. realigned_normal_vectors, whichever is nearer to n.  Returns (n, |grad|).
// solid() returns the node's solid normal n_s and contact angle (radians, .w);
// it is called only at wall nodes.
template <class SolidNormal>
__device__ __forceinline__ float4 wetted_normal_from(const StepParams &P, uint32_t lk, const SolidNormal &solid,
                                                     float gx, float gy, float gz) {
  const float gm = sqrtf(gx * gx + gy * gy + gz * gz);
  float nx_ = 0.f, ny_ = 0.f, nz_ = 0.f;
  if (gm >= GRAD_EPS) {
    const float inv = 1.0f / gm;
    nx_ = gx * inv;
    ny_ = gy * inv;
    nz_ = gz * inv;
    if ((lk & BIT_WALL) && (lk & BIT_NS_OK)) {
      const float4 s = solid();
      float sin_th, cos_th;
      sincosf(s.w, &sin_th, &cos_th);
      const float c = s.x * nx_ + s.y * ny_ + s.z * nz_;          // cos(theta')
      const float tx = nx_ - c * s.x, ty = ny_ - c * s.y, tz = nz_ - c * s.z;
      const float st2 = tx * tx + ty * ty + tz * tz;              // sin^2(theta')
      if (st2 >= SIN2_EPS) {
        const float a_n = sin_th / sqrtf(st2), a_s = a_n * c;
        const float px = (cos_th - a_s) * s.x + a_n * nx_;
        const float py = (cos_th - a_s) * s.y + a_n * ny_;
        const float pz = (cos_th - a_s) * s.z + a_n * nz_;
        const float mx = (cos_th + a_s) * s.x - a_n * nx_;
        const float my = (cos_th + a_s) * s.y - a_n * ny_;
        const float mz = (cos_th + a_s) * s.z - a_n * nz_;
        const float dp = (px - nx_) * (px - nx_) + (py - ny_) * (py - ny_) + (pz - nz_) * (pz - nz_);
        const float dm = (mx - nx_) * (mx - nx_) + (my - ny_) * (my - ny_) + (mz - nz_) * (mz - nz_);
        if (dp <= dm) {
          nx_ = px; ny_ = py; nz_ = pz;
        } else {
          nx_ = mx; ny_ = my; nz_ = mz;
        }
      }
    }
  }
  return make_float4(nx_, ny_, nz_, gm);
}
__device__ __forceinline__ float4 wetted_normal(const StepParams &P, uint32_t lk, const float4 *__restrict__ ns,
                                                unsigned node, float gx, float gy, float gz) {
  return wetted_normal_from(P, lk, [&] { return ns[node]; }, gx, gy, gz);
}

// a4 + a5 over the lattice (one thread per node)
__global__ void __launch_bounds__(256) k_normal(Lattice L, StepParams P, const float *__restrict__ rhoN,
                                                const uint32_t *__restrict__ link, const float4 *__restrict__ ns,
                                                float4 *__restrict__ nrm) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  const bool inside = x < L.nx && y < L.ny;
  const long long node = inside ? nidx(L, x, y, z) : 0;
  const uint32_t lk = inside ? link[node] : BIT_SOLID;
  const bool fluid = !(lk & BIT_SOLID);
  if (!__any_sync(0xffffffffu, fluid) || !inside) return;
  if (!fluid) {   // full-sector stores; solid nodes next to the fluid are filled by k_normal_solid
    nrm[node] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  StencilOffsets S;
  S.init(L, x, y, z);
  float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
  for (int i = 0; i < Q - 1; ++i) {
    const float v = 3.0f * W[i] * rhoN[S.nb(CX[i], CY[i], CZ[i])];
    gx += CX[i] * v;
    gy += CY[i] * v;
    gz += CZ[i] * v;
  }
  nrm[node] = wetted_normal(P, lk, ns, (unsigned)node, gx, gy, gz);
}

// n at solid nodes next to the fluid: lattice-weighted average of the fluid
// neighbours' wetted n, renormalised (needed by the curvature stencil)
__global__ void k_normal_solid(Lattice L, const uint32_t *__restrict__ list, long long count,
                               const uint32_t *__restrict__ link, float4 *__restrict__ nrm) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const uint32_t pk = list[t];
  const int x = (int)(pk & 1023u), y = (int)((pk >> 10) & 1023u), z = (int)((pk >> 20) & 2047u);
  StencilOffsets S;
  S.init(L, x, y, z);
  const uint32_t lk = link[S.own];
  float ax = 0.f, ay = 0.f, az = 0.f;
#pragma unroll
  for (int i = 0; i < Q - 1; ++i) {
    if ((lk >> i) & 1u) {
      const float4 v = nrm[S.nb(CX[i], CY[i], CZ[i])];
      ax += W[i] * v.x;
      ay += W[i] * v.y;
      az += W[i] * v.z;
    }
  }
  const float m = sqrtf(ax * ax + ay * ay + az * az);
  if (m >= GRAD_EPS) {
    const float inv = 1.0f / m;
    nrm[S.own] = make_float4(ax * inv, ay * inv, az * inv, 0.f);
  } else {
    nrm[S.own] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// a6: H = -sum_ab (delta_ab - n_a n_b) d_a n_b, d_a n_b by Eq. finite_difference_scheme;
// nb(i) returns the normal at x + c_i
// LEAN (the FP16-storage main kernel): the 18 neighbours as 9 opposite pairs,
// c_opp = -c, each pair adding 3 w c_a (n_b(x + c) - n_b(x - c)): one difference per
// component instead of a second product per nonzero c_a.  The FP32 kernel keeps the
// direction-by-direction sum, which holds fewer values at a time: at its 64-register
// budget the pair form spills and is 3 us slower on the 128x128x256 column, while
// the FP16 kernel gains.
template <bool LEAN = false, class NbNormal>
__device__ __forceinline__ float curvature(const float4 nme, const NbNormal &nb) {
  float d[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  if constexpr (LEAN) {
    constexpr int PAIR[9] = {0, 2, 4, 6, 7, 8, 9, 14, 15};   // i < OPP[i]
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int i = PAIR[k];
      const float4 a = nb(i), b = nb(OPP[i]);
      const float vx = a.x - b.x, vy = a.y - b.y, vz = a.z - b.z;
      const float w3 = 3.0f * W[i];
      if (CX[i]) { d[0][0] += w3 * CX[i] * vx; d[0][1] += w3 * CX[i] * vy; d[0][2] += w3 * CX[i] * vz; }
      if (CY[i]) { d[1][0] += w3 * CY[i] * vx; d[1][1] += w3 * CY[i] * vy; d[1][2] += w3 * CY[i] * vz; }
      if (CZ[i]) { d[2][0] += w3 * CZ[i] * vx; d[2][1] += w3 * CZ[i] * vy; d[2][2] += w3 * CZ[i] * vz; }
    }
  } else {
#pragma unroll
    for (int i = 0; i < Q - 1; ++i) {
      const float4 v = nb(i);
      const float w3 = 3.0f * W[i];
      if (CX[i]) { d[0][0] += w3 * CX[i] * v.x; d[0][1] += w3 * CX[i] * v.y; d[0][2] += w3 * CX[i] * v.z; }
      if (CY[i]) { d[1][0] += w3 * CY[i] * v.x; d[1][1] += w3 * CY[i] * v.y; d[1][2] += w3 * CY[i] * v.z; }
      if (CZ[i]) { d[2][0] += w3 * CZ[i] * v.x; d[2][1] += w3 * CZ[i] * v.y; d[2][2] += w3 * CZ[i] * v.z; }
    }
  }
  const float n3[3] = {nme.x, nme.y, nme.z};
  float proj = d[0][0] + d[1][1] + d[2][2];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) proj -= n3[a] * n3[b] * d[a][b];
  return -proj;
}

// a2, a7 - a10 at one fluid node.  In: fr, fp, g = pulled f^r, f^p, g (g only in
// reaction mode 0), nme = (n, |grad rho^N|), H.  Out: fr, fp, g = post-collision
// f^r*, f^p*, g*.  Returns the reaction amount delta.
// LEAN selects the recolouring loop's form (see below); both compute the same values.
template <bool LEAN = false>
__device__ __forceinline__ float collide_node(const StepParams &P, uint32_t lk, float (&fr)[Q], float (&fp)[Q],
                                              float (&g)[Q7], const float4 nme, float H) {
  // a2: moments
  float rr = 0.f, rp = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
  float pxx = 0.f, pyy = 0.f, pzz = 0.f, pxy = 0.f, pxz = 0.f, pyz = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    rr += fr[i];
    rp += fp[i];
    const float m = fr[i] + fp[i];
    fr[i] = m;   // fr now holds f^m
    if (CX[i]) jx += CX[i] * m;
    if (CY[i]) jy += CY[i] * m;
    if (CZ[i]) jz += CZ[i] * m;
    if (CX[i]) pxx += m;
    if (CY[i]) pyy += m;
    if (CZ[i]) pzz += m;
    if (CX[i] && CY[i]) pxy += CX[i] * CY[i] * m;
    if (CX[i] && CZ[i]) pxz += CX[i] * CZ[i] * m;
    if (CY[i] && CZ[i]) pyz += CY[i] * CZ[i] * m;
  }
  const float rho = rr + rp;
  const float inv_rho = 1.0f / rho;
  const float ux = jx * inv_rho, uy = jy * inv_rho, uz = jz * inv_rho;
  // a7: du = (sigma/2) H |grad rho^N| n / rho^m + a (same for both components)
  const float fs = P.half_sigma * H * nme.w * inv_rho;
  const float dux = fs * nme.x + P.ax, duy = fs * nme.y + P.ay, duz = fs * nme.z + P.az;
  // a8: central moments k5..k9 of f^m about u (Eq. post_collision_moments)
  const float k5 = P.omega_cm * ((pxx - pyy) - rho * (ux * ux - uy * uy));
  const float k6 = P.omega_cm * ((pyy - pzz) - rho * (uy * uy - uz * uz));
  const float k7 = P.omega_cm * (pxy - rho * ux * uy);
  const float k8 = P.omega_cm * (pxz - rho * ux * uz);
  const float k9 = P.omega_cm * (pyz - rho * uy * uz);
  float bt[Q];
  back_transform(ux, uy, uz, k5, k6, k7, k8, k9, bt);
  const float vx = ux + dux, vy = uy + duy, vz = uz + duz;
  const float vv = vx * vx + vy * vy + vz * vz;
  // a10: reaction amount (explicit Euler, post-streaming densities)
  const float psi = rr * inv_rho;
  float delta = 0.f;
  const uint32_t nn = (lk >> NN_SHIFT) & 7u;
  float conc = 0.f;
  if (P.reaction_mode == 0) {
#pragma unroll
    for (int j = 0; j < Q7; ++j) conc += g[j];
    if (lk & BIT_REACTIVE) delta = fminf(fminf(P.k_rate * (float)nn * conc * psi, conc), rr);
  } else {
    if (lk & BIT_REACTIVE) delta = fminf(P.xi * (float)nn, 1.0f) * rr;
  }
  delta = fmaxf(delta, 0.f);
  // a9: recolouring + reaction transfer.  The rest population is taken from
  // mass conservation (sum_i f^m*_i = rho^m holds exactly in exact arithmetic):
  // the FP32-rounded weights sum to 1 + 2.5e-8, which would otherwise add that
  // much mass per node and step.
  const float Brec = P.beta * rr * rp * inv_rho;
  if constexpr (!LEAN) {
    float msum = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      float fm_star;
      if (i < Q - 1) {
        const float cu = cdot(i, vx, vy, vz);
        fm_star = W[i] * rho * (1.0f + 3.0f * cu + 4.5f * cu * cu - 1.5f * vv) + bt[i];
        msum += fm_star;
      } else {
        fm_star = rho - msum;
      }
      const float cn = cdot(i, nme.x, nme.y, nme.z) * INVNORM[i];
      const float r_star = psi * fm_star + W[i] * (Brec * cn - delta);
      fr[i] = r_star;
      fp[i] = fm_star - r_star;
    }
  } else {
    // LEAN: node-level factors first, so that each direction costs a few operations:
    // f^eq_i = w_i rho (A + c.u (3 + 4.5 c.u)), A = 1 - 1.5 u.u, and the recolouring
    // and reaction term w_i (Brec cos(phi_i) - delta) = +-b_a +- b_b - w_i delta with
    // b = w_i Brec n / |c_i| for the axis (|c| = 1) and diagonal (|c| = sqrt 2) classes.
    // Fewer instructions, more values live across the loop: faster in the FP16 main
    // kernel, 3 us slower (register spills) in the FP32 one.
    const float A = 1.0f - 1.5f * vv;
    const float wr1 = W1 * rho, wr2 = W2 * rho;
    const float b1 = W1 * Brec, b2 = W2 * Brec * RSQRT2;
    const float b1x = b1 * nme.x, b1y = b1 * nme.y, b1z = b1 * nme.z;
    const float b2x = b2 * nme.x, b2y = b2 * nme.y, b2z = b2 * nme.z;
    const float d1 = W1 * delta, d2 = W2 * delta;
    float msum = 0.f;
#pragma unroll
    for (int i = 0; i < Q - 1; ++i) {
      const bool axis = i < 6;
      const float cu = cdot(i, vx, vy, vz);
      const float fm_star = (axis ? wr1 : wr2) * fmaf(cu, fmaf(4.5f, cu, 3.0f), A) + bt[i];
      msum += fm_star;
      const float rec = axis ? cdot(i, b1x, b1y, b1z) - d1 : cdot(i, b2x, b2y, b2z) - d2;
      const float r_star = fmaf(psi, fm_star, rec);
      fr[i] = r_star;
      fp[i] = fm_star - r_star;
    }
    {
      const float fm_star = rho - msum;   // rest population: cos(phi) = 0
      const float r_star = fmaf(psi, fm_star, -W0 * delta);
      fr[Q - 1] = r_star;
      fp[Q - 1] = fm_star - r_star;
    }
  }
  if (P.reaction_mode == 0) {
    // D3Q7 BGK of C advected by the physical velocity u + du/2, minus the reacted amount
    const float wx = ux + 0.5f * dux, wy = uy + 0.5f * duy, wz = uz + 0.5f * duz;
#pragma unroll
    for (int j = 0; j < Q7; ++j) {
      const int dd = GDIR[j];
      const float geq = W7[j] * conc * (1.0f + 4.0f * cdot(dd, wx, wy, wz));
      g[j] = g[j] + (geq - g[j]) * P.inv_tau_g - W7[j] * delta;
    }
  }
  return delta;
}

// FP64 block sum -> cumulative total acc[0] and this step's slot acc[2 + slot]
__device__ __forceinline__ void block_delta_sum(double dsum, double *acc, int slot) {
  __shared__ double red[32];
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  dsum = warp_sum(dsum);
  if ((tid & 31) == 0) red[tid >> 5] = dsum;
  __syncthreads();
  if (tid < 32) {
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
    double s = tid < nw ? red[tid] : 0.0;
    s = warp_sum(s);
    if (tid == 0 && s != 0.0) {
      atomicAdd(acc + 0, s);
      atomicAdd(acc + 2 + slot, s);
    }
  }
}

// a1, a2, a6 - a10 at fluid node (x, y, z) with link word lk, dense layout: pull,
// curvature, collision, recolouring, reaction, transport, stores, outlet ghost.
// Returns delta.
__device__ __forceinline__ float main_node(const Lattice &L, const StepParams &P, const float *__restrict__ fin,
                                           float *__restrict__ fout, const float4 *__restrict__ nrm, int x, int y,
                                           int z, unsigned node, uint32_t lk, float *__restrict__ dbg_H,
                                           float *__restrict__ dbg_delta) {
  const unsigned ps = (unsigned)L.pstride;
  PullOffsets O;
  O.init(L, x, y, z);
  StencilOffsets S;
  S.init(L, x, y, z);
  // a6 first, so that its loads do not overlap the 45 live populations
  const float4 nme = nrm[node];
  const float H =
      nme.w >= GRAD_EPS ? curvature(nme, [&](int i) { return nrm[S.nb(CX[i], CY[i], CZ[i])]; }) : 0.f;
  // a1: pull with bounce-back
  float fr[Q], fp[Q], g[Q7];
  {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const bool bb = (lk >> i) & 1u;
      const unsigned off = bb ? O.own : O.src(CX[i], CY[i], CZ[i]);
      const unsigned pr = bb ? (unsigned)OPP[i] : (unsigned)i;
      fr[i] = fin[pr * ps + off];
      fp[i] = fin[(pr + Q) * ps + off];
    }
    if (P.reaction_mode == 0) {
#pragma unroll
      for (int j = 0; j < Q7; ++j) {
        const int d = GDIR[j];
        const bool bb = (lk >> d) & 1u;
        const unsigned off = bb ? O.own : O.src(CX[d], CY[d], CZ[d]);
        const unsigned pj = bb ? (unsigned)GOPP[j] : (unsigned)j;
        g[j] = fin[(2 * Q + pj) * ps + off];
      }
    }
  }
  const float delta = collide_node(P, lk, fr, fp, g, nme, H);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    fout[(unsigned)i * ps + O.own] = fr[i];
    fout[(unsigned)(Q + i) * ps + O.own] = fp[i];
  }
  float g5 = 0.f;
  if (P.reaction_mode == 0) {
#pragma unroll
    for (int j = 0; j < Q7; ++j) fout[(unsigned)(2 * Q + j) * ps + O.own] = g[j];
    g5 = g[5];
  } else {
    g5 = fin[(unsigned)(2 * Q + 5) * ps + O.own];
  }
  if (L.bc_z == 1 && z == L.nz - 1) write_outlet_ghost(L, fout, x, y, fr, fp, g5, P.rho_out);
  if (dbg_H) dbg_H[node] = H;
  if (dbg_delta) dbg_delta[node] = delta;
  return delta;
}

// Main update, dense layout, one thread per lattice node (used by the
// allocation-free entry point).
__global__ void __launch_bounds__(128, 5) k_main(Lattice L, StepParams P, const float *__restrict__ fin,
                                              float *__restrict__ fout, const uint32_t *__restrict__ link,
                                              const float4 *__restrict__ nrm, double *__restrict__ acc,
                                              int slot, float *__restrict__ dbg_H, float *__restrict__ dbg_delta) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  double dsum = 0.0;
  if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 && threadIdx.y == 0)
    acc[2 + (slot ^ 1)] = 0.0;   // clear the other per-step slot for the next step
  const bool inside = x < L.nx && y < L.ny;
  const unsigned node = inside ? (unsigned)nidx(L, x, y, z) : 0u;
  const uint32_t lk = inside ? link[node] : BIT_SOLID;
  if (!(lk & BIT_SOLID))
    dsum = (double)main_node(L, P, fin, fout, nrm, x, y, z, node, lk, dbg_H, dbg_delta);
  block_delta_sum(dsum, acc, slot);
}

// ---------------------------------------------------------------------------
// a11: observables of the stored state (FP64 block reductions)
// ---------------------------------------------------------------------------
// acc layout: 0 mass_r, 1 mass_p, 2 mass_c, 3 sum (1 - rho^N)/2, 4 flux_in, 5 flux_out, 6 n_bad
__global__ void k_observables(Lattice L, const float *__restrict__ f, const uint32_t *__restrict__ link,
                              double *__restrict__ acc) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  double v[7] = {0, 0, 0, 0, 0, 0, 0};
  const bool inside = x < L.nx && y < L.ny;
  const long long node = inside ? nidx(L, x, y, z) : 0;
  if (inside && !(link[node] & BIT_SOLID)) {
    // per-node sums in FP32 (19 terms), accumulation over the lattice in FP64
    float rr = 0.f, rp = 0.f, cc = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const float a = f[pidx(L, i, z + 1, y, x)], b = f[pidx(L, Q + i, z + 1, y, x)];
      rr += a;
      rp += b;
      if (CZ[i]) jz += CZ[i] * (a + b);
    }
#pragma unroll
    for (int j = 0; j < Q7; ++j) cc += f[pidx(L, 2 * Q + j, z + 1, y, x)];
    const float rho = rr + rp;
    v[0] = rr;
    v[1] = rp;
    v[2] = cc;
    const bool bad = !(rho > 0.f) || !isfinite(rho) || !isfinite(cc);
    if (!bad) {
      v[3] = 0.5f * (1.0f - (rr - rp) / rho);
      if (z == 0) v[4] = jz / rho * cc;
      if (z == L.nz - 1) v[5] = jz / rho * cc;
    }
    v[6] = bad ? 1.0 : 0.0;
  }
  block_accumulate<7>(v, acc);
}

}  // namespace cglbm
