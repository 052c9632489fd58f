// Compact population layout: only fluid nodes (and the column ghost planes) own
// population slots.
//
// In the paper's bicontinuous supports about half the lattice is solid.  A
// dense structure-of-arrays layout moves the solid nodes' slots with every
// 32-byte sector that also holds fluid data, and the fluid-only stores leave
// sectors partly written, which the memory system completes with an extra
// read.  Here population p of slot s sits at f[p * ns + s]; slots 0 .. nf-1 are
// the fluid nodes in lattice order, slots nf .. nf + 2 * plane - 1 the inlet and
// outlet ghost planes (column mode).  gidx maps every stored lattice position
// (plane z + 1 in [0, nz + 1]) to its slot, or -1 for a solid node.  Fields
// that stencils read (rho^N, n, link words, n_s) stay dense, indexed by node.
//
// Storage type T: float (FP32 values) or __half (FP16 deviations from fixed
// reference equilibria: f^r_i - w_i, f^p_i, g_j - w_j, i.e. reactant liquid at
// rest with C = 1; all arithmetic in FP32).
#pragma once
#include <cuda_fp16.h>

#include "kernels.cuh"

// launch shapes (the defaults are the measured best on B300)
#ifndef CGLBM_MAIN_BLOCK
#define CGLBM_MAIN_BLOCK 128
#endif
#ifndef CGLBM_MAIN_MINB
#define CGLBM_MAIN_MINB 8
#endif
#ifndef CGLBM_DENS_MINB
#define CGLBM_DENS_MINB 1
#endif

namespace cglbm {

struct Compact {
  int nf;   // fluid slots
  int ns;   // slot stride of one population (>= nf + ghost slots, multiple of 64)
};

// reference value subtracted before FP16 storage of population p
__device__ __forceinline__ float pop_ref(int p) { return p < Q ? W[p] : (p < 2 * Q ? 0.f : W7[p - 2 * Q]); }

template <typename T>
struct Store;
template <>
struct Store<float> {
  static __device__ __forceinline__ float ld(const float *__restrict__ f, unsigned idx, int) { return f[idx]; }
  static __device__ __forceinline__ void st(float *__restrict__ f, unsigned idx, int, float v) { f[idx] = v; }
};
template <>
struct Store<__half> {
  static __device__ __forceinline__ float ld(const __half *__restrict__ f, unsigned idx, int p) {
    return __half2float(f[idx]) + pop_ref(p);
  }
  static __device__ __forceinline__ void st(__half *__restrict__ f, unsigned idx, int p, float v) {
    f[idx] = __float2half_rn(v - pop_ref(p));
  }
};

__device__ __forceinline__ void unpack(uint32_t pk, int &x, int &y, int &z) {
  x = (int)(pk & 1023u);
  y = (int)((pk >> 10) & 1023u);
  z = (int)((pk >> 20) & 2047u);
}

// pull of the 45 (38) populations of fluid slot t at (x, y, z), halfway bounce-back
// where the source is solid (gidx < 0)
template <typename T>
__device__ __forceinline__ void pull_compact(const Compact &C, const StepParams &P, const T *__restrict__ fin,
                                             const int *__restrict__ gidx, const PullOffsets &O, unsigned t,
                                             float (&fr)[Q], float (&fp)[Q], float (&g)[Q7]) {
  const unsigned ns = (unsigned)C.ns;
  int src[Q];
#pragma unroll
  for (int i = 0; i < Q - 1; ++i) src[i] = __ldg(gidx + O.src(CX[i], CY[i], CZ[i]));
  src[Q - 1] = (int)t;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const bool bb = src[i] < 0;
    const unsigned s = bb ? t : (unsigned)src[i];
    const unsigned pr = bb ? (unsigned)OPP[i] : (unsigned)i;
    // the reference of population OPP[i] equals that of i (w is even in c)
    fr[i] = Store<T>::ld(fin, pr * ns + s, i);
    fp[i] = Store<T>::ld(fin, (pr + Q) * ns + s, Q + i);
  }
  if (P.reaction_mode == 0) {
#pragma unroll
    for (int j = 0; j < Q7; ++j) {
      const int d = GDIR[j];
      const bool bb = src[d] < 0;
      const unsigned s = bb ? t : (unsigned)src[d];
      const unsigned pj = bb ? (unsigned)GOPP[j] : (unsigned)j;
      g[j] = Store<T>::ld(fin, (2 * Q + pj) * ns + s, 2 * Q + j);
    }
  }
}

// a1 + a2 over the fluid slots: colour function rho^N (dense field)
template <typename T>
__global__ void __launch_bounds__(256, CGLBM_DENS_MINB) k_density_c(Lattice L, Compact C, const T *__restrict__ f,
                                                                    const int *__restrict__ gidx,
                                                                    const uint32_t *__restrict__ cnode,
                                                                    float *__restrict__ rhoN) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (unsigned)C.nf) return;
  int x, y, z;
  unpack(cnode[t], x, y, z);
  PullOffsets O;
  O.init(L, x, y, z);
  const unsigned ns = (unsigned)C.ns;
  float rr = 0.f, rp = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int si = i == Q - 1 ? (int)t : __ldg(gidx + O.src(CX[i], CY[i], CZ[i]));
    const bool bb = si < 0;
    const unsigned s = bb ? t : (unsigned)si;
    const unsigned pr = bb ? (unsigned)OPP[i] : (unsigned)i;
    rr += Store<T>::ld(f, pr * ns + s, i);
    rp += Store<T>::ld(f, (pr + Q) * ns + s, Q + i);
  }
  rhoN[nidx(L, x, y, z)] = (rr - rp) / (rr + rp);
}

// a4 + a5 over the fluid slots (same arithmetic as k_normal)
__global__ void __launch_bounds__(256) k_normal_c(Lattice L, StepParams P, Compact C,
                                                  const uint32_t *__restrict__ cnode, const float *__restrict__ rhoN,
                                                  const uint32_t *__restrict__ link, const float4 *__restrict__ ns,
                                                  float4 *__restrict__ nrm) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (unsigned)C.nf) return;
  int x, y, z;
  unpack(cnode[t], x, y, z);
  StencilOffsets S;
  S.init(L, x, y, z);
  const unsigned node = S.own;
  const uint32_t lk = link[node];
  float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
  for (int i = 0; i < Q - 1; ++i) {
    const float v = 3.0f * W[i] * rhoN[S.nb(CX[i], CY[i], CZ[i])];
    gx += CX[i] * v;
    gy += CY[i] * v;
    gz += CZ[i] * v;
  }
  nrm[node] = wetted_normal(P, lk, ns, node, gx, gy, gz);
}

// outlet ghost (column mode) of slot gs from the post-collision populations of a
// fluid node of plane nz - 1 (same arithmetic as write_outlet_ghost)
template <typename T>
__device__ __forceinline__ void write_outlet_ghost_c(const Compact &C, T *__restrict__ f, unsigned gs,
                                                     const float (&fr)[Q], const float (&fp)[Q], float g5,
                                                     float rho_out) {
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
  const unsigned ns = (unsigned)C.ns;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (CZ[i] != -1) continue;
    const float corr = feq19(i, rho_out - rho, vx, vy, vz, vv);
    Store<T>::st(f, (unsigned)i * ns + gs, i, fr[i] + psi * corr);
    Store<T>::st(f, (unsigned)(Q + i) * ns + gs, Q + i, fp[i] + (1.0f - psi) * corr);
  }
  Store<T>::st(f, (unsigned)(2 * Q + 5) * ns + gs, 2 * Q + 5, g5);
}

// a1, a2, a6 - a10 over the fluid slots; stores are coalesced and whole-sector
template <typename T>
__global__ void __launch_bounds__(CGLBM_MAIN_BLOCK, CGLBM_MAIN_MINB) k_main_c(
    Lattice L, Compact C, StepParams P, const T *__restrict__ fin, T *__restrict__ fout,
    const int *__restrict__ gidx, const uint32_t *__restrict__ cnode, const uint32_t *__restrict__ link,
    const float4 *__restrict__ nrm, double *__restrict__ acc, int slot, float *__restrict__ dbg_H,
    float *__restrict__ dbg_delta) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  double dsum = 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) acc[2 + (slot ^ 1)] = 0.0;
  if (t < (unsigned)C.nf) {
    int x, y, z;
    unpack(cnode[t], x, y, z);
    StencilOffsets S;
    S.init(L, x, y, z);
    const unsigned node = S.own;
    const uint32_t lk = link[node];
    const float4 nme = nrm[node];
    const float H =
        nme.w >= GRAD_EPS ? curvature(nme, [&](int i) { return nrm[S.nb(CX[i], CY[i], CZ[i])]; }) : 0.f;
    PullOffsets O;
    O.init(L, x, y, z);
    float fr[Q], fp[Q], g[Q7];
    pull_compact<T>(C, P, fin, gidx, O, t, fr, fp, g);
    const float delta = collide_node(P, lk, fr, fp, g, nme, H);
    const unsigned ns = (unsigned)C.ns;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      Store<T>::st(fout, (unsigned)i * ns + t, i, fr[i]);
      Store<T>::st(fout, (unsigned)(Q + i) * ns + t, Q + i, fp[i]);
    }
    float g5;
    if (P.reaction_mode == 0) {
#pragma unroll
      for (int j = 0; j < Q7; ++j) Store<T>::st(fout, (unsigned)(2 * Q + j) * ns + t, 2 * Q + j, g[j]);
      g5 = g[5];
    } else {
      g5 = Store<T>::ld(fin, (unsigned)(2 * Q + 5) * ns + t, 2 * Q + 5);
    }
    if (L.bc_z == 1 && z == L.nz - 1) {
      const unsigned gs = (unsigned)(C.nf + L.plane) + (unsigned)(y * L.nx + x);
      write_outlet_ghost_c<T>(C, fout, gs, fr, fp, g5, P.rho_out);
    }
    if (dbg_H) dbg_H[node] = H;
    if (dbg_delta) dbg_delta[node] = delta;
    dsum = (double)delta;
  }
  block_delta_sum(dsum, acc, slot);
}

// equilibrium start of the fluid slots from dense fields (null: uniform values)
template <typename T>
__global__ void k_init_c(Lattice L, Compact C, const uint32_t *__restrict__ cnode, const float *__restrict__ rho_r,
                         const float *__restrict__ rho_p, const float *__restrict__ conc, const float *__restrict__ u,
                         float rr0, float rp0, float c0, T *__restrict__ fa, T *__restrict__ fb) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (unsigned)C.nf) return;
  int x, y, z;
  unpack(cnode[t], x, y, z);
  const long long node = nidx(L, x, y, z);
  const float rr = rho_r ? rho_r[node] : rr0;
  const float rp = rho_p ? rho_p[node] : rp0;
  const float cc = conc ? conc[node] : c0;
  const float ux = u ? u[node] : 0.f, uy = u ? u[L.n + node] : 0.f, uz = u ? u[2 * L.n + node] : 0.f;
  const float uu = ux * ux + uy * uy + uz * uz;
  const unsigned ns = (unsigned)C.ns;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float a = feq19(i, rr, ux, uy, uz, uu), b = feq19(i, rp, ux, uy, uz, uu);
    Store<T>::st(fa, (unsigned)i * ns + t, i, a);
    Store<T>::st(fb, (unsigned)i * ns + t, i, a);
    Store<T>::st(fa, (unsigned)(Q + i) * ns + t, Q + i, b);
    Store<T>::st(fb, (unsigned)(Q + i) * ns + t, Q + i, b);
  }
#pragma unroll
  for (int j = 0; j < Q7; ++j) {
    const int d = GDIR[j];
    const float gv = W7[j] * cc * (1.0f + 4.0f * (CX[d] * ux + CY[d] * uy + CZ[d] * uz));
    Store<T>::st(fa, (unsigned)(2 * Q + j) * ns + t, 2 * Q + j, gv);
    Store<T>::st(fb, (unsigned)(2 * Q + j) * ns + t, 2 * Q + j, gv);
  }
}

// Column ghost slots of both buffers: constant inlet, outlet from plane nz - 1 of
// fa (resting reactant equilibrium above solid nodes).
template <typename T>
__global__ void k_ghost_init_c(Lattice L, Compact C, const int *__restrict__ gidx, float u_in, float c_in,
                               float rho_out, T *__restrict__ fa, T *__restrict__ fb) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= L.nx || y >= L.ny) return;
  const unsigned ns = (unsigned)C.ns;
  const unsigned gin = (unsigned)C.nf + (unsigned)(y * L.nx + x);
  const unsigned gout = gin + (unsigned)L.plane;
  const float uu = u_in * u_in;
#pragma unroll
  for (int p = 0; p < NPOP; ++p) {
    Store<T>::st(fa, (unsigned)p * ns + gin, p, 0.f);
    Store<T>::st(fb, (unsigned)p * ns + gin, p, 0.f);
    Store<T>::st(fa, (unsigned)p * ns + gout, p, 0.f);
    Store<T>::st(fb, (unsigned)p * ns + gout, p, 0.f);
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (CZ[i] != 1) continue;
    const float v = feq19(i, 1.0f, 0.f, 0.f, u_in, uu);
    Store<T>::st(fa, (unsigned)i * ns + gin, i, v);
    Store<T>::st(fb, (unsigned)i * ns + gin, i, v);
  }
  const float g4 = W7[4] * c_in * (1.0f + 4.0f * u_in);
  Store<T>::st(fa, (unsigned)(2 * Q + 4) * ns + gin, 2 * Q + 4, g4);
  Store<T>::st(fb, (unsigned)(2 * Q + 4) * ns + gin, 2 * Q + 4, g4);
  const int s = gidx[(long long)L.nz * L.plane + (long long)y * L.nx + x];   // stored plane nz = z nz-1
  if (s < 0) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (CZ[i] != -1) continue;
      Store<T>::st(fa, (unsigned)i * ns + gout, i, W[i] * rho_out);
      Store<T>::st(fb, (unsigned)i * ns + gout, i, W[i] * rho_out);
    }
  } else {
    float fr[Q], fp[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      fr[i] = Store<T>::ld(fa, (unsigned)i * ns + (unsigned)s, i);
      fp[i] = Store<T>::ld(fa, (unsigned)(Q + i) * ns + (unsigned)s, Q + i);
    }
    const float g5 = Store<T>::ld(fa, (unsigned)(2 * Q + 5) * ns + (unsigned)s, 2 * Q + 5);
    write_outlet_ghost_c<T>(C, fa, gout, fr, fp, g5, rho_out);
  }
}

// a11 over the fluid slots (FP32 per node, FP64 block accumulation); acc layout
// as k_observables
template <typename T>
__global__ void k_observables_c(Lattice L, Compact C, const T *__restrict__ f, const uint32_t *__restrict__ cnode,
                                double *__restrict__ acc) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  double v[7] = {0, 0, 0, 0, 0, 0, 0};
  if (t < (unsigned)C.nf) {
    int x, y, z;
    unpack(cnode[t], x, y, z);
    const unsigned ns = (unsigned)C.ns;
    float rr = 0.f, rp = 0.f, cc = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const float a = Store<T>::ld(f, (unsigned)i * ns + t, i);
      const float b = Store<T>::ld(f, (unsigned)(Q + i) * ns + t, Q + i);
      rr += a;
      rp += b;
      if (CZ[i]) jz += CZ[i] * (a + b);
    }
#pragma unroll
    for (int j = 0; j < Q7; ++j) cc += Store<T>::ld(f, (unsigned)(2 * Q + j) * ns + t, 2 * Q + j);
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

// state transfer helpers: stored populations of the fluid slots <-> FP32 values
// in a [45][nf] buffer
template <typename T>
__global__ void k_slots_to_f32(Compact C, const T *__restrict__ src, float *__restrict__ dst) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (unsigned)C.nf) return;
#pragma unroll
  for (int p = 0; p < NPOP; ++p) dst[(size_t)p * C.nf + t] = Store<T>::ld(src, (unsigned)p * C.ns + t, p);
}
template <typename T>
__global__ void k_f32_to_slots(Compact C, const float *__restrict__ src, T *__restrict__ a, T *__restrict__ b) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (unsigned)C.nf) return;
#pragma unroll
  for (int p = 0; p < NPOP; ++p) {
    const float v = src[(size_t)p * C.nf + t];
    Store<T>::st(a, (unsigned)p * C.ns + t, p, v);
    Store<T>::st(b, (unsigned)p * C.ns + t, p, v);
  }
}

}  // namespace cglbm
