// Compact, batched population layout and the per-step kernels that use it.
//
// Only fluid nodes (and the column ghost planes) own population slots.  In the
// paper's bicontinuous supports about half the lattice is solid; a dense
// structure-of-arrays layout moves the solid nodes' slots with every 32-byte
// sector that also holds fluid data, and fluid-only stores leave sectors partly
// written, which the memory system completes with an extra read.
//
// A batch holds one or more independent lattices ("instances", each with its
// own size, mask and parameters).  All their slots share one slot space:
// instance k owns the fluid slots [slot_off, slot_off + nf) in lattice order and,
// in column mode, the ghost slots [ghost, ghost + 2 * plane) (inlet plane, then
// outlet plane).  The populations of global slot s sit in the slot layout below
// (pop_index: f^r_i and f^p_i of s adjacent, g_j at 2 Q ns + j ns + s).  Every
// per-step kernel is one launch over all slots of all instances; a thread finds
// its node (packed x | y << 10 | z << 20, or kNoNode) and its instance (the
// per-slot instance array, absent for a single instance) and reads the
// instance's lattice, parameters and offsets from a small table.  Per-node
// fields that stencils read (rho^N, n, link words, n_s) stay dense per instance,
// at the instance's node offset; gidx maps each stored lattice position
// (plane z + 1 in [0, nz + 1]) to a global slot, or -1 for a solid node.
//
// Storage type T: float (FP32) or __half (FP16 deviations from fixed reference
// equilibria: f^r_i - w_i, f^p_i, g_j - w_j, i.e. reactant liquid at rest with
// C = 1, scaled by 2^12; all arithmetic in FP32).
#pragma once
#include <cuda_fp16.h>

#include <type_traits>

#include "kernels.cuh"

namespace cglbm {

constexpr uint32_t kNoNode = 0xFFFFFFFFu;

struct Inst {
  Lattice L;
  StepParams P;
  int nf;        // fluid slots
  int slot_off;  // first global fluid slot
  int ghost;     // first global ghost slot (column mode)
  int node_off;  // offset of the instance in the dense per-node fields
  int gidx_off;  // offset of the instance in gidx
  int pad;
};

struct Slots {
  const Inst *__restrict__ inst;     // instance table
  const uint16_t *__restrict__ kid;  // instance of each slot, or null (single instance)
  const uint32_t *__restrict__ node; // packed coordinates of each slot, kNoNode for ghost / padding
  int nslots;                        // slots covered by the launch grid
  int ns;                            // population stride
};

__device__ __forceinline__ int slot_instance(const Slots &S, unsigned t) { return S.kid ? (int)S.kid[t] : 0; }

__device__ __forceinline__ void unpack(uint32_t pk, int &x, int &y, int &z) {
  x = (int)(pk & 1023u);
  y = (int)((pk >> 10) & 1023u);
  z = (int)((pk >> 20) & 2047u);
}

// Reference values subtracted before FP16 storage: the weights w_i of f^r_i on a
// 2^-20 grid, summing to exactly 1 (6 x 58254 + 12 x 29127 + 349528 = 2^20), 0 for
// f^p_i and w_j (exact binary fractions) for g_j.  A reference is only an offset:
// any value near w_i serves, and the stored deviation is taken against the same
// one.  On the grid every partial sum of the references is exact in FP32, so the
// rounding of the sum of a node's 19 pulled f^r_i comes from the deviations alone.
// With the FP32-rounded w_i (whose low bits are the same at every node) that
// rounding leans one way whenever the deviations are coarse, as FP16 deviations
// are: +4e-8 per node and step, a steady gain of red mass (0.03 % over 5000 steps
// of the 64^3 crop of the 256^3 precision box).
constexpr float WR1 = 58254.0f / 1048576.0f, WR2 = 29127.0f / 1048576.0f, WR0 = 349528.0f / 1048576.0f;
__device__ constexpr float WREF[Q] = {WR1, WR1, WR1, WR1, WR1, WR1, WR2, WR2, WR2, WR2,
                                      WR2, WR2, WR2, WR2, WR2, WR2, WR2, WR2, WR0};
__device__ __forceinline__ float pop_ref(int p) { return p < Q ? WREF[p] : (p < 2 * Q ? 0.f : W7[p - 2 * Q]); }

// Population storage.  Population p of slot t: ld / st / st_r address it by
// (p, t) with ns the population stride; ld2 / st2_r move f^r_i and f^p_i of one
// slot together (i < Q), the pair the pull and the main kernel always access
// together.  ld2 reads the pair of direction i and adds the references of
// direction iref (the same value: the weights are even in c, so a bounced pair
// read from the opposite direction keeps the compile-time reference).
template <typename T>
struct Store;
// Slot layout shared by both storage types: f^r_i and f^p_i of slot t are
// adjacent (elements 2 (i ns + t) and 2 (i ns + t) + 1), so the pull, the density
// pass and the main kernel move the pair with one access; g_j follows at
// 2 Q ns + j ns + t.  (The adjoint's own arrays keep population-major order.)
__device__ __forceinline__ unsigned pop_index(unsigned ns, unsigned p, unsigned t) {
  return p < (unsigned)Q ? 2u * (p * ns + t) : (p < 2u * Q ? 2u * ((p - Q) * ns + t) + 1u : p * ns + t);
}

template <>
struct Store<float> {
  static __device__ __forceinline__ float ld(const float *__restrict__ f, unsigned ns, unsigned p, unsigned t) {
    return f[pop_index(ns, p, t)];
  }
  static __device__ __forceinline__ void st(float *__restrict__ f, unsigned ns, unsigned p, unsigned t, float v) {
    f[pop_index(ns, p, t)] = v;
  }
  static __device__ __forceinline__ void st_r(float *__restrict__ f, unsigned ns, unsigned p, unsigned t, float v,
                                              uint32_t) {
    f[pop_index(ns, p, t)] = v;
  }
  static __device__ __forceinline__ void ld2(const float *__restrict__ f, unsigned ns, unsigned i, unsigned t, int,
                                             float &a, float &b) {
    const float2 v = reinterpret_cast<const float2 *>(f)[i * ns + t];
    a = v.x;
    b = v.y;
  }
  static __device__ __forceinline__ void st2_r(float *__restrict__ f, unsigned ns, unsigned i, unsigned t, float a,
                                               float b, uint32_t) {
    reinterpret_cast<float2 *>(f)[i * ns + t] = make_float2(a, b);
  }
};
// FP32 -> FP16 with stochastic rounding: round away from zero with probability equal
// to the discarded fraction of an FP16 spacing, so that per-step changes smaller than
// half a spacing (which round-to-nearest drops every step) survive in expectation.
// The conversion is the hardware's (cvt.rs.f16x2.f32, sm_100 family): for each half,
// the 13 discarded mantissa bits and 13 random bits are added and the sum truncated,
// so the value rounds up exactly when they carry.  The low half takes its random bits
// from rbits[12:0], the high half from rbits[28:16] (measured on the B300 with single
// bits set against values whose discarded bits are known).  The stored deviations
// are scaled by 2^12 first (kHalfScale): FP16's normal range then starts at 1.5e-8
// instead of 6.1e-5, and deviations up to 16 in magnitude are representable
// (populations of a run near rho = 1 stay far below).  The rounding is unbiased only
// if the random bits are independent of the value's discarded bits, also from one
// step to the next: a node whose value repeats must not round the same way every
// step.  The per-step stores of the main kernel therefore draw their bits from the
// slot and a step counter (node_seed); the one-time writes (start, set_state, ghost
// set-up) hash the value's bits and the population's logical index p * ns + t
// (round_bits).  Both are deterministic and reproducible.
__device__ __forceinline__ uint32_t cvt_rs_half2(float hi, float lo, uint32_t rbits) {
  uint32_t d;
  asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
  return d;
}
__device__ __forceinline__ __half half_rs(float x, uint32_t r13) {   // r13: 13 random bits
  return __ushort_as_half((unsigned short)(cvt_rs_half2(0.f, x, r13) & 0xFFFFu));
}
__device__ __forceinline__ uint32_t round_bits(uint32_t bits, unsigned idx) {
  uint32_t h = (bits ^ idx) * 0x9E3779B9u;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  return h;
}
constexpr float kHalfScale = 4096.f, kHalfUnscale = 1.f / 4096.f;
__device__ __forceinline__ __half half_stochastic(float x, unsigned idx) {
  return half_rs(x, round_bits(__float_as_uint(x), idx) >> 19);
}

// The main kernel stores 45 values per node (and its outlet ghost's): it hashes
// the slot t and the step counter once per node (node_seed) and derives the random
// word of a store from seed * K_p, K_p an odd constant per population -- one
// multiply per store (per f^r_i / f^p_i pair) instead of a hash per store.  The
// value's bits do not enter the hash: a seed drawn from them repeats whenever the
// node's state does, and a node at rest then rounds the same way step after step (a
// steady mass drift: 36 mass units in 5000 steps of a 64^3 droplet box, against 1.0
// for FP32 storage).  v is the node's post-collision rest population, a function of
// every pulled value (through rho and C); a node where it is not finite gets seed 0
// (the conversion keeps a NaN a NaN whatever the random bits).
__device__ __forceinline__ uint32_t node_seed(float v, unsigned t, uint32_t step) {
  uint32_t h = ((t * 0x85EBCA6Bu) ^ (step * 0xC2B2AE35u)) * 0x9E3779B9u;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 13;
  return isfinite(v) ? h * 0x27D4EB2Fu : 0u;
}
__device__ __forceinline__ uint32_t pop_random(uint32_t seed, int p) {
  return seed * ((0x9E3779B9u ^ ((uint32_t)p * 0x632BE5ABu)) | 1u);
}

template <>
struct Store<__half> {
  // FP16 deviations from the reference equilibria, 2^12 (f^r_i - w~_i), 2^12 f^p_i,
  // 2^12 (g_j - w_j) with w~ the weights on the 2^-20 grid (WREF), in the slot layout
  // above (the f^r_i / f^p_i pair of a slot in one 32-bit word).
  static __device__ __forceinline__ unsigned hidx(unsigned ns, unsigned p, unsigned t) { return pop_index(ns, p, t); }
  static __device__ __forceinline__ float ld(const __half *__restrict__ f, unsigned ns, unsigned p, unsigned t) {
    return fmaf(__half2float(f[hidx(ns, p, t)]), kHalfUnscale, pop_ref(p));
  }
  static __device__ __forceinline__ void st(__half *__restrict__ f, unsigned ns, unsigned p, unsigned t, float v) {
    f[hidx(ns, p, t)] = half_stochastic(fmaf(v, kHalfScale, -kHalfScale * pop_ref(p)), p * ns + t);
  }
  // the same rounding with the random word r supplied by the caller (its top 13 bits)
  static __device__ __forceinline__ void st_r(__half *__restrict__ f, unsigned ns, unsigned p, unsigned t, float v,
                                              uint32_t r) {
    f[hidx(ns, p, t)] = half_rs(fmaf(v, kHalfScale, -kHalfScale * pop_ref(p)), r >> 19);
  }
  static __device__ __forceinline__ void ld2(const __half *__restrict__ f, unsigned ns, unsigned i, unsigned t,
                                             int iref, float &a, float &b) {
    const float2 v = __half22float2(reinterpret_cast<const __half2 *>(f)[i * ns + t]);
    a = fmaf(v.x, kHalfUnscale, WREF[iref]);
    b = fmaf(v.y, kHalfUnscale, 0.f);   // the reference of f^p is 0 (as in ld)
  }
  // f^r_i (low half) and f^p_i (high half) of slot t with one random word r: f^p_i
  // takes its top 13 bits (rbits[28:16] = r[31:19]), f^r_i bits 3 to 15
  static __device__ __forceinline__ void st2_r(__half *__restrict__ f, unsigned ns, unsigned i, unsigned t, float a,
                                               float b, uint32_t r) {
    reinterpret_cast<uint32_t *>(f)[i * ns + t] =
        cvt_rs_half2(b * kHalfScale, fmaf(a, kHalfScale, -kHalfScale * WREF[i]), r >> 3);
  }
};

// Sum NV doubles of every thread of the block into acc[k * stride + j], k the
// thread's instance: one atomic per value and block when the block holds one
// instance (the usual case: slots are contiguous per instance), else per thread.
template <int NV>
__device__ __forceinline__ void block_accumulate_inst(double (&v)[NV], int k, double *acc, int stride) {
  __shared__ double red[32][NV];
  __shared__ int k0s;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  if (tid == 0) k0s = k;
  __syncthreads();
  const int k0 = k0s;
  if (__syncthreads_and(k == k0)) {
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = warp_sum(v[j]);
    if (lane == 0) {
#pragma unroll
      for (int j = 0; j < NV; ++j) red[warp][j] = v[j];
    }
    __syncthreads();
    if (warp == 0) {
      const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        double s = lane < nw ? red[lane][j] : 0.0;
        s = warp_sum(s);
        if (lane == 0 && s != 0.0) atomicAdd(acc + (long long)k0 * stride + j, s);
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < NV; ++j)
      if (v[j] != 0.0) atomicAdd(acc + (long long)k * stride + j, v[j]);
  }
}

// Reaction sums of instance k: acc[4k + 2 slot] = sum of delta over the step with
// parity slot, acc[4k + 2 slot + 1] = cumulative sum after it (the pair is adjacent, so
// one 16-byte copy reads both).  The step's colour-function pass sets the pair to (0,
// cumulative sum after the previous step), see k_density_c; the main kernel adds
// each block's sum to both (per thread when the block spans instances).
template <bool BATCH>
__device__ __forceinline__ void block_delta_inst(double d, int k, double *acc, int slot) {
  __shared__ double red[32];
  __shared__ int k0s;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  int k0 = 0;
  if (BATCH) {
    if (tid == 0) k0s = k;
    __syncthreads();
    k0 = k0s;
  }
  if (!BATCH || __syncthreads_and(k == k0)) {
    d = warp_sum(d);
    if (lane == 0) red[warp] = d;
    __syncthreads();
    if (warp == 0) {
      const int nw = (blockDim.x + 31) >> 5;
      double s = lane < nw ? red[lane] : 0.0;
      s = warp_sum(s);
      if (lane == 0 && s != 0.0) {
        atomicAdd(acc + 4 * k0 + 2 * slot, s);
        atomicAdd(acc + 4 * k0 + 2 * slot + 1, s);
      }
    }
  } else if (d != 0.0) {
    atomicAdd(acc + 4 * k + 2 * slot, d);
    atomicAdd(acc + 4 * k + 2 * slot + 1, d);
  }
}

// Programmatic dependent launch of the step's kernels: let the next kernel of the
// step be scheduled now (its blocks take the SM slots that this grid's last wave
// frees), then wait until the kernel before this one has completed and its writes
// are visible.  Every step kernel triggers first thing and has at least one thread
// that waits (the thread of a fluid slot or of a list entry: the solid kernels are
// not launched for an empty list), so a grid completes only after its predecessor
// did, and so on back to the first kernel of the step.  Both instructions are no-ops
// for a launch without the programmatic attribute.
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
// The same in two halves, for kernels that first load what no step writes (slot
// map, node words, link words, solid normals, boundary lists): those loads are
// issued before the wait, so a block resident before its predecessor finishes
// has them in flight while it waits.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// source slots of the pull of fluid slot t at (x, y, z): the slot of x - c_i, or
// -1 where that node is solid (halfway bounce-back); the rest population's is t
__device__ __forceinline__ void pull_sources(const int *__restrict__ gidx, const PullOffsets &O, unsigned t,
                                             int (&src)[Q]) {
#pragma unroll
  for (int i = 0; i < Q - 1; ++i) src[i] = __ldg(gidx + O.src(CX[i], CY[i], CZ[i]));
  src[Q - 1] = (int)t;
}

// pull of the 45 (38) populations of fluid slot t from its source slots
template <typename T>
__device__ __forceinline__ void pull_compact(int ns_, const StepParams &P, const T *__restrict__ fin,
                                             const int (&src)[Q], unsigned t, float (&fr)[Q], float (&fp)[Q],
                                             float (&g)[Q7]) {
  const unsigned ns = (unsigned)ns_;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const bool bb = src[i] < 0;
    const unsigned s = bb ? t : (unsigned)src[i];
    const unsigned pr = bb ? (unsigned)OPP[i] : (unsigned)i;
    // the reference of population OPP[i] equals that of i (w is even in c)
    Store<T>::ld2(fin, ns, pr, s, i, fr[i], fp[i]);
  }
  if (P.reaction_mode == 0) {
#pragma unroll
    for (int j = 0; j < Q7; ++j) {
      const int d = GDIR[j];
      const bool bb = src[d] < 0;
      const unsigned s = bb ? t : (unsigned)src[d];
      const unsigned pj = bb ? (unsigned)GOPP[j] : (unsigned)j;
      g[j] = Store<T>::ld(fin, ns, 2 * Q + pj, s);
    }
  }
}

// a1 + a2 over the fluid slots: colour function rho^N (dense field)
// With BATCH false the kernel serves one lattice whose table entry travels as a
// kernel parameter (constant bank); with BATCH true each thread reads its
// lattice's entry from the table.
template <bool BATCH>
__device__ __forceinline__ const Inst &inst_of(const Slots &S, const Inst &single, int k) {
  return BATCH ? S.inst[k] : single;
}

template <typename T, int BLOCK, bool BATCH>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) k_density_c(Slots S, const __grid_constant__ Inst single,
                                                     const T *__restrict__ f, const int *__restrict__ gidx,
                                                     float *__restrict__ rhoN, double *__restrict__ acc, int n_inst,
                                                     int slot) {
  pdl_trigger();
  // The reaction-sum pairs of this step (block_delta_inst) are set up here: the
  // colour-function pass is the step's first kernel, launched after the previous step
  // has completed, and the main kernel starts only after it has.  A batch sets them
  // up in its first block, one instance per thread; one lattice, at the end of slot
  // 0's thread (the same code at the start of the kernel cost the FP16 pass 0.8 us).
  if (BATCH && acc && blockIdx.x == 0) {
    for (int k = threadIdx.x; k < n_inst; k += blockDim.x) {
      acc[4 * k + 2 * slot] = 0.0;
      acc[4 * k + 2 * slot + 1] = acc[4 * k + 2 * (slot ^ 1) + 1];
    }
  }
  // the blocks walk the slots from the end: the first ones read what the main kernel
  // of the previous step wrote last, which is still in L2 (67.5 -> 65.1 us on the
  // 128x128x256 column)
  const unsigned t = (gridDim.x - 1 - blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= (unsigned)S.nslots) return;
  const uint32_t pk = S.node[t];
  if (pk == kNoNode) return;
  const Inst &I = inst_of<BATCH>(S, single, BATCH ? slot_instance(S, t) : 0);
  int x, y, z;
  unpack(pk, x, y, z);
  PullOffsets O;
  O.init(I.L, x, y, z);
  const unsigned ns = (unsigned)S.ns;
  int src[Q];
  pull_sources(gidx + (BATCH ? I.gidx_off : 0), O, t, src);
  pdl_wait();
  float rr = 0.f, rp = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int si = src[i];
    const bool bb = si < 0;
    const unsigned s = bb ? t : (unsigned)si;
    const unsigned pr = bb ? (unsigned)OPP[i] : (unsigned)i;
    float a, b;
    Store<T>::ld2(f, ns, pr, s, i, a, b);
    rr += a;
    rp += b;
  }
  rhoN[(BATCH ? I.node_off : 0) + nidx(I.L, x, y, z)] = (rr - rp) / (rr + rp);
  if (!BATCH && acc && t == 0) {   // slot 0 is a fluid slot: its thread gets here
    acc[2 * slot] = 0.0;
    acc[2 * slot + 1] = acc[2 * (slot ^ 1) + 1];
  }
}

// a4 + a5 over the fluid slots
template <int BLOCK, bool BATCH>
__global__ void __launch_bounds__(BLOCK) k_normal_c(Slots S, const __grid_constant__ Inst single,
                                                    const float *__restrict__ rhoN, const uint32_t *__restrict__ link,
                                                    const float4 *__restrict__ ns, float4 *__restrict__ nrm) {
  pdl_trigger();
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (unsigned)S.nslots) return;
  const uint32_t pk = S.node[t];
  if (pk == kNoNode) return;
  const Inst &I = inst_of<BATCH>(S, single, BATCH ? slot_instance(S, t) : 0);
  int x, y, z;
  unpack(pk, x, y, z);
  StencilOffsets St;
  St.init(I.L, x, y, z);
  const float *rn = rhoN + (BATCH ? I.node_off : 0);
  const unsigned node = St.own;
  // the link word and the solid normal are loaded with the gathers, not after them
  // (the solid normal is needed at wall nodes only; 30.8 -> 29.2 us on the
  // 128x128x256 column)
  const int noff = BATCH ? I.node_off : 0;
  const uint32_t lk = __ldg(link + noff + node);
  const float4 s = __ldg(ns + noff + node);
  pdl_wait();
  float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
  for (int i = 0; i < Q - 1; ++i) {
    const float v = 3.0f * W[i] * rn[St.nb(CX[i], CY[i], CZ[i])];
    if (CX[i]) gx += CX[i] * v;   // zero components skipped: 0 * v does not fold away
    if (CY[i]) gy += CY[i] * v;
    if (CZ[i]) gz += CZ[i] * v;
  }
  nrm[noff + node] = wetted_normal_from(I.P, lk, [&] { return s; }, gx, gy, gz);
}

// a3 / solid normals over the list of solid nodes next to the fluid (packed
// coordinates, instance array kid or null, and each entry's link word, which
// marks in bit i whether x + c_i is fluid).  The colour average loads all 18 neighbour
// values unconditionally (every neighbour index is inside the lattice) and drops
// the solid ones by a select, so the loads are in flight together instead of one
// branch at a time (17 -> 15 us on the 128x128x256 column); for the float4
// normals the same form doubles the loaded bytes and is slower, so they keep the
// conditional loads.
template <bool BATCH>
__global__ void __launch_bounds__(128) k_color_solid_c(const Inst *__restrict__ inst, const __grid_constant__ Inst single,
                                const uint32_t *__restrict__ list, const uint16_t *__restrict__ kid, int count,
                                const uint32_t *__restrict__ list_link, float *__restrict__ rhoN) {
  pdl_trigger();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const Inst &I = BATCH ? inst[kid[t]] : single;
  int x, y, z;
  unpack(list[t], x, y, z);
  const uint32_t lk = list_link[t];   // the entry's link word, loaded beside it
  StencilOffsets St;
  St.init(I.L, x, y, z);
  float *rn = rhoN + I.node_off;
  pdl_wait();
  float v[Q - 1];
#pragma unroll
  for (int i = 0; i < Q - 1; ++i) v[i] = rn[St.nb(CX[i], CY[i], CZ[i])];
  float num = 0.f, den = 0.f;
#pragma unroll
  for (int i = 0; i < Q - 1; ++i) {
    const bool fl = (lk >> i) & 1u;
    num += fl ? W[i] * v[i] : 0.f;
    den += fl ? W[i] : 0.f;
  }
  rn[St.own] = den > 0.f ? num / den : 0.f;
}

template <bool BATCH>
__global__ void k_normal_solid_c(const Inst *__restrict__ inst, const __grid_constant__ Inst single,
                                 const uint32_t *__restrict__ list, const uint16_t *__restrict__ kid, int count,
                                 const uint32_t *__restrict__ list_link, float4 *__restrict__ nrm) {
  pdl_trigger();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const Inst &I = BATCH ? inst[kid[t]] : single;
  int x, y, z;
  unpack(list[t], x, y, z);
  const uint32_t lk = list_link[t];   // the entry's link word, loaded beside it
  StencilOffsets St;
  St.init(I.L, x, y, z);
  pdl_wait();
  float4 *nn = nrm + I.node_off;
  float ax = 0.f, ay = 0.f, az = 0.f;
#pragma unroll
  for (int i = 0; i < Q - 1; ++i) {
    if ((lk >> i) & 1u) {
      const float4 v = nn[St.nb(CX[i], CY[i], CZ[i])];
      ax += W[i] * v.x;
      ay += W[i] * v.y;
      az += W[i] * v.z;
    }
  }
  const float m = sqrtf(ax * ax + ay * ay + az * az);
  if (m >= GRAD_EPS) {
    const float inv = 1.0f / m;
    nn[St.own] = make_float4(ax * inv, ay * inv, az * inv, 0.f);
  } else {
    nn[St.own] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// ---------------------------------------------------------------------------
// a3, a4, a5 and the normals at solids in one launch, marching through z with
// shared-memory planes.  A block owns a TX x TY column of the lattice and a
// chunk of z-planes [zb, ze).  It walks the planes z = zb - 3 .. ze + 2 and
// keeps rings of the last few planes in shared memory: rho^N with a halo of
// three nodes in x and y (x, y periodic), the link words, the solid normals of
// the wall nodes and the wetted normals.  With the planes of rho^N and of the
// link words of z arriving (cp.async, issued one iteration ahead), a block
//   forms the colour at the boundary solids of plane z - 1  (Eq. color_lattice_weighted_average,
//                                                           xy box + 2),
//   the wetted normals of the fluid nodes of plane z - 2    (Eq. finite_difference_scheme,
//                                                           Eq. realigned_normal_vectors, box + 1),
//   the normals at the boundary solids of plane z - 3       (weighted average, renormalised, box),
// and writes n (with |grad rho^N|) for its fluid and boundary-solid nodes and
// rho^N at its boundary solids.  Each value is computed with the same operations
// in the same order as the separate kernels (k_color_solid_c, k_normal_c,
// k_normal_solid_c), so the two forms agree bit for bit; the halo values (the xy
// ring, three planes below and above the chunk) are recomputed by every block
// that needs them.  z is periodic or, in column mode, a node on plane 0
// (nz - 1) takes itself for its z - 1 (z + 1) neighbour; planes outside the
// lattice are then neither loaded nor computed.
template <int TX, int TY>
struct MarchTile {
  static constexpr int H = 3;                                   // xy halo of the staged planes
  static constexpr int PX = TX + 2 * H, PY = TY + 2 * H, PN = PX * PY;
  static constexpr int RING_R = 5, RING_L = 5, RING_S = 2, RING_N = 3;
  static constexpr size_t smem_bytes() {
    return sizeof(float4) * PN * RING_S + sizeof(float) * PN * RING_R + sizeof(uint32_t) * PN * RING_L +
           sizeof(float) * 3 * PN * RING_N + sizeof(int) * (PX + PY);
  }
};

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ int ring(int z, int n) { return ((z % n) + n) % n; }

// blocks of one lattice: ntx x nty columns times ceil(nz / chunk) chunks, x fastest
__device__ __forceinline__ void march_block(const Lattice &L, int tx, int ty, int chunk, int t, int &x0, int &y0,
                                            int &zb, int &ze) {
  const int ntx = (L.nx + tx - 1) / tx, nty = (L.ny + ty - 1) / ty;
  x0 = (t % ntx) * tx;
  y0 = ((t / ntx) % nty) * ty;
  zb = (t / (ntx * nty)) * chunk;
  ze = min(zb + chunk, L.nz);
}

template <int TX, int TY, bool BATCH>
__global__ void __launch_bounds__(256) k_fields_march(const Inst *__restrict__ inst, const __grid_constant__ Inst single,
                                                      const int *__restrict__ block_off, int n_inst, int chunk,
                                                      const uint32_t *__restrict__ link,
                                                      const float4 *__restrict__ ns, float *__restrict__ rhoN,
                                                      float4 *__restrict__ nrm) {
  using MT = MarchTile<TX, TY>;
  constexpr int H = MT::H, PX = MT::PX, PY = MT::PY, PN = MT::PN;
  pdl_begin();
  extern __shared__ __align__(16) unsigned char msm[];
  float4 *S = reinterpret_cast<float4 *>(msm);                  // solid normals (+ angle) of wall nodes
  float *R = reinterpret_cast<float *>(S + PN * MT::RING_S);    // rho^N; colour at boundary solids
  uint32_t *Lk = reinterpret_cast<uint32_t *>(R + PN * MT::RING_R);
  float *N = reinterpret_cast<float *>(Lk + PN * MT::RING_L);   // wetted normals, 3 components per plane
  int *xs = reinterpret_cast<int *>(N + 3 * PN * MT::RING_N);
  int *ys = xs + PX;
  int k = 0, t = blockIdx.x;
  if (BATCH) {
    int lo = 0, hi = n_inst - 1;                                 // last k with block_off[k] <= blockIdx.x
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (block_off[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    k = lo;
    t = blockIdx.x - block_off[k];
  }
  const Inst &I = BATCH ? inst[k] : single;
  const Lattice &L = I.L;
  int x0, y0, zb, ze;
  march_block(L, TX, TY, chunk, t, x0, y0, zb, ze);
  const bool clampz = L.bc_z != 0;
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int c = tid; c < PX + PY; c += nth) {
    if (c < PX)
      xs[c] = ((x0 + c - H) % L.nx + L.nx) % L.nx;
    else
      ys[c - PX] = ((y0 + c - PX - H) % L.ny + L.ny) % L.ny;
  }
  __syncthreads();
  const uint32_t *lk_ = link + I.node_off;
  const float4 *ns_ = ns + I.node_off;
  float *rn = rhoN + I.node_off;
  float4 *nn = nrm + I.node_off;
  const long long nx = L.nx, plane = L.plane;
  auto exists = [&](int z) { return !clampz || (z >= 0 && z < L.nz); };
  auto gplane = [&](int z) { return (long long)(clampz ? z : ring(z, L.nz)) * plane; };
  auto zdn = [&](int z) { return (clampz && z == 0) ? z : z - 1; };
  auto zup = [&](int z) { return (clampz && z == L.nz - 1) ? z : z + 1; };
  // rho^N of plane z (xy box + 3) and its link words (box + 2)
  auto load_plane = [&](int z) {
    if (!exists(z)) return;
    const long long zo = gplane(z);
    float *Rs = R + ring(z, MT::RING_R) * PN;
    uint32_t *Ls = Lk + ring(z, MT::RING_L) * PN;
    for (int c = tid; c < PN; c += nth) {
      const int i = c % PX, j = c / PX;
      const long long g = zo + ys[j] * nx + xs[i];
      cp_async4(Rs + c, rn + g);
      if (i >= 1 && i < PX - 1 && j >= 1 && j < PY - 1) cp_async4(Ls + c, lk_ + g);
    }
  };
  // solid normals of plane z (box + 1; zero away from wall nodes)
  auto load_solid = [&](int z) {
    if (!exists(z)) return;
    const long long zo = gplane(z);
    float4 *Ss = S + ring(z, MT::RING_S) * PN;
    for (int c = tid; c < PN; c += nth) {
      const int i = c % PX, j = c / PX;
      if (i >= 2 && i < PX - 2 && j >= 2 && j < PY - 2) cp_async16(Ss + c, ns_ + zo + ys[j] * nx + xs[i]);
    }
  };
  auto owned = [&](int i, int j) {
    return i >= H && i < H + TX && j >= H && j < H + TY && x0 + i - H < L.nx && y0 + j - H < L.ny;
  };
  load_plane(zb - 3);
  cp_async_commit();
  for (int zl = zb - 3; zl <= ze + 2; ++zl) {
    cp_async_wait_all();
    __syncthreads();   // plane zl (rho^N, links) and the solid normals of plane zl - 2 have landed
    if (zl + 1 <= ze + 2) load_plane(zl + 1);
    if (zl - 1 >= zb - 1 && zl - 1 <= ze) load_solid(zl - 1);
    cp_async_commit();
    // colour at the boundary solids of plane zc = zl - 1, box + 2
    const int zc = zl - 1;
    if (zc >= zb - 2 && exists(zc)) {
      float *Rc = R + ring(zc, MT::RING_R) * PN;
      const float *Rd = R + ring(zdn(zc), MT::RING_R) * PN, *Ru = R + ring(zup(zc), MT::RING_R) * PN;
      const uint32_t *Lc = Lk + ring(zc, MT::RING_L) * PN;
      for (int c = tid; c < PN; c += nth) {
        const int i = c % PX, j = c / PX;
        if (i < 1 || i >= PX - 1 || j < 1 || j >= PY - 1) continue;
        const uint32_t lk = Lc[c];
        if (!(lk & BIT_SOLID_BND)) continue;
        float num = 0.f, den = 0.f;
#pragma unroll
        for (int d = 0; d < Q - 1; ++d) {
          const bool fl = (lk >> d) & 1u;
          const float *Rp = CZ[d] < 0 ? Rd : (CZ[d] > 0 ? Ru : Rc);
          const float v = fl ? Rp[c + CX[d] + CY[d] * PX] : 0.f;   // fluid cells only: never written here
          num += fl ? W[d] * v : 0.f;
          den += fl ? W[d] : 0.f;
        }
        Rc[c] = den > 0.f ? num / den : 0.f;
      }
    }
    __syncthreads();
    // wetted normals of the fluid nodes of plane zn = zl - 2, box + 1
    const int zn = zl - 2;
    if (zn >= zb - 1 && exists(zn)) {
      const float *Rc = R + ring(zn, MT::RING_R) * PN;
      const float *Rd = R + ring(zdn(zn), MT::RING_R) * PN, *Ru = R + ring(zup(zn), MT::RING_R) * PN;
      const uint32_t *Lc = Lk + ring(zn, MT::RING_L) * PN;
      const float4 *Ss = S + ring(zn, MT::RING_S) * PN;
      float *Nx = N + ring(zn, MT::RING_N) * 3 * PN, *Ny = Nx + PN, *Nz = Ny + PN;
      const long long zo = gplane(zn);
      const bool out = zn >= zb && zn < ze;
      for (int c = tid; c < PN; c += nth) {
        const int i = c % PX, j = c / PX;
        if (i < 2 || i >= PX - 2 || j < 2 || j >= PY - 2) continue;
        const uint32_t lk = Lc[c];
        float4 n = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!(lk & BIT_SOLID)) {
          float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
          for (int d = 0; d < Q - 1; ++d) {
            const float *Rp = CZ[d] < 0 ? Rd : (CZ[d] > 0 ? Ru : Rc);
            const float v = 3.0f * W[d] * Rp[c + CX[d] + CY[d] * PX];
            if (CX[d]) gx += CX[d] * v;
            if (CY[d]) gy += CY[d] * v;
            if (CZ[d]) gz += CZ[d] * v;
          }
          n = wetted_normal_from(I.P, lk, [&] { return Ss[c]; }, gx, gy, gz);
          if (out && owned(i, j)) nn[zo + ys[j] * nx + xs[i]] = n;
        }
        Nx[c] = n.x;
        Ny[c] = n.y;
        Nz[c] = n.z;
      }
    }
    __syncthreads();
    // normals at the boundary solids of plane zs = zl - 3, box
    const int zs = zl - 3;
    if (zs >= zb && exists(zs)) {
      const uint32_t *Lc = Lk + ring(zs, MT::RING_L) * PN;
      const float *Rc = R + ring(zs, MT::RING_R) * PN;
      const float *Nc = N + ring(zs, MT::RING_N) * 3 * PN;
      const float *Nd = N + ring(zdn(zs), MT::RING_N) * 3 * PN, *Nu = N + ring(zup(zs), MT::RING_N) * 3 * PN;
      const long long zo = gplane(zs);
      for (int c = tid; c < PN; c += nth) {
        const int i = c % PX, j = c / PX;
        if (!owned(i, j)) continue;
        const uint32_t lk = Lc[c];
        if (!(lk & BIT_SOLID_BND)) continue;
        float ax = 0.f, ay = 0.f, az = 0.f;
#pragma unroll
        for (int d = 0; d < Q - 1; ++d) {
          if ((lk >> d) & 1u) {
            const float *Np = CZ[d] < 0 ? Nd : (CZ[d] > 0 ? Nu : Nc);
            const int q = c + CX[d] + CY[d] * PX;
            ax += W[d] * Np[q];
            ay += W[d] * Np[PN + q];
            az += W[d] * Np[2 * PN + q];
          }
        }
        const float m = sqrtf(ax * ax + ay * ay + az * az);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (m >= GRAD_EPS) {
          const float inv = 1.0f / m;
          v = make_float4(ax * inv, ay * inv, az * inv, 0.f);
        }
        const long long g = zo + ys[j] * nx + xs[i];
        nn[g] = v;
        rn[g] = Rc[c];
      }
    }
  }
  cp_async_wait_all();
}

// outlet ghost (column mode) of slot gs from the post-collision populations of a
// fluid node of plane nz - 1 (same arithmetic as write_outlet_ghost)
template <typename T>
__device__ __forceinline__ void write_outlet_ghost_c(int ns_, T *__restrict__ f, unsigned gs, const float (&fr)[Q],
                                                     const float (&fp)[Q], float g5, float rho_out, uint32_t seed) {
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
  const unsigned ns = (unsigned)ns_;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (CZ[i] != -1) continue;
    const float corr = feq19(i, rho_out - rho, vx, vy, vz, vv);
    Store<T>::st_r(f, ns, i, gs, fr[i] + psi * corr, pop_random(seed, NPOP + i));
    Store<T>::st_r(f, ns, Q + i, gs, fp[i] + (1.0f - psi) * corr, pop_random(seed, NPOP + Q + i));
  }
  Store<T>::st_r(f, ns, 2 * Q + 5, gs, g5, pop_random(seed, NPOP + 2 * Q + 5));
}

// a1, a2, a6 - a10 over the fluid slots; stores are coalesced and whole-sector.
// acc holds 4 doubles per instance: cumulative delta, unused, per-step slots 0/1.
template <typename T, int BLOCK, bool BATCH>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) k_main_c(Slots S, const __grid_constant__ Inst single,
                                                               int n_inst, const T *__restrict__ fin,
                                                               T *__restrict__ fout, const int *__restrict__ gidx,
                                                               const uint32_t *__restrict__ link,
                                                               const float4 *__restrict__ nrm, double *__restrict__ acc,
                                                               int slot, uint32_t *__restrict__ rstep,
                                                               float *__restrict__ dbg_H,
                                                               float *__restrict__ dbg_delta) {
  pdl_trigger();
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = BATCH ? slot_instance(S, t < (unsigned)S.nslots ? t : (unsigned)S.nslots - 1) : 0;
  const uint32_t pk = t < (unsigned)S.nslots ? S.node[t] : kNoNode;
  // FP16 storage: the source slots and the link word are loaded before the wait
  // (step 223.9 -> 221.4 us on the 128x128x256 column); FP32 storage loads them after
  // the curvature, as holding the 18 sources across it spills at 64 registers (the
  // step 0.6 % slower)
  constexpr bool EARLY = std::is_same<T, __half>::value;
  int src[Q];
  uint32_t lk = 0;
  if (EARLY && pk != kNoNode) {
    const Inst &I = inst_of<BATCH>(S, single, k);
    int x, y, z;
    unpack(pk, x, y, z);
    PullOffsets O;
    O.init(I.L, x, y, z);
    pull_sources(gidx + (BATCH ? I.gidx_off : 0), O, t, src);
    lk = __ldg(link + (BATCH ? I.node_off : 0) + nidx(I.L, x, y, z));
  }
  pdl_wait();
  // step counter of the FP16 rounding: read from this step's slot, the next value
  // written to the other one (read by the next step's main kernel)
  const uint32_t step = rstep[slot];
  if (blockIdx.x == 0 && threadIdx.x == 0) rstep[slot ^ 1] = step + 1u;
  double dsum[1] = {0.0};
  if (pk != kNoNode) {
    const Inst &I = inst_of<BATCH>(S, single, k);
    int x, y, z;
    unpack(pk, x, y, z);
    StencilOffsets St;
    St.init(I.L, x, y, z);
    const unsigned node = St.own;
    const int noff = BATCH ? I.node_off : 0;
    const float4 *nn = nrm + noff;
    if (!EARLY) lk = link[noff + node];
    const float4 nme = nn[node];
    constexpr bool LEAN = std::is_same<T, __half>::value;
    const float H =
        nme.w >= GRAD_EPS ? curvature<LEAN>(nme, [&](int i) { return nn[St.nb(CX[i], CY[i], CZ[i])]; }) : 0.f;
    if (!EARLY) {
      PullOffsets O;
      O.init(I.L, x, y, z);
      pull_sources(gidx + (BATCH ? I.gidx_off : 0), O, t, src);
    }
    float fr[Q], fp[Q], g[Q7];
    pull_compact<T>(S.ns, I.P, fin, src, t, fr, fp, g);
    const float delta = collide_node<LEAN>(I.P, lk, fr, fp, g, nme, H);
    const unsigned ns = (unsigned)S.ns;
    // FP16 rounding bits (unused for FP32); fr + fp of the rest population sums rho
    // and, in reaction mode 0, g[6] carries C: both enter the finiteness check
    const uint32_t seed = node_seed(fr[Q - 1] + fp[Q - 1] + (I.P.reaction_mode == 0 ? g[Q7 - 1] : 0.f), t, step);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      Store<T>::st2_r(fout, ns, i, t, fr[i], fp[i], pop_random(seed, i));
    }
    float g5;
    if (I.P.reaction_mode == 0) {
#pragma unroll
      for (int j = 0; j < Q7; ++j)
        Store<T>::st_r(fout, ns, 2 * Q + j, t, g[j], pop_random(seed, 2 * Q + j));
      g5 = g[5];
    } else {
      g5 = Store<T>::ld(fin, ns, 2 * Q + 5, t);
    }
    if (I.L.bc_z == 1 && z == I.L.nz - 1) {
      const unsigned gs = (unsigned)(I.ghost + I.L.plane) + (unsigned)(y * I.L.nx + x);
      write_outlet_ghost_c<T>(S.ns, fout, gs, fr, fp, g5, I.P.rho_out, seed);
    }
    if (dbg_H) dbg_H[noff + node] = H;
    if (dbg_delta) dbg_delta[noff + node] = delta;
    dsum[0] = (double)delta;
  }
  // per instance: this step's sum and the cumulative sum, acc[4k + 2 slot] and acc[4k + 2 slot + 1]
  block_delta_inst<BATCH>(dsum[0], k, acc, slot);
}

// equilibrium start of instance I's fluid slots from dense fields (null: uniform values)
template <typename T>
__global__ void k_init_c(Inst I, int ns_, const uint32_t *__restrict__ node, const float *__restrict__ rho_r,
                         const float *__restrict__ rho_p, const float *__restrict__ conc, const float *__restrict__ u,
                         float rr0, float rp0, float c0, T *__restrict__ fa, T *__restrict__ fb) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= I.nf) return;
  const unsigned t = (unsigned)(I.slot_off + l);
  int x, y, z;
  unpack(node[t], x, y, z);
  const long long nd = nidx(I.L, x, y, z);
  const float rr = rho_r ? rho_r[nd] : rr0;
  const float rp = rho_p ? rho_p[nd] : rp0;
  const float cc = conc ? conc[nd] : c0;
  const float ux = u ? u[nd] : 0.f, uy = u ? u[I.L.n + nd] : 0.f, uz = u ? u[2 * I.L.n + nd] : 0.f;
  const float uu = ux * ux + uy * uy + uz * uz;
  const unsigned ns = (unsigned)ns_;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float a = feq19(i, rr, ux, uy, uz, uu), b = feq19(i, rp, ux, uy, uz, uu);
    Store<T>::st(fa, ns, i, t, a);
    Store<T>::st(fb, ns, i, t, a);
    Store<T>::st(fa, ns, Q + i, t, b);
    Store<T>::st(fb, ns, Q + i, t, b);
  }
#pragma unroll
  for (int j = 0; j < Q7; ++j) {
    const int d = GDIR[j];
    const float gv = W7[j] * cc * (1.0f + 4.0f * (CX[d] * ux + CY[d] * uy + CZ[d] * uz));
    Store<T>::st(fa, ns, 2 * Q + j, t, gv);
    Store<T>::st(fb, ns, 2 * Q + j, t, gv);
  }
}

// Column ghost slots of instance I in both buffers: constant inlet, outlet from
// plane nz - 1 of fa (resting reactant equilibrium above solid nodes).
template <typename T>
__global__ void k_ghost_init_c(Inst I, int ns_, const int *__restrict__ gidx, float u_in, float c_in, float rho_out,
                               T *__restrict__ fa, T *__restrict__ fb) {
  const Lattice &L = I.L;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= L.nx || y >= L.ny) return;
  const unsigned ns = (unsigned)ns_;
  const unsigned gin = (unsigned)I.ghost + (unsigned)(y * L.nx + x);
  const unsigned gout = gin + (unsigned)L.plane;
  const float uu = u_in * u_in;
#pragma unroll
  for (int p = 0; p < NPOP; ++p) {
    Store<T>::st(fa, ns, p, gin, 0.f);
    Store<T>::st(fb, ns, p, gin, 0.f);
    Store<T>::st(fa, ns, p, gout, 0.f);
    Store<T>::st(fb, ns, p, gout, 0.f);
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (CZ[i] != 1) continue;
    const float v = feq19(i, 1.0f, 0.f, 0.f, u_in, uu);
    Store<T>::st(fa, ns, i, gin, v);
    Store<T>::st(fb, ns, i, gin, v);
  }
  const float g4 = W7[4] * c_in * (1.0f + 4.0f * u_in);
  Store<T>::st(fa, ns, 2 * Q + 4, gin, g4);
  Store<T>::st(fb, ns, 2 * Q + 4, gin, g4);
  const int s = gidx[I.gidx_off + (long long)L.nz * L.plane + (long long)y * L.nx + x];   // z = nz - 1
  if (s < 0) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (CZ[i] != -1) continue;
      Store<T>::st(fa, ns, i, gout, W[i] * rho_out);
      Store<T>::st(fb, ns, i, gout, W[i] * rho_out);
    }
  } else {
    float fr[Q], fp[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      Store<T>::ld2(fa, ns, i, (unsigned)s, i, fr[i], fp[i]);
    }
    const float g5 = Store<T>::ld(fa, ns, 2 * Q + 5, (unsigned)s);
    write_outlet_ghost_c<T>(ns_, fa, gout, fr, fp, g5, rho_out,
                            node_seed(fr[Q - 1] + fp[Q - 1] + g5, gout, 0xFFFFFFFFu));
  }
}

// a11 over the fluid slots (FP32 per node, FP64 block accumulation per instance).
// obs holds 8 doubles per instance: mass_r, mass_p, mass_c, sum (1 - rho^N)/2,
// flux_in, flux_out, n_bad.
template <typename T, bool BATCH>
__global__ void k_observables_c(Slots S, const __grid_constant__ Inst single, const T *__restrict__ f,
                                double *__restrict__ obs) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  double v[7] = {0, 0, 0, 0, 0, 0, 0};
  const int k = BATCH ? slot_instance(S, t < (unsigned)S.nslots ? t : (unsigned)S.nslots - 1) : 0;
  const uint32_t pk = t < (unsigned)S.nslots ? S.node[t] : kNoNode;
  if (pk != kNoNode) {
    const Inst &I = inst_of<BATCH>(S, single, k);
    int x, y, z;
    unpack(pk, x, y, z);
    const unsigned ns = (unsigned)S.ns;
    float rr = 0.f, rp = 0.f, cc = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      float a, b;
      Store<T>::ld2(f, ns, i, t, i, a, b);
      rr += a;
      rp += b;
      if (CZ[i]) jz += CZ[i] * (a + b);
    }
#pragma unroll
    for (int j = 0; j < Q7; ++j) cc += Store<T>::ld(f, ns, 2 * Q + j, t);
    const float rho = rr + rp;
    v[0] = rr;
    v[1] = rp;
    v[2] = cc;
    const bool bad = !(rho > 0.f) || !isfinite(rho) || !isfinite(cc);
    if (!bad) {
      v[3] = 0.5f * (1.0f - (rr - rp) / rho);
      if (z == 0) v[4] = jz / rho * cc;
      if (z == I.L.nz - 1) v[5] = jz / rho * cc;
    }
    v[6] = bad ? 1.0 : 0.0;
  }
  block_accumulate_inst<7>(v, k, obs, 8);
}

}  // namespace cglbm
