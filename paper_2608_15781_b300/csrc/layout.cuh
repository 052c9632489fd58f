// Slot space of a lattice, built on the GPU from its link words (one-time set-up).
//
// Fluid nodes get consecutive slots in lattice order (x fastest, then y, then z),
// solid nodes next to the fluid get consecutive entries of the boundary-solid
// list in the same order, and in column mode the two ghost planes follow the
// fluid slots.  Three passes over the dense nodes of one lattice, in blocks of
// kLayoutBlock nodes: count (fluid, boundary-solid and wall nodes per block),
// scan (exclusive prefix of the block counts, one block of threads), fill (each
// node's rank inside its block from warp ballots, plus the block's prefix).
// The result is the same layout as one sequential pass over the nodes.
#pragma once
#include <cstdint>

#include "compact.cuh"

namespace cglbm {

constexpr int kLayoutBlock = 256;   // nodes per block of the count and fill passes (= threads)

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Exclusive rank of flag within the block and the block's total (blockDim.x = kLayoutBlock).
__device__ __forceinline__ int block_rank(bool flag, int &total) {
  __shared__ int wsum[kLayoutBlock / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned bal = __ballot_sync(0xffffffffu, flag);
  if (lane == 0) wsum[warp] = __popc(bal);
  __syncthreads();
  int before = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < kLayoutBlock / 32; ++w) {
    before += w < warp ? wsum[w] : 0;
    tot += wsum[w];
  }
  __syncthreads();   // wsum may be reused by the next call
  total = tot;
  return before + __popc(bal & lanemask_lt());
}

// per block: fluid, boundary-solid and wall node counts
__global__ void __launch_bounds__(kLayoutBlock) k_layout_count(long long n, const uint32_t *__restrict__ link,
                                                               int *__restrict__ cf, int *__restrict__ cb,
                                                               int *__restrict__ cw) {
  const long long node = (long long)blockIdx.x * kLayoutBlock + threadIdx.x;
  const uint32_t lk = node < n ? link[node] : BIT_SOLID;
  int tf, tb, tw;
  block_rank(node < n && !(lk & BIT_SOLID), tf);
  block_rank(node < n && (lk & BIT_SOLID_BND), tb);
  block_rank(node < n && !(lk & BIT_SOLID) && (lk & BIT_WALL), tw);
  if (threadIdx.x == 0) {
    cf[blockIdx.x] = tf;
    cb[blockIdx.x] = tb;
    cw[blockIdx.x] = tw;
  }
}

// exclusive prefix of cf and cb over nb blocks (in place); totals of cf, cb, cw into tot[0..2].
// One block of 1024 threads: thread j sums its own run of ceil(nb / 1024) consecutive
// entries, the block scans the 1024 run sums, and each thread rewrites its run from
// its run's offset.
__device__ __forceinline__ long long block_exclusive_scan_1024(long long v, long long &total) {
  __shared__ long long wsum[32];
  __shared__ long long wtot;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const long long w = wsum[lane];
    long long wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long u = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += u;
    }
    wsum[lane] = wi - w;   // exclusive prefix of the warp sums
    if (lane == 31) wtot = wi;
  }
  __syncthreads();
  const long long r = wsum[warp] + incl - v;
  total = wtot;
  __syncthreads();   // wsum and wtot may be reused by the next call
  return r;
}

__global__ void __launch_bounds__(1024) k_layout_scan(int nb, int *__restrict__ cf, int *__restrict__ cb,
                                                      const int *__restrict__ cw, long long *__restrict__ tot) {
  const int run = (nb + 1023) / 1024;
  const int i0 = min(nb, (int)threadIdx.x * run), i1 = min(nb, i0 + run);
  long long sf = 0, sb = 0, sw = 0;
  for (int i = i0; i < i1; ++i) {
    sf += cf[i];
    sb += cb[i];
    sw += cw[i];
  }
  long long tf, tb, tw;
  long long of = block_exclusive_scan_1024(sf, tf);
  long long ob = block_exclusive_scan_1024(sb, tb);
  (void)block_exclusive_scan_1024(sw, tw);
  for (int i = i0; i < i1; ++i) {
    const int vf = cf[i], vb = cb[i];
    cf[i] = (int)of;
    cb[i] = (int)ob;
    of += vf;
    ob += vb;
  }
  if (threadIdx.x == 0) {
    tot[0] = tf;
    tot[1] = tb;
    tot[2] = tw;
  }
}

// Slots of instance k: gidx (lattice planes 0 .. nz - 1 at gi + plane), packed node
// coordinates and instance of each fluid slot, boundary-solid list with each entry's
// link word (read next to the entry by the solid kernels) and its instances.
__global__ void __launch_bounds__(kLayoutBlock) k_layout_fill(Lattice L, int k, int slot_off, int bnd_off,
                                                              const uint32_t *__restrict__ link,
                                                              const int *__restrict__ cf, const int *__restrict__ cb,
                                                              int *__restrict__ gi, uint32_t *__restrict__ node,
                                                              uint16_t *__restrict__ kid, uint32_t *__restrict__ bnd,
                                                              uint32_t *__restrict__ bnd_link,
                                                              uint16_t *__restrict__ bnd_kid) {
  const long long i = (long long)blockIdx.x * kLayoutBlock + threadIdx.x;
  const bool in = i < L.n;
  const uint32_t lk = in ? link[i] : BIT_SOLID;
  const bool fluid = in && !(lk & BIT_SOLID), bs = in && (lk & BIT_SOLID_BND);
  int tf, tb;
  const int rf = block_rank(fluid, tf), rb = block_rank(bs, tb);
  if (!in) return;
  const int x = (int)(i % L.nx), y = (int)((i / L.nx) % L.ny), z = (int)(i / L.plane);
  const uint32_t pk = (uint32_t)x | ((uint32_t)y << 10) | ((uint32_t)z << 20);
  if (fluid) {
    const int s = slot_off + cf[blockIdx.x] + rf;
    gi[L.plane + i] = s;
    node[s] = pk;
    if (kid) kid[s] = (uint16_t)k;
  } else {
    gi[L.plane + i] = -1;
    if (bs) {
      const int b = bnd_off + cb[blockIdx.x] + rb;
      bnd[b] = pk;
      bnd_link[b] = lk;
      if (bnd_kid) bnd_kid[b] = (uint16_t)k;
    }
  }
}

// the slot-map planes z = -1 and z = nz of instance k (ghost slots in column mode,
// -1 in a periodic box) and the ghost slots' node words and instance
__global__ void k_layout_ghosts(Lattice L, int k, int ghost, int *__restrict__ gi, uint32_t *__restrict__ node,
                                uint16_t *__restrict__ kid) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= L.plane) return;
  const bool col = L.bc_z == 1;
  gi[q] = col ? (int)(ghost + q) : -1;
  gi[(long long)(L.nz + 1) * L.plane + q] = col ? (int)(ghost + L.plane + q) : -1;
  if (col) {
    node[ghost + q] = kNoNode;
    node[ghost + L.plane + q] = kNoNode;
    if (kid) {
      kid[ghost + q] = (uint16_t)k;
      kid[ghost + L.plane + q] = (uint16_t)k;
    }
  }
}

// every slot-map entry is a slot of the space or -1; bad entries set *err
__global__ void k_layout_check(long long count, const int *__restrict__ gi, int nslots, int *__restrict__ err) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < count && (gi[q] < -1 || gi[q] >= nslots)) atomicOr(err, 1);
}

// populations of instance I's fluid slots (storage type T) <-> FP32 dense [45][n] arrays
template <typename T>
__global__ void k_slots_to_dense(Inst I, int ns_, const uint32_t *__restrict__ node, const T *__restrict__ src,
                                 float *__restrict__ dst) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= I.nf) return;
  const unsigned t = (unsigned)(I.slot_off + l);
  int x, y, z;
  unpack(node[t], x, y, z);
  const long long nd = nidx(I.L, x, y, z);
#pragma unroll
  for (int p = 0; p < NPOP; ++p) dst[(long long)p * I.L.n + nd] = Store<T>::ld(src, (unsigned)ns_, p, t);
}
// an adjoint array (population-major p * ns + t, not the state's slot layout) -> dense
__global__ void k_soa_to_dense(Inst I, int ns_, const uint32_t *__restrict__ node, const float *__restrict__ src,
                               float *__restrict__ dst) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= I.nf) return;
  const unsigned t = (unsigned)(I.slot_off + l);
  int x, y, z;
  unpack(node[t], x, y, z);
  const long long nd = nidx(I.L, x, y, z);
#pragma unroll
  for (int p = 0; p < NPOP; ++p) dst[(long long)p * I.L.n + nd] = src[(unsigned)p * (unsigned)ns_ + t];
}
template <typename T>
__global__ void k_dense_to_slots(Inst I, int ns_, const uint32_t *__restrict__ node, const float *__restrict__ src,
                                 T *__restrict__ a, T *__restrict__ b) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= I.nf) return;
  const unsigned t = (unsigned)(I.slot_off + l);
  int x, y, z;
  unpack(node[t], x, y, z);
  const long long nd = nidx(I.L, x, y, z);
#pragma unroll
  for (int p = 0; p < NPOP; ++p) {
    const float v = src[(long long)p * I.L.n + nd];
    Store<T>::st(a, (unsigned)ns_, p, t, v);
    Store<T>::st(b, (unsigned)ns_, p, t, v);
  }
}

}  // namespace cglbm
