// Host side of the C ABI declared in include/cglbm.h: batches of lattices in the
// compact slot layout (a single context is a batch of one), the launch sequence
// of one time step (optionally replayed as a CUDA graph), observables, state
// transfer, launch-shape tuning, profiling, and the allocation-free step.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <memory>
#include <new>
#include <type_traits>
#include <vector>

#include "adjoint.cuh"
#include "cglbm.h"
#include "compact.cuh"
#include "layout.cuh"
#include "kernels.cuh"

using namespace cglbm;

namespace {

struct InstHost {
  Inst d{};                           // the instance's device-table entry
  lbm_params prm{};
  long long n_fluid = 0, n_wall = 0, n_bnd = 0;
  double mc0 = 0.0;                   // reactant mass when the state was set
};

// One or more independent lattices sharing one slot space (see compact.cuh).
struct Batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool half = false;                  // FP16 deviation storage
  int n = 0;
  std::vector<InstHost> h;
  // slot space
  Inst *inst = nullptr;
  uint16_t *kid = nullptr;            // instance of each slot (null for one instance)
  uint32_t *node = nullptr;           // packed coordinates of each slot
  int nslots = 0, ns = 0;
  void *fa = nullptr, *fb = nullptr, *buf0 = nullptr, *buf1 = nullptr;
  int *gidx = nullptr;
  // dense per-node fields of all instances
  uint32_t *link = nullptr;
  float4 *nsv = nullptr, *nrm = nullptr;
  float *rhoN = nullptr;
  long long nodes = 0;
  uint32_t *bnd = nullptr, *bnd_link = nullptr;   // boundary-solid list and each entry's link word
  uint16_t *bnd_kid = nullptr;
  int n_bnd = 0;
  double *acc = nullptr, *acc_scratch = nullptr, *obs = nullptr;
  int *err = nullptr;
  uint32_t *rstep = nullptr;          // step counter of the FP16 rounding bits (two entries, by step parity)
  float *dbg_H = nullptr, *dbg_delta = nullptr;
  bool debug = false;
  float *h_out = nullptr;             // the main kernel's curvature per node, when set (adjoint recompute)
  size_t device_bytes = 0;
  int64_t step = 0;
  int sticky = LBM_OK;
  // launch shapes (lbm_tune picks them by timing)
  int main_block = 128, dens_block = 256, norm_block = 256;
  bool pdl = true;                    // programmatic dependent launch of the step's kernels after the first
  int fields = 0;                     // 0: colour, normals, solid normals as three kernels; 1, 2, 3: one
                                      // z-marching launch with chunks of kChunk[fields - 1] planes
  int *block_off = nullptr;           // first marching block of each instance, per chunk option ((n + 1) x 3)
  int n_blocks[3] = {0, 0, 0};        // marching blocks of all instances, per chunk option
  // CUDA graphs of one step, for even and odd steps
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  bool graphs_valid = false;
  // profiling
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_kind;
  size_t ev_used = 0;
  bool profiling = false;
  // reverse mode (lbm_adjoint_forward / lbm_adjoint_backward)
  struct Adj {
    std::vector<float *> cp;      // checkpoints f_{sK}, s = 0 .. nseg - 1
    std::vector<float *> store;   // the states of one segment, recomputed
    std::vector<float *> seg_rhoN;     // rho^N of each state of the segment (dense)
    std::vector<float4 *> seg_nrm;     // wetted normals and |grad rho^N| of each state
    std::vector<float *> seg_H;        // curvature H of each state (written by the recompute's main kernel)
    float *lam0 = nullptr, *lam1 = nullptr;   // slot-space adjoints (without their density terms)
    float *hbar = nullptr, *rho = nullptr, *rnbar = nullptr;   // dense per-node fields
    float4 *nbar = nullptr;
    float2 *coef = nullptr;
    double *thbar = nullptr, *uin = nullptr;
    size_t bytes = 0;
    int64_t nsteps = 0, K = 0, nseg = 0, end_step = -1;
    double phi_in = 0.0, phi_out = 0.0;
    bool ready = false;
  } adj;
};

}  // namespace

struct lbm_ctx {
  Batch b;
};
struct lbm_batch {
  Batch b;
};

namespace {

int cuda_fail(Batch &b, cudaError_t e) {
  if (e == cudaSuccess) return LBM_OK;
  b.sticky = LBM_ECUDA;
  return e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
}

#define CK(call)                                     \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_fail(b, e_);  \
  } while (0)

int dalloc(Batch &b, void **p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    (void)cudaGetLastError();
    return LBM_ENOMEM;
  }
  b.device_bytes += bytes;
  return LBM_OK;
}

dim3 node_block() { return dim3(kGeomBX, kGeomBY, 1); }   // k_geom stages its tile for this shape
dim3 node_grid(const Lattice &L) { return dim3((L.nx + 31) / 32, (L.ny + 3) / 4, L.nz); }

void prof_begin(Batch &b, int kind, cudaStream_t st) {
  if (!b.profiling || b.ev_used + 2 > b.ev.size()) return;
  cudaEventRecord(b.ev[b.ev_used], st);
  b.ev_kind[b.ev_used / 2] = kind;
}
void prof_end(Batch &b, cudaStream_t st) {
  if (!b.profiling || b.ev_used + 2 > b.ev.size()) return;
  cudaEventRecord(b.ev[b.ev_used + 1], st);
  b.ev_used += 2;
}

void drop_graphs(Batch &b) {
  for (auto &g : b.graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  b.graphs_valid = false;
}

void free_all(Batch &b) {
  drop_graphs(b);
  void *ptrs[] = {b.inst, b.kid, b.node, b.buf0, b.buf1, b.gidx, b.link, b.nsv, b.nrm, b.rhoN, b.bnd, b.bnd_link, b.bnd_kid,
                  b.acc, b.acc_scratch, b.obs, b.err, b.rstep, b.dbg_H, b.dbg_delta, b.block_off};
  for (void *p : ptrs) cudaFree(p);
  for (cudaEvent_t e : b.ev) cudaEventDestroy(e);
  b.ev.clear();
  Batch::Adj &a = b.adj;
  for (float *p : a.cp) cudaFree(p);
  for (float *p : a.store) cudaFree(p);
  for (float *p : a.seg_rhoN) cudaFree(p);
  for (float4 *p : a.seg_nrm) cudaFree(p);
  for (float *p : a.seg_H) cudaFree(p);
  void *aptrs[] = {a.lam0, a.lam1, a.hbar, a.rho, a.rnbar, a.nbar, a.coef, a.thbar, a.uin};
  for (void *p : aptrs) cudaFree(p);
  a = Batch::Adj{};
}

int check_params(const lbm_params *p) {
  if (!p) return LBM_EINVAL;
  if (!(p->tau > 0.5) || !std::isfinite(p->tau)) return LBM_EINVAL;
  if (!(p->diffusivity > 0.0) || !std::isfinite(p->diffusivity)) return LBM_EINVAL;
  if (!(p->beta >= 0.0) || !std::isfinite(p->sigma) || !std::isfinite(p->theta_deg)) return LBM_EINVAL;
  if (p->reaction_mode != 0 && p->reaction_mode != 1) return LBM_EINVAL;
  if (p->storage != 0 && p->storage != 1) return LBM_EINVAL;
  if (!(p->k_rate >= 0.0) || !(p->xi >= 0.0) || !(p->rho_out > 0.0)) return LBM_EINVAL;
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(p->accel[a])) return LBM_EINVAL;
  return LBM_OK;
}

int check_geometry(const lbm_geometry *g) {
  if (!g || !g->solid) return LBM_EINVAL;
  if (g->nx < 1 || g->ny < 1 || g->nz < 1) return LBM_EINVAL;
  if (g->bc_z != 0 && g->bc_z != 1) return LBM_EINVAL;
  if (g->bc_z == 1 && g->nz < 2) return LBM_EINVAL;
  // packed slot coordinates (10 + 10 + 11 bits)
  if (g->nx > 1024 || g->ny > 1024 || g->nz > 2048) return LBM_EINVAL;
  return LBM_OK;
}

float theta_rad(const lbm_params &p) { return (float)(p.theta_deg * 3.14159265358979323846 / 180.0); }

StepParams make_step_params(const lbm_params &p) {
  StepParams s{};
  s.omega_cm = (float)(1.0 - 1.0 / p.tau);
  s.half_sigma = (float)(0.5 * p.sigma);
  s.beta = (float)p.beta;
  s.ax = (float)p.accel[0];
  s.ay = (float)p.accel[1];
  s.az = (float)p.accel[2];
  s.inv_tau_g = (float)(1.0 / (4.0 * p.diffusivity + 0.5));
  s.k_rate = (float)p.k_rate;
  s.xi = (float)p.xi;
  s.rho_out = (float)p.rho_out;
  s.reaction_mode = p.reaction_mode;
  return s;
}

Lattice make_lattice(const lbm_geometry &g) {
  Lattice L{};
  L.nx = g.nx;
  L.ny = g.ny;
  L.nz = g.nz;
  L.bc_z = g.bc_z;
  L.n = (long long)g.nx * g.ny * g.nz;
  L.plane = (long long)g.nx * g.ny;
  L.pstride = L.plane * (g.nz + 2);
  return L;
}

// run f((T *)nullptr) with T the batch's population storage type
template <class F>
void with_storage(const Batch &b, F &&f) {
  if (b.half)
    f((__half *)nullptr);
  else
    f((float *)nullptr);
}

Slots slots(const Batch &b) { return Slots{b.inst, b.kid, b.node, b.nslots, b.ns}; }

// Launch of a step kernel that follows another step kernel on the same stream:
// with pdl, as a programmatic dependent launch (the kernel itself waits for its
// predecessor in pdl_begin), else a plain launch.
template <typename... KArgs, typename... Args>
void launch_step_kernel_smem(bool pdl, void (*k)(KArgs...), unsigned grid, unsigned block, size_t smem,
                             cudaStream_t st, Args... args) {
  if (!pdl) {
    k<<<grid, block, smem, st>>>(args...);
    return;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, args...);
}
template <typename... KArgs, typename... Args>
void launch_step_kernel(bool pdl, void (*k)(KArgs...), unsigned grid, unsigned block, cudaStream_t st,
                        Args... args) {
  launch_step_kernel_smem(pdl, k, grid, block, 0, st, args...);
}

// acc: the reaction-sum pairs that the step with parity slot accumulates into (its
// colour-function pass sets them up), or null where nobody reads them
template <typename T, bool BT>
void launch_density_t(const Batch &b, cudaStream_t st, const void *fin, double *acc, int slot) {
  const Slots S = slots(b);
  const Inst &I = b.h[0].d;
  const T *f = (const T *)fin;
  switch (b.dens_block) {
    case 128:
      k_density_c<T, 128, BT><<<(S.nslots + 127) / 128, 128, 0, st>>>(S, I, f, b.gidx, b.rhoN, acc, b.n, slot);
      break;
    case 512:
      k_density_c<T, 512, BT><<<(S.nslots + 511) / 512, 512, 0, st>>>(S, I, f, b.gidx, b.rhoN, acc, b.n, slot);
      break;
    default:
      k_density_c<T, 256, BT><<<(S.nslots + 255) / 256, 256, 0, st>>>(S, I, f, b.gidx, b.rhoN, acc, b.n, slot);
  }
}
template <typename T>
void launch_density(const Batch &b, cudaStream_t st, const void *fin, double *acc = nullptr, int slot = 0) {
  if (b.n > 1)
    launch_density_t<T, true>(b, st, fin, acc, slot);
  else
    launch_density_t<T, false>(b, st, fin, acc, slot);
}

template <bool BT>
void launch_normal_t(const Batch &b, cudaStream_t st) {
  const Slots S = slots(b);
  const Inst &I = b.h[0].d;
  const float *rn = b.rhoN;
  const uint32_t *lk = b.link;
  const float4 *nsv = b.nsv;
  float4 *nrm = b.nrm;
  switch (b.norm_block) {
    case 128:
      launch_step_kernel(b.pdl, k_normal_c<128, BT>, (S.nslots + 127) / 128, 128, st, S, I, rn, lk, nsv, nrm);
      break;
    case 512:
      launch_step_kernel(b.pdl, k_normal_c<512, BT>, (S.nslots + 511) / 512, 512, st, S, I, rn, lk, nsv, nrm);
      break;
    default:
      launch_step_kernel(b.pdl, k_normal_c<256, BT>, (S.nslots + 255) / 256, 256, st, S, I, rn, lk, nsv, nrm);
  }
}
void launch_normal(const Batch &b, cudaStream_t st) {
  if (b.n > 1)
    launch_normal_t<true>(b, st);
  else
    launch_normal_t<false>(b, st);
}

template <typename T, bool BT>
void launch_main_t(const Batch &b, cudaStream_t st, const void *fin, void *fout, double *acc, int slot) {
  const Slots S = slots(b);
  const Inst &I = b.h[0].d;
  float *dh = b.h_out ? b.h_out : (b.debug ? b.dbg_H : nullptr), *dd = b.debug ? b.dbg_delta : nullptr;
  const T *fi = (const T *)fin;
  T *fo = (T *)fout;
  const int *gi = b.gidx;
  const uint32_t *lk = b.link;
  const float4 *nrm = b.nrm;
  const int n = b.n;
  switch (b.main_block) {
    case 64:
      launch_step_kernel(b.pdl, k_main_c<T, 64, BT>, (S.nslots + 63) / 64, 64, st, S, I, n, fi, fo, gi, lk, nrm, acc,
                         slot, b.rstep, dh, dd);
      break;
    case 256:
      launch_step_kernel(b.pdl, k_main_c<T, 256, BT>, (S.nslots + 255) / 256, 256, st, S, I, n, fi, fo, gi, lk, nrm,
                         acc, slot, b.rstep, dh, dd);
      break;
    default:
      launch_step_kernel(b.pdl, k_main_c<T, 128, BT>, (S.nslots + 127) / 128, 128, st, S, I, n, fi, fo, gi, lk, nrm,
                         acc, slot, b.rstep, dh, dd);
  }
}
template <typename T>
void launch_main(const Batch &b, cudaStream_t st, const void *fin, void *fout, double *acc, int slot) {
  if (b.n > 1)
    launch_main_t<T, true>(b, st, fin, fout, acc, slot);
  else
    launch_main_t<T, false>(b, st, fin, fout, acc, slot);
}

void launch_solids(const Batch &b, cudaStream_t st, bool colour) {
  const Inst &I = b.h[0].d;
  const unsigned g = (unsigned)((b.n_bnd + 127) / 128), g256 = (unsigned)((b.n_bnd + 255) / 256);
  const Inst *in = b.inst;
  const uint32_t *bnd = b.bnd, *lk = b.bnd_link;
  const uint16_t *bk = b.bnd_kid;
  const int nb = b.n_bnd;
  if (colour) {
    if (b.n > 1)
      launch_step_kernel(b.pdl, k_color_solid_c<true>, g, 128, st, in, I, bnd, bk, nb, lk, b.rhoN);
    else
      launch_step_kernel(b.pdl, k_color_solid_c<false>, g, 128, st, in, I, bnd, bk, nb, lk, b.rhoN);
  } else {
    if (b.n > 1)
      launch_step_kernel(b.pdl, k_normal_solid_c<true>, g256, 256, st, in, I, bnd, bk, nb, lk, b.nrm);
    else
      launch_step_kernel(b.pdl, k_normal_solid_c<false>, g256, 256, st, in, I, bnd, bk, nb, lk, b.nrm);
  }
}

// xy tile of the z-marching field kernel (k_fields_march) and its chunk lengths in z
constexpr int FTX = 32, FTY = 16;
constexpr int kChunk[3] = {16, 32, 64};
using FTile = MarchTile<FTX, FTY>;

int march_blocks(const Lattice &L, int chunk) {
  return ((L.nx + FTX - 1) / FTX) * ((L.ny + FTY - 1) / FTY) * ((L.nz + chunk - 1) / chunk);
}

// the shared-memory opt-in of the marching field kernel, on the current device
int fields_attributes() {
  const int bytes = (int)FTile::smem_bytes();
  if (cudaFuncSetAttribute(k_fields_march<FTX, FTY, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_fields_march<FTX, FTY, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) !=
          cudaSuccess) {
    (void)cudaGetLastError();
    return LBM_ECUDA;
  }
  return LBM_OK;
}

// a3 - a5 and the normals at solids of every instance in one launch (see k_fields_march)
void launch_fields_march(const Batch &b, cudaStream_t st) {
  const Inst &I = b.h[0].d;
  const int opt = b.fields - 1, chunk = kChunk[opt];
  const int *off = b.block_off ? b.block_off + opt * (b.n + 1) : nullptr;
  if (b.n > 1)
    launch_step_kernel_smem(b.pdl, k_fields_march<FTX, FTY, true>, (unsigned)b.n_blocks[opt], 256,
                            FTile::smem_bytes(), st, (const Inst *)b.inst, I, off, b.n, chunk,
                            (const uint32_t *)b.link, (const float4 *)b.nsv, b.rhoN, b.nrm);
  else
    launch_step_kernel_smem(b.pdl, k_fields_march<FTX, FTY, false>, (unsigned)b.n_blocks[opt], 256,
                            FTile::smem_bytes(), st, (const Inst *)b.inst, I, off, b.n, chunk,
                            (const uint32_t *)b.link, (const float4 *)b.nsv, b.rhoN, b.nrm);
}

// the kernels of one step (in -> out), on stream st
void enqueue_step(Batch &b, cudaStream_t st, const void *fin, void *fout, int slot, bool prof,
                  double *acc = nullptr) {
  auto pb = [&](int k) { if (prof) prof_begin(b, k, st); };
  auto pe = [&]() { if (prof) prof_end(b, st); };
  with_storage(b, [&](auto *tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    pb(0);
    launch_density<T>(b, st, fin, acc ? acc : b.acc, slot);
    pe();
    if (b.fields) {
      pb(6);
      launch_fields_march(b, st);
      pe();
    } else {
      if (b.n_bnd > 0) {
        pb(1);
        launch_solids(b, st, true);
        pe();
      }
      pb(2);
      launch_normal(b, st);
      pe();
      if (b.n_bnd > 0) {
        pb(3);
        launch_solids(b, st, false);
        pe();
      }
    }
    pb(4);
    launch_main<T>(b, st, fin, fout, acc ? acc : b.acc, slot);
    pe();
  });
}

// two graphs of one step: even steps read buf0 and write buf1, odd steps the reverse
int build_graphs(Batch &b) {
  drop_graphs(b);
  cudaStream_t cs;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  int rc = LBM_OK;
  for (int parity = 0; parity < 2 && rc == LBM_OK; ++parity) {
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      rc = LBM_ECUDA;
      break;
    }
    enqueue_step(b, cs, parity ? b.buf1 : b.buf0, parity ? b.buf0 : b.buf1, parity, false);
    if (cudaStreamEndCapture(cs, &g) != cudaSuccess || !g) {
      rc = LBM_ECUDA;
      break;
    }
    if (cudaGraphInstantiate(&b.graph[parity], g, 0) != cudaSuccess) rc = LBM_ECUDA;
    cudaGraphDestroy(g);
  }
  cudaStreamDestroy(cs);
  if (rc != LBM_OK) {
    (void)cudaGetLastError();
    drop_graphs(b);
    return LBM_OK;   // graphs are an optimisation: fall back to plain launches
  }
  b.graphs_valid = true;
  return LBM_OK;
}

int launch_observables(Batch &b) {
  CK(cudaMemsetAsync(b.obs, 0, 8 * sizeof(double) * b.n, b.stream));
  prof_begin(b, 5, b.stream);
  with_storage(b, [&](auto *tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    if (b.n > 1)
      k_observables_c<T, true><<<(b.nslots + 255) / 256, 256, 0, b.stream>>>(slots(b), b.h[0].d, (const T *)b.fa,
                                                                             b.obs);
    else
      k_observables_c<T, false><<<(b.nslots + 255) / 256, 256, 0, b.stream>>>(slots(b), b.h[0].d, (const T *)b.fa,
                                                                              b.obs);
  });
  prof_end(b, b.stream);
  CK(cudaGetLastError());
  return LBM_OK;
}

// after the state changed (it is in both buffers): buffer order, ghost planes, counters, m^C(0)
int reset_after_state(Batch &b) {
  b.fa = b.buf0;
  b.fb = b.buf1;
  for (int k = 0; k < b.n; ++k) {
    const Inst &I = b.h[k].d;
    if (I.L.bc_z != 1) continue;
    const dim3 blk(32, 4, 1), grd((I.L.nx + 31) / 32, (I.L.ny + 3) / 4, 1);
    const lbm_params &p = b.h[k].prm;
    with_storage(b, [&](auto *tag) {
      using T = std::remove_pointer_t<decltype(tag)>;
      k_ghost_init_c<T><<<grd, blk, 0, b.stream>>>(I, b.ns, b.gidx, (float)p.u_in, (float)p.c_in,
                                                    (float)p.rho_out, (T *)b.fa, (T *)b.fb);
    });
    CK(cudaGetLastError());
  }
  CK(cudaMemsetAsync(b.acc, 0, 4 * sizeof(double) * b.n, b.stream));
  CK(cudaMemsetAsync(b.rstep, 0, 2 * sizeof(uint32_t), b.stream));   // FP16 rounding bits restart with the steps
  int rc = launch_observables(b);
  if (rc) return rc;
  std::vector<double> hobs(8 * (size_t)b.n);
  CK(cudaMemcpyAsync(hobs.data(), b.obs, hobs.size() * sizeof(double), cudaMemcpyDeviceToHost, b.stream));
  CK(cudaStreamSynchronize(b.stream));
  for (int k = 0; k < b.n; ++k) b.h[k].mc0 = hobs[8 * k + 2];
  b.step = 0;
  return LBM_OK;
}

int step_n(Batch &b, int64_t nsteps) {
  if (nsteps < 0) return LBM_EINVAL;
  if (b.sticky) return b.sticky;
  cudaSetDevice(b.device);
  const bool use_graph = !b.profiling && !b.debug;
  if (use_graph && !b.graphs_valid && nsteps > 0) {
    int rc = build_graphs(b);
    if (rc) return rc;
  }
  for (int64_t s = 0; s < nsteps; ++s) {
    const int parity = (int)(b.step & 1);
    if (use_graph && b.graphs_valid) {
      CK(cudaGraphLaunch(b.graph[parity], b.stream));
    } else {
      enqueue_step(b, b.stream, b.fa, b.fb, parity, b.profiling);
      CK(cudaGetLastError());
    }
    void *t = b.fa;
    b.fa = b.fb;
    b.fb = t;
    b.step += 1;
  }
  return LBM_OK;
}

int fill_obs(Batch &b, lbm_obs *out, int count) {
  if (b.sticky) return b.sticky;
  cudaSetDevice(b.device);
  int rc = launch_observables(b);
  if (rc) return rc;
  std::vector<double> hobs(8 * (size_t)b.n), hacc(4 * (size_t)b.n);
  int derr = 0;
  CK(cudaMemcpyAsync(hobs.data(), b.obs, hobs.size() * sizeof(double), cudaMemcpyDeviceToHost, b.stream));
  CK(cudaMemcpyAsync(hacc.data(), b.acc, hacc.size() * sizeof(double), cudaMemcpyDeviceToHost, b.stream));
  CK(cudaMemcpyAsync(&derr, b.err, sizeof(int), cudaMemcpyDeviceToHost, b.stream));
  CK(cudaStreamSynchronize(b.stream));
  if (derr) {
    b.sticky = LBM_ECUDA;
    return LBM_ECUDA;
  }
  bool bad = false;
  for (int k = 0; k < count; ++k) {
    const double *h = &hobs[8 * k], *a = &hacc[4 * k];
    lbm_obs &o = out[k];
    std::memset(&o, 0, sizeof(o));
    o.mass_r = h[0];
    o.mass_p = h[1];
    o.mass_c = h[2];
    const int s = (int)((b.step - 1) & 1);   // parity of the last step
    o.consumed = b.step > 0 ? a[2 * s + 1] : 0.0;
    o.rate = b.step > 0 ? a[2 * s] : 0.0;
    o.gas_saturation = h[3] / (double)b.h[k].n_fluid;
    o.flux_in = h[4];
    o.flux_out = h[5];
    o.n_bad = (int64_t)h[6];
    o.step = b.step;
    o.n_fluid = b.h[k].n_fluid;
    if (b.h[k].d.L.bc_z == 1)
      o.conversion = o.flux_in != 0.0 ? 1.0 - o.flux_out / o.flux_in : 0.0;
    else
      o.conversion = b.h[k].mc0 != 0.0 ? o.consumed / b.h[k].mc0 : 0.0;
    bad |= o.n_bad != 0;
  }
  return bad ? LBM_ENAN : LBM_OK;
}

// Build a batch: validate, precompute every instance's geometry and lay out the
// slot space on the GPU, start from equilibrium.
int batch_create(Batch &b, int n, const lbm_geometry *geoms, const lbm_params *params, void *stream) {
  if (n < 1 || n > 65535 || !geoms || !params) return LBM_EINVAL;
  for (int k = 0; k < n; ++k) {
    if (check_geometry(&geoms[k]) || check_params(&params[k])) return LBM_EINVAL;
    if (params[k].storage != params[0].storage) return LBM_EINVAL;
  }
  cudaGetDevice(&b.device);
  b.stream = (cudaStream_t)stream;
  b.half = params[0].storage == 1;
  b.n = n;
  b.h.resize(n);
  // per-instance node / gidx offsets and static geometry
  long long nodes = 0, gtot = 0;
  for (int k = 0; k < n; ++k) {
    InstHost &ih = b.h[k];
    ih.prm = params[k];
    ih.d.L = make_lattice(geoms[k]);
    ih.d.P = make_step_params(params[k]);
    ih.d.node_off = (int)nodes;
    ih.d.gidx_off = (int)gtot;
    nodes += ih.d.L.n;
    gtot += ih.d.L.plane * (ih.d.L.nz + 2);
    if (nodes > (1ll << 31) - 1 || gtot > (1ll << 31) - 1) return LBM_EINVAL;
  }
  b.nodes = nodes;
  int rc = LBM_OK;
  rc = rc ? rc : dalloc(b, (void **)&b.link, nodes * sizeof(uint32_t));
  rc = rc ? rc : dalloc(b, (void **)&b.nsv, nodes * sizeof(float4));
  rc = rc ? rc : dalloc(b, (void **)&b.rhoN, nodes * sizeof(float));
  rc = rc ? rc : dalloc(b, (void **)&b.nrm, nodes * sizeof(float4));
  rc = rc ? rc : dalloc(b, (void **)&b.gidx, gtot * sizeof(int));
  rc = rc ? rc : dalloc(b, (void **)&b.acc, 4 * sizeof(double) * n);
  rc = rc ? rc : dalloc(b, (void **)&b.acc_scratch, 4 * sizeof(double) * n);
  rc = rc ? rc : dalloc(b, (void **)&b.obs, 8 * sizeof(double) * n);
  rc = rc ? rc : dalloc(b, (void **)&b.err, sizeof(int));
  rc = rc ? rc : dalloc(b, (void **)&b.rstep, 2 * sizeof(uint32_t));
  if (rc) return rc;
  CK(cudaMemsetAsync(b.err, 0, sizeof(int), b.stream));
  CK(cudaMemsetAsync(b.rstep, 0, 2 * sizeof(uint32_t), b.stream));
  {
    // geometry kernels, one instance at a time (one-time set-up).  The host mask,
    // reactive flags and contact angles are staged in the normal field (16 B per node,
    // unused until the first step; 6 B per node needed), copied on the context's stream
    // so that each kernel reads its instance's data and the next copy follows it
    auto up = [](long long x) { return (x + 255) / 256 * 256; };
    long long maxn = 0;
    for (int k = 0; k < n; ++k) maxn = std::max(maxn, b.h[k].d.L.n);
    const size_t need = (size_t)(2 * up(maxn) + 4 * maxn);
    struct Own {   // a buffer of its own when the normal field is too small (lattices of a few nodes)
      void *p = nullptr;
      ~Own() { cudaFree(p); }
    } own;
    uint8_t *d_solid = reinterpret_cast<uint8_t *>(b.nrm);
    if (need > (size_t)nodes * sizeof(float4)) {
      if (cudaMalloc(&own.p, need) != cudaSuccess) {
        (void)cudaGetLastError();
        return LBM_ENOMEM;
      }
      d_solid = static_cast<uint8_t *>(own.p);
    }
    uint8_t *const d_react = d_solid + up(maxn);
    float *const d_theta = reinterpret_cast<float *>(d_react + up(maxn));
    for (int k = 0; k < n; ++k) {
      const Lattice &L = b.h[k].d.L;
      CK(cudaMemcpyAsync(d_solid, geoms[k].solid, L.n, cudaMemcpyHostToDevice, b.stream));
      if (geoms[k].reactive) CK(cudaMemcpyAsync(d_react, geoms[k].reactive, L.n, cudaMemcpyHostToDevice, b.stream));
      k_geom<<<node_grid(L), node_block(), 0, b.stream>>>(L, d_solid, geoms[k].reactive ? d_react : nullptr,
                                                          theta_rad(params[k]), b.link + b.h[k].d.node_off,
                                                          b.nsv + b.h[k].d.node_off);
      if (geoms[k].theta_deg) {
        CK(cudaMemcpyAsync(d_theta, geoms[k].theta_deg, L.n * sizeof(float), cudaMemcpyHostToDevice, b.stream));
        k_wall_theta<<<node_grid(L), node_block(), 0, b.stream>>>(L, b.link + b.h[k].d.node_off, d_theta,
                                                                  theta_rad(params[k]), b.nsv + b.h[k].d.node_off);
      }
      CK(cudaGetLastError());
    }
    if (own.p) CK(cudaStreamSynchronize(b.stream));   // before the buffer is freed
  }
  // slot space, built on the GPU (layout.cuh): per instance the block counts and
  // their scan, the totals to the host, then the fills at the instances' offsets
  std::vector<long long> nblk(n + 1, 0);
  for (int k = 0; k < n; ++k) nblk[k + 1] = nblk[k] + (b.h[k].d.L.n + kLayoutBlock - 1) / kLayoutBlock;
  // the counts and totals are staged in the colour field (4 B per node, unused until
  // the first step) when they fit, which they do unless the batch holds many lattices
  // of a few nodes; else in a buffer of their own
  int *d_cnt = nullptr;
  long long *d_tot = nullptr;
  struct Scratch {   // frees an own buffer on every return path
    void *p = nullptr;
    ~Scratch() { cudaFree(p); }
  } scratch;
  {
    const size_t cnt_bytes = (3 * (size_t)nblk[n] * sizeof(int) + 255) / 256 * 256;
    const size_t need = cnt_bytes + 3 * (size_t)n * sizeof(long long);
    char *base = reinterpret_cast<char *>(b.rhoN);
    if (need > (size_t)nodes * sizeof(float)) {
      if (cudaMalloc(&scratch.p, need) != cudaSuccess) {
        (void)cudaGetLastError();
        return LBM_ENOMEM;
      }
      base = static_cast<char *>(scratch.p);
    }
    d_cnt = reinterpret_cast<int *>(base);
    d_tot = reinterpret_cast<long long *>(base + cnt_bytes);
  }
  int *const cf = d_cnt, *const cb = d_cnt + nblk[n], *const cw = d_cnt + 2 * nblk[n];
  for (int k = 0; k < n; ++k) {
    const Lattice &L = b.h[k].d.L;
    const long long o = nblk[k];
    const int nb = (int)(nblk[k + 1] - o);
    k_layout_count<<<nb, kLayoutBlock, 0, b.stream>>>(L.n, b.link + b.h[k].d.node_off, cf + o, cb + o, cw + o);
    k_layout_scan<<<1, 1024, 0, b.stream>>>(nb, cf + o, cb + o, cw + o, d_tot + 3 * k);
  }
  CK(cudaGetLastError());
  std::vector<long long> tot(3 * (size_t)n);
  CK(cudaMemcpyAsync(tot.data(), d_tot, tot.size() * sizeof(long long), cudaMemcpyDeviceToHost, b.stream));
  CK(cudaStreamSynchronize(b.stream));
  long long s = 0, nbnd_tot = 0;
  std::vector<long long> bnd0(n);
  for (int k = 0; k < n; ++k) {
    InstHost &ih = b.h[k];
    const Lattice &L = ih.d.L;
    const long long nf = tot[3 * k];
    ih.n_bnd = tot[3 * k + 1];
    ih.n_wall = tot[3 * k + 2];
    if (nf == 0) return LBM_EINVAL;
    bnd0[k] = nbnd_tot;
    ih.d.slot_off = (int)s;
    ih.d.nf = (int)nf;
    ih.n_fluid = nf;
    ih.d.ghost = (int)(s + nf);
    s += nf + (L.bc_z == 1 ? 2 * L.plane : 0);
    nbnd_tot += ih.n_bnd;
    if (s > (1ll << 31) - 1 || nbnd_tot > (1ll << 31) - 1) return LBM_EINVAL;
  }
  b.nslots = (int)s;
  b.ns = (int)((s + 63) / 64 * 64);
  if ((long long)NPOP * b.ns >= (1ll << 32)) return LBM_EINVAL;   // 32-bit population offsets
  b.n_bnd = (int)nbnd_tot;
  // blocks of the marching field kernel, numbered instance by instance, per chunk option
  std::vector<int> hblock(3 * (size_t)(n + 1), 0);
  for (int o = 0; o < 3; ++o) {
    int *hb = hblock.data() + o * (n + 1);
    for (int k = 0; k < n; ++k) {
      const long long nb = (long long)hb[k] + march_blocks(b.h[k].d.L, kChunk[o]);
      if (nb > (1ll << 31) - 1) return LBM_EINVAL;
      hb[k + 1] = (int)nb;
    }
    b.n_blocks[o] = hb[n];
  }
  if (fields_attributes() != LBM_OK) b.fields = 0;   // no shared-memory opt-in: the three kernels
  const size_t elt = b.half ? sizeof(__half) : sizeof(float);
  const size_t pop_bytes = (size_t)NPOP * b.ns * elt;
  rc = rc ? rc : dalloc(b, &b.buf0, pop_bytes);
  rc = rc ? rc : dalloc(b, &b.buf1, pop_bytes);
  rc = rc ? rc : dalloc(b, (void **)&b.node, (size_t)s * sizeof(uint32_t));
  rc = rc ? rc : dalloc(b, (void **)&b.inst, n * sizeof(Inst));
  if (n > 1) rc = rc ? rc : dalloc(b, (void **)&b.kid, (size_t)s * sizeof(uint16_t));
  if (n > 1) rc = rc ? rc : dalloc(b, (void **)&b.block_off, hblock.size() * sizeof(int));
  if (b.n_bnd > 0) {
    rc = rc ? rc : dalloc(b, (void **)&b.bnd, (size_t)nbnd_tot * sizeof(uint32_t));
    rc = rc ? rc : dalloc(b, (void **)&b.bnd_link, (size_t)nbnd_tot * sizeof(uint32_t));
    if (n > 1) rc = rc ? rc : dalloc(b, (void **)&b.bnd_kid, (size_t)nbnd_tot * sizeof(uint16_t));
  }
  if (rc) return rc;
  for (int k = 0; k < n; ++k) {
    const InstHost &ih = b.h[k];
    const Lattice &L = ih.d.L;
    const long long o = nblk[k];
    int *gi = b.gidx + ih.d.gidx_off;
    k_layout_fill<<<(unsigned)(nblk[k + 1] - o), kLayoutBlock, 0, b.stream>>>(
        L, k, ih.d.slot_off, (int)bnd0[k], b.link + ih.d.node_off, cf + o, cb + o, gi, b.node, b.kid, b.bnd,
        b.bnd_link, b.bnd_kid);
    k_layout_ghosts<<<(unsigned)((L.plane + 255) / 256), 256, 0, b.stream>>>(L, k, ih.d.ghost, gi, b.node, b.kid);
  }
  // every slot-map entry is a slot of the space or -1 (solid): the kernels index
  // population arrays with these values
  k_layout_check<<<(unsigned)((gtot + 255) / 256), 256, 0, b.stream>>>(gtot, b.gidx, b.nslots, b.err);
  CK(cudaGetLastError());
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, b.err, sizeof(int), cudaMemcpyDeviceToHost, b.stream));
  std::vector<Inst> hinst(n);
  for (int k = 0; k < n; ++k) hinst[k] = b.h[k].d;
  CK(cudaMemcpyAsync(b.inst, hinst.data(), n * sizeof(Inst), cudaMemcpyHostToDevice, b.stream));
  if (b.block_off)
    CK(cudaMemcpyAsync(b.block_off, hblock.data(), hblock.size() * sizeof(int), cudaMemcpyHostToDevice, b.stream));
  CK(cudaStreamSynchronize(b.stream));
  if (bad) return LBM_EINVAL;
  // the colour and normal fields held set-up data (geometry inputs, layout counts)
  CK(cudaMemsetAsync(b.rhoN, 0, nodes * sizeof(float), b.stream));
  CK(cudaMemsetAsync(b.nrm, 0, nodes * sizeof(float4), b.stream));
  CK(cudaMemsetAsync(b.buf0, 0, pop_bytes, b.stream));
  CK(cudaMemsetAsync(b.buf1, 0, pop_bytes, b.stream));
  b.fa = b.buf0;
  b.fb = b.buf1;
  for (int k = 0; k < n; ++k) {
    const Inst &I = b.h[k].d;
    with_storage(b, [&](auto *tag) {
      using T = std::remove_pointer_t<decltype(tag)>;
      k_init_c<T><<<(I.nf + 255) / 256, 256, 0, b.stream>>>(I, b.ns, b.node, nullptr, nullptr, nullptr, nullptr, 1.0f,
                                                            0.0f, (float)b.h[k].prm.c_init, (T *)b.fa, (T *)b.fb);
    });
    CK(cudaGetLastError());
  }
  return reset_after_state(b);
}

// Before one instance's state is replaced: make buf0 hold every instance's
// current state (and buf1 too), so the step parity can restart at 0.
int normalise_buffers(Batch &b) {
  const size_t pop_bytes = (size_t)NPOP * b.ns * (b.half ? sizeof(__half) : sizeof(float));
  if (b.fa != b.buf0) CK(cudaMemcpyAsync(b.buf0, b.buf1, pop_bytes, cudaMemcpyDeviceToDevice, b.stream));
  CK(cudaMemcpyAsync(b.buf1, b.buf0, pop_bytes, cudaMemcpyDeviceToDevice, b.stream));
  b.fa = b.buf0;
  b.fb = b.buf1;
  return LBM_OK;
}

int init_fields(Batch &b, int k, const float *rho_r, const float *rho_p, const float *conc, const float *u) {
  if (!rho_r || !rho_p || !conc || k < 0 || k >= b.n) return LBM_EINVAL;
  if (b.sticky) return b.sticky;
  cudaSetDevice(b.device);
  const Inst &I = b.h[k].d;
  const size_t nb = (size_t)I.L.n * sizeof(float);
  float *d = nullptr;
  if (cudaMalloc((void **)&d, nb * (u ? 6 : 3)) != cudaSuccess) {
    (void)cudaGetLastError();
    return LBM_ENOMEM;
  }
  int rc = LBM_OK;
  if (cudaMemcpy(d, rho_r, nb, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy((char *)d + nb, rho_p, nb, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy((char *)d + 2 * nb, conc, nb, cudaMemcpyHostToDevice) != cudaSuccess ||
      (u && cudaMemcpy((char *)d + 3 * nb, u, 3 * nb, cudaMemcpyHostToDevice) != cudaSuccess))
    rc = cuda_fail(b, cudaErrorUnknown);
  if (!rc) rc = normalise_buffers(b);
  if (!rc) {
    const float *fd = d;
    with_storage(b, [&](auto *tag) {
      using T = std::remove_pointer_t<decltype(tag)>;
      k_init_c<T><<<(I.nf + 255) / 256, 256, 0, b.stream>>>(I, b.ns, b.node, fd, fd + I.L.n, fd + 2 * I.L.n,
                                                            u ? fd + 3 * I.L.n : nullptr, 0.f, 0.f, 0.f,
                                                            (T *)b.fa, (T *)b.fb);
    });
    if (cudaGetLastError() != cudaSuccess) rc = cuda_fail(b, cudaErrorLaunchFailure);
  }
  if (!rc) rc = reset_after_state(b);
  cudaStreamSynchronize(b.stream);
  cudaFree(d);
  return rc;
}

// slot-space populations src (storage type T, the state's slot layout, or with SOA an
// adjoint array in population-major order) of instance k -> host [45][n], zero at
// solids (scattered into a dense device array, then one copy)
template <typename T, bool SOA = false>
int slots_to_host(Batch &b, int k, const T *src, float *dst, size_t bytes) {
  const InstHost &ih = b.h[k];
  float *d = nullptr;
  if (cudaMalloc((void **)&d, bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    return LBM_ENOMEM;
  }
  cudaError_t e = cudaMemsetAsync(d, 0, bytes, b.stream);   // solid nodes hold no populations
  if (e == cudaSuccess) {
    if constexpr (SOA)
      k_soa_to_dense<<<(unsigned)((ih.d.nf + 255) / 256), 256, 0, b.stream>>>(ih.d, b.ns, b.node, src, d);
    else
      k_slots_to_dense<T><<<(unsigned)((ih.d.nf + 255) / 256), 256, 0, b.stream>>>(ih.d, b.ns, b.node, src, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(dst, d, bytes, cudaMemcpyDeviceToHost, b.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b.stream);
  cudaFree(d);
  return cuda_fail(b, e);
}

int get_state(Batch &b, int k, float *dst, size_t bytes) {
  if (!dst || k < 0 || k >= b.n) return LBM_EINVAL;
  if (bytes != (size_t)NPOP * b.h[k].d.L.n * sizeof(float)) return LBM_EINVAL;
  if (b.sticky) return b.sticky;
  cudaSetDevice(b.device);
  int rc = LBM_OK;
  with_storage(b, [&](auto *tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    rc = slots_to_host<T>(b, k, (const T *)b.fa, dst, bytes);
  });
  return rc;
}

int set_state(Batch &b, int k, const float *src, size_t bytes) {
  if (!src || k < 0 || k >= b.n) return LBM_EINVAL;
  const InstHost &ih = b.h[k];
  if (bytes != (size_t)NPOP * ih.d.L.n * sizeof(float)) return LBM_EINVAL;
  if (b.sticky) return b.sticky;
  cudaSetDevice(b.device);
  float *d = nullptr;
  if (cudaMalloc((void **)&d, bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    return LBM_ENOMEM;
  }
  cudaError_t e = cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, b.stream);
  if (e == cudaSuccess && normalise_buffers(b) != LBM_OK) e = cudaErrorUnknown;
  if (e == cudaSuccess) {
    with_storage(b, [&](auto *tag) {
      using T = std::remove_pointer_t<decltype(tag)>;
      k_dense_to_slots<T><<<(unsigned)((ih.d.nf + 255) / 256), 256, 0, b.stream>>>(ih.d, b.ns, b.node, d, (T *)b.fa,
                                                                                   (T *)b.fb);
    });
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(b.stream);
  }
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(b, e);
  return reset_after_state(b);
}

// time each launch shape of the tunable kernels on the current state (the
// candidate launches write only the output buffer, the per-node fields and a
// scratch accumulator, which the next step recomputes) and keep the fastest
int tune(Batch &b, int32_t *chosen) {
  if (b.sticky) return b.sticky;
  cudaSetDevice(b.device);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int reps = 5;
  auto time_it = [&](auto &&launch) {
    launch();
    cudaEventRecord(e0, b.stream);
    for (int r = 0; r < reps; ++r) launch();
    cudaEventRecord(e1, b.stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
  };
  const int cand_main[3] = {64, 128, 256}, cand_other[3] = {128, 256, 512};
  float best = 1e30f;
  int pick = b.main_block;
  for (int c : cand_main) {
    b.main_block = c;
    const float t = time_it([&] {
      with_storage(b, [&](auto *tag) {
        using T = std::remove_pointer_t<decltype(tag)>;
        launch_main<T>(b, b.stream, b.fa, b.fb, b.acc_scratch, 0);
      });
    });
    if (t < best) {
      best = t;
      pick = c;
    }
  }
  b.main_block = pick;
  best = 1e30f;
  pick = b.dens_block;
  for (int c : cand_other) {
    b.dens_block = c;
    const float t = time_it([&] {
      with_storage(b, [&](auto *tag) {
        using T = std::remove_pointer_t<decltype(tag)>;
        launch_density<T>(b, b.stream, b.fa);
      });
    });
    if (t < best) {
      best = t;
      pick = c;
    }
  }
  b.dens_block = pick;
  best = 1e30f;
  pick = b.norm_block;
  for (int c : cand_other) {
    b.norm_block = c;
    const float t = time_it([&] { launch_normal(b, b.stream); });
    if (t < best) {
      best = t;
      pick = c;
    }
  }
  b.norm_block = pick;
  // the three field kernels or the z-marching one (three chunk lengths), over whole steps
  best = 1e30f;
  int pick_fields = b.fields;
  for (int v = 3; v >= 0; --v) {
    if (v > 0 && fields_attributes() != LBM_OK) continue;
    b.fields = v;
    const float t = time_it([&] { enqueue_step(b, b.stream, b.fa, b.fb, 0, false, b.acc_scratch); });
    if (t < best) {
      best = t;
      pick_fields = v;
    }
  }
  b.fields = pick_fields;
  // programmatic dependent launch of the step's later kernels, on or off, over whole steps
  best = 1e30f;
  bool pick_pdl = b.pdl;
  for (int v = 1; v >= 0; --v) {
    b.pdl = v == 1;
    const float t = time_it([&] { enqueue_step(b, b.stream, b.fa, b.fb, 0, false, b.acc_scratch); });
    if (t < best) {
      best = t;
      pick_pdl = b.pdl;
    }
  }
  b.pdl = pick_pdl;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaGetLastError());
  // the fields touched by the candidates are recomputed by the next step from fa
  drop_graphs(b);
  if (chosen) {
    chosen[0] = b.main_block;
    chosen[1] = b.dens_block;
    chosen[2] = b.norm_block;
    chosen[3] = b.pdl ? 1 : 0;
    chosen[4] = b.fields;
  }
  return LBM_OK;
}

int set_launch(Batch &b, const int32_t *blocks) {
  if (!blocks) return LBM_EINVAL;
  const auto one_of = [](int v, int a, int c, int d) { return v == a || v == c || v == d; };
  if (!one_of(blocks[0], 64, 128, 256) || !one_of(blocks[1], 128, 256, 512) || !one_of(blocks[2], 128, 256, 512) ||
      (blocks[3] != 0 && blocks[3] != 1) || blocks[4] < 0 || blocks[4] > 3)
    return LBM_EINVAL;
  if (blocks[4] > 0 && fields_attributes() != LBM_OK) return LBM_ECUDA;
  b.main_block = blocks[0];
  b.dens_block = blocks[1];
  b.norm_block = blocks[2];
  b.pdl = blocks[3] == 1;
  b.fields = blocks[4];
  drop_graphs(b);
  return LBM_OK;
}

int get_field(Batch &b, int k, int32_t which, float *dst, size_t bytes) {
  if (!dst || k < 0 || k >= b.n) return LBM_EINVAL;
  if (b.sticky) return b.sticky;
  cudaSetDevice(b.device);
  const InstHost &ih = b.h[k];
  const size_t n = (size_t)ih.d.L.n;
  const size_t one = n * sizeof(float);
  const size_t off = (size_t)ih.d.node_off;
  if (which == LBM_FIELD_RHON || which == LBM_FIELD_GRADMAG || which == LBM_FIELD_NN || which == LBM_FIELD_CURV ||
      which == LBM_FIELD_DELTA) {
    if (bytes != one) return LBM_EINVAL;
  } else if (which == LBM_FIELD_NORMAL || which == LBM_FIELD_NS) {
    if (bytes != 3 * one) return LBM_EINVAL;
  } else {
    return LBM_EINVAL;
  }
  CK(cudaStreamSynchronize(b.stream));
  if (which == LBM_FIELD_RHON) {
    CK(cudaMemcpy(dst, b.rhoN + off, one, cudaMemcpyDeviceToHost));
    return LBM_OK;
  }
  if (which == LBM_FIELD_CURV || which == LBM_FIELD_DELTA) {
    if (!b.dbg_H) return LBM_EINVAL;
    CK(cudaMemcpy(dst, (which == LBM_FIELD_CURV ? b.dbg_H : b.dbg_delta) + off, one, cudaMemcpyDeviceToHost));
    return LBM_OK;
  }
  if (which == LBM_FIELD_NN) {
    std::vector<uint32_t> hv(n);
    CK(cudaMemcpy(hv.data(), b.link + off, n * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < n; ++i) dst[i] = (hv[i] & BIT_SOLID) ? 0.f : (float)((hv[i] >> NN_SHIFT) & 7u);
    return LBM_OK;
  }
  std::vector<float4> hv(n);
  CK(cudaMemcpy(hv.data(), (which == LBM_FIELD_NS ? b.nsv : b.nrm) + off, n * sizeof(float4), cudaMemcpyDeviceToHost));
  if (which == LBM_FIELD_GRADMAG) {
    for (size_t i = 0; i < n; ++i) dst[i] = hv[i].w;
    return LBM_OK;
  }
  for (size_t i = 0; i < n; ++i) {
    dst[i] = hv[i].x;
    dst[n + i] = hv[i].y;
    dst[2 * n + i] = hv[i].z;
  }
  return LBM_OK;
}

int set_debug(Batch &b, int32_t enable) {
  cudaSetDevice(b.device);
  if (enable && !b.dbg_H) {
    const size_t nb = (size_t)b.nodes * sizeof(float);
    if (dalloc(b, (void **)&b.dbg_H, nb) || dalloc(b, (void **)&b.dbg_delta, nb)) return LBM_ENOMEM;
    CK(cudaMemset(b.dbg_H, 0, nb));
    CK(cudaMemset(b.dbg_delta, 0, nb));
  }
  b.debug = enable != 0;
  drop_graphs(b);
  return LBM_OK;
}

int profile(Batch &b, int32_t max_launches) {
  if (max_launches < 0) return LBM_EINVAL;
  cudaSetDevice(b.device);
  const size_t need = (size_t)max_launches * 2;
  while (b.ev.size() < need) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    b.ev.push_back(e);
  }
  b.ev_kind.assign(b.ev.size() / 2 + 1, 0);
  b.ev_used = 0;
  b.profiling = max_launches > 0;
  return LBM_OK;
}

int profile_read(Batch &b, double *ms, int64_t *launches, int32_t n) {
  if (!ms || !launches || n < 1 || n > LBM_NKERNELS) return LBM_EINVAL;
  cudaSetDevice(b.device);
  CK(cudaStreamSynchronize(b.stream));
  for (int k = 0; k < n; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
  }
  for (size_t i = 0; i + 1 < b.ev_used; i += 2) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, b.ev[i], b.ev[i + 1]));
    const int k = b.ev_kind[i / 2];
    if (k < n) {
      ms[k] += t;
      launches[k] += 1;
    }
  }
  return LBM_OK;
}

// ---------------------------------------------------------------------------
// wettability field and inlet (parameters of the adjoint)
// ---------------------------------------------------------------------------
int set_wetting(Batch &b, int k, const float *theta_deg) {
  if (k < 0 || k >= b.n) return LBM_EINVAL;
  if (b.sticky) return b.sticky;
  cudaSetDevice(b.device);
  const InstHost &ih = b.h[k];
  const Lattice &L = ih.d.L;
  float *d = nullptr;
  if (theta_deg) {
    for (long long i = 0; i < L.n; ++i)
      if (!std::isfinite(theta_deg[i])) return LBM_EINVAL;
    if (cudaMalloc((void **)&d, L.n * sizeof(float)) != cudaSuccess) {
      (void)cudaGetLastError();
      return LBM_ENOMEM;
    }
    if (cudaMemcpyAsync(d, theta_deg, L.n * sizeof(float), cudaMemcpyHostToDevice, b.stream) != cudaSuccess) {
      cudaFree(d);
      return cuda_fail(b, cudaErrorUnknown);
    }
  }
  k_wall_theta<<<node_grid(L), node_block(), 0, b.stream>>>(L, b.link + ih.d.node_off, d, theta_rad(ih.prm),
                                                            b.nsv + ih.d.node_off);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(b.stream);
  cudaFree(d);
  b.adj.ready = false;
  return cuda_fail(b, e);
}

int set_inlet(Batch &b, int k, double u_in, double c_in) {
  if (k < 0 || k >= b.n || !std::isfinite(u_in) || !std::isfinite(c_in)) return LBM_EINVAL;
  InstHost &ih = b.h[k];
  if (ih.d.L.bc_z != 1) return LBM_EINVAL;
  if (b.sticky) return b.sticky;
  cudaSetDevice(b.device);
  ih.prm.u_in = u_in;
  ih.prm.c_in = c_in;
  const Inst &I = ih.d;
  const dim3 blk(32, 4, 1), grd((I.L.nx + 31) / 32, (I.L.ny + 3) / 4, 1);
  with_storage(b, [&](auto *tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    k_ghost_init_c<T><<<grd, blk, 0, b.stream>>>(I, b.ns, b.gidx, (float)u_in, (float)c_in, (float)ih.prm.rho_out,
                                                  (T *)b.fa, (T *)b.fb);
  });
  CK(cudaGetLastError());
  b.adj.ready = false;
  return LBM_OK;
}

// ---------------------------------------------------------------------------
// reverse mode: checkpointed forward, then one adjoint step per forward step
// ---------------------------------------------------------------------------
int adj_alloc(Batch &b, int64_t nseg, int64_t K) {
  Batch::Adj &a = b.adj;
  const size_t sb = (size_t)NPOP * b.ns * sizeof(float);
  const size_t nodes = (size_t)b.nodes;
  auto grab = [&](void **p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      *p = nullptr;
      (void)cudaGetLastError();
      return false;
    }
    a.bytes += bytes;
    return true;
  };
  if (!a.lam0) {
    bool ok = grab((void **)&a.lam0, sb) && grab((void **)&a.lam1, sb) &&
              grab((void **)&a.hbar, nodes * sizeof(float)) && grab((void **)&a.rho, nodes * sizeof(float)) &&
              grab((void **)&a.rnbar, nodes * sizeof(float)) && grab((void **)&a.nbar, nodes * sizeof(float4)) &&
              grab((void **)&a.coef, nodes * sizeof(float2)) && grab((void **)&a.thbar, nodes * sizeof(double)) &&
              grab((void **)&a.uin, sizeof(double));
    if (!ok) return LBM_ENOMEM;
  }
  while ((int64_t)a.cp.size() < nseg) {
    float *p = nullptr;
    if (!grab((void **)&p, sb)) return LBM_ENOMEM;
    a.cp.push_back(p);
  }
  while ((int64_t)a.store.size() < K) {
    float *p = nullptr;
    float *r = nullptr;
    float4 *q = nullptr;
    float *h = nullptr;
    if (!grab((void **)&p, sb) || !grab((void **)&r, nodes * sizeof(float)) ||
        !grab((void **)&q, nodes * sizeof(float4)) || !grab((void **)&h, nodes * sizeof(float))) {
      cudaFree(p);
      cudaFree(r);
      cudaFree(q);
      cudaFree(h);
      return LBM_ENOMEM;
    }
    // interior solids are never written and read as zero by the stencils
    if (cudaMemset(r, 0, nodes * sizeof(float)) != cudaSuccess ||
        cudaMemset(q, 0, nodes * sizeof(float4)) != cudaSuccess) {
      cudaFree(p);
      cudaFree(r);
      cudaFree(q);
      cudaFree(h);
      return LBM_ECUDA;
    }
    a.store.push_back(p);
    a.seg_rhoN.push_back(r);
    a.seg_nrm.push_back(q);
    a.seg_H.push_back(h);
  }
  return LBM_OK;
}

int adjoint_forward(Batch &b, int64_t nsteps, int64_t every, double *objective) {
  if (b.n != 1 || b.half || nsteps < 1) return LBM_EINVAL;
  const InstHost &ih = b.h[0];
  if (ih.d.L.bc_z != 1 || ih.prm.reaction_mode != 0) return LBM_EINVAL;
  if (b.sticky) return b.sticky;
  cudaSetDevice(b.device);
  Batch::Adj &a = b.adj;
  a.ready = false;
  int64_t K = every > 0 ? every : (int64_t)std::ceil(std::sqrt((double)nsteps));
  K = std::max<int64_t>(1, std::min(K, nsteps));
  const int64_t nseg = (nsteps + K - 1) / K;
  int rc = adj_alloc(b, nseg, K);
  if (rc) return rc;
  const size_t sb = (size_t)NPOP * b.ns * sizeof(float);
  for (int64_t s = 0; s < nsteps; s += K) {
    CK(cudaMemcpyAsync(a.cp[s / K], b.fa, sb, cudaMemcpyDeviceToDevice, b.stream));
    rc = step_n(b, std::min(K, nsteps - s));   // the segment's steps as one run of graph replays
    if (rc) return rc;
  }
  rc = launch_observables(b);
  if (rc) return rc;
  double h[8];
  CK(cudaMemcpyAsync(h, b.obs, sizeof(h), cudaMemcpyDeviceToHost, b.stream));
  CK(cudaStreamSynchronize(b.stream));
  if (!(h[4] != 0.0) || !std::isfinite(h[4]) || !std::isfinite(h[5])) return LBM_ENAN;
  a.phi_in = h[4];
  a.phi_out = h[5];
  a.nsteps = nsteps;
  a.K = K;
  a.nseg = nseg;
  a.end_step = b.step;
  a.ready = true;
  if (objective) *objective = 1.0 - a.phi_out / a.phi_in;
  return LBM_OK;
}

// the forward fields of state fin (rho^N, colour at solids, wetted normals, normals
// at solids) into b.rhoN / b.nrm
void launch_fields(Batch &b, cudaStream_t st, const float *fin) {
  launch_density<float>(b, st, fin);
  if (b.fields) {
    launch_fields_march(b, st);
    return;
  }
  if (b.n_bnd > 0) launch_solids(b, st, true);
  launch_normal(b, st);
  if (b.n_bnd > 0) launch_solids(b, st, false);
}

// lambda_t from lambda_{t+1} (lam_in) and the state f_t, whose forward fields are
// in b.rhoN / b.nrm
int reverse_step(Batch &b, const float *ft, const float *Hs, const float *lam_in, float *lam_out) {
  Batch::Adj &a = b.adj;
  const cudaStream_t st = b.stream;
  const Slots S = slots(b);
  const Inst &I = b.h[0].d;
  const unsigned g128 = (unsigned)((S.nslots + 127) / 128), g256 = (unsigned)((S.nslots + 255) / 256);
  const unsigned gb = (unsigned)((b.n_bnd + 255) / 256);
  const lbm_params &p = b.h[0].prm;
  CK(cudaMemsetAsync(a.nbar, 0, (size_t)b.nodes * sizeof(float4), st));
  CK(cudaMemsetAsync(a.rnbar, 0, (size_t)b.nodes * sizeof(float), st));
  // a.coef holds the coefficients of the reverse step t + 1 until k_adj_coef replaces them
  k_adj_collide<<<g128, 128, 0, st>>>(S, I, ft, b.gidx, b.link, b.nrm, Hs, lam_in, a.coef, (float)p.u_in,
                                      (float)p.c_in, lam_out, a.nbar, a.hbar, a.rho, a.uin);
  k_adj_curv<<<g256, 256, 0, st>>>(S, I, b.nrm, a.hbar, a.nbar);
  if (b.n_bnd > 0) k_adj_nsolid<<<gb, 256, 0, st>>>(I, b.bnd, b.n_bnd, b.link, b.nrm, a.nbar);
  k_adj_normal<<<g256, 256, 0, st>>>(S, I, b.rhoN, b.link, b.nsv, a.nbar, a.rnbar, a.thbar);
  if (b.n_bnd > 0) k_adj_csolid<<<gb, 256, 0, st>>>(I, b.bnd, b.n_bnd, b.link, a.rnbar);
  k_adj_coef<<<g256, 256, 0, st>>>(S, I, b.rhoN, a.rho, a.rnbar, (float)p.u_in, a.coef, a.uin);
  CK(cudaGetLastError());
  return LBM_OK;
}

int adjoint_backward(Batch &b, double seed, double *dtheta, double *du_in, float *dstate, size_t state_bytes) {
  Batch::Adj &a = b.adj;
  if (!a.ready || b.step != a.end_step || !std::isfinite(seed)) return LBM_EINVAL;
  const InstHost &ih = b.h[0];
  if (dstate && state_bytes != (size_t)NPOP * ih.d.L.n * sizeof(float)) return LBM_EINVAL;
  if (b.sticky) return b.sticky;
  cudaSetDevice(b.device);
  const size_t sb = (size_t)NPOP * b.ns * sizeof(float);
  // the recompute buffers take the constant ghost planes of the current state
  for (int64_t j = 0; j < a.K; ++j) CK(cudaMemcpyAsync(a.store[j], b.fa, sb, cudaMemcpyDeviceToDevice, b.stream));
  CK(cudaMemsetAsync(a.thbar, 0, (size_t)b.nodes * sizeof(double), b.stream));
  CK(cudaMemsetAsync(a.uin, 0, sizeof(double), b.stream));
  // the objective's seed has no density terms; the ghost populations that no node pulls
  // are never written by the push and must read 0
  CK(cudaMemsetAsync(a.coef, 0, (size_t)b.nodes * sizeof(float2), b.stream));
  CK(cudaMemsetAsync(a.lam1, 0, sb, b.stream));
  const double a_in = seed * a.phi_out / (a.phi_in * a.phi_in), a_out = -seed / a.phi_in;
  const Slots S = slots(b);
  k_adj_seed<<<(unsigned)((S.nslots + 255) / 256), 256, 0, b.stream>>>(S, ih.d, (const float *)b.fa, (float)a_in,
                                                                       (float)a_out, a.lam0);
  CK(cudaGetLastError());
  float *lam = a.lam0, *lamn = a.lam1;
  float *const rhoN0 = b.rhoN;
  float4 *const nrm0 = b.nrm;
  int rc = LBM_OK;
  for (int64_t s = a.nseg - 1; s >= 0 && rc == LBM_OK; --s) {
    const int64_t t0 = s * a.K, t1 = std::min(t0 + a.K, a.nsteps);
    CK(cudaMemcpyAsync(a.store[0], a.cp[s], sb, cudaMemcpyDeviceToDevice, b.stream));
    // recompute the segment, keeping every state, its forward fields and (from the
    // main kernel) its curvature; the last state of the segment has no main step,
    // and the collide kernel computes its curvature itself
    for (int64_t t = t0; t < t1; ++t) {
      const int64_t j = t - t0;
      b.rhoN = a.seg_rhoN[j];
      b.nrm = a.seg_nrm[j];
      launch_fields(b, b.stream, a.store[j]);
      b.h_out = a.seg_H[j];
      if (t + 1 < t1) launch_main<float>(b, b.stream, a.store[j], a.store[j + 1], b.acc_scratch, 0);
      b.h_out = nullptr;
    }
    if (cudaGetLastError() != cudaSuccess) rc = LBM_ECUDA;
    for (int64_t t = t1 - 1; t >= t0 && rc == LBM_OK; --t) {
      b.rhoN = a.seg_rhoN[t - t0];
      b.nrm = a.seg_nrm[t - t0];
      rc = reverse_step(b, a.store[t - t0], t + 1 < t1 ? a.seg_H[t - t0] : nullptr, lam, lamn);
      std::swap(lam, lamn);
    }
  }
  b.rhoN = rhoN0;
  b.nrm = nrm0;
  if (rc) return cuda_fail(b, cudaErrorUnknown);
  if (dtheta) {
    CK(cudaMemcpyAsync(dtheta, a.thbar, (size_t)ih.d.L.n * sizeof(double), cudaMemcpyDeviceToHost, b.stream));
  }
  double u = 0.0;
  CK(cudaMemcpyAsync(&u, a.uin, sizeof(double), cudaMemcpyDeviceToHost, b.stream));
  CK(cudaStreamSynchronize(b.stream));
  if (du_in) *du_in = u;
  if (dstate) {
    k_adj_finish<<<(unsigned)((S.nslots + 255) / 256), 256, 0, b.stream>>>(S, ih.d, b.link, a.coef, lam);
    k_adj_ghost0<<<(unsigned)((S.nslots + 255) / 256), 256, 0, b.stream>>>(S, ih.d, a.cp[0], lam);
    CK(cudaGetLastError());
    const int rc = slots_to_host<float, true>(b, 0, lam, dstate, state_bytes);   // adjoint order
    if (rc) return rc;
  }
  return LBM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// allocation-free step: scratch in a fixed device array (see lbm_step_static)
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kStaticAlign = 256;
constexpr size_t kStaticNodes = LBM_STATIC_MAX_NODES;
__host__ __device__ constexpr size_t round_up(size_t v) { return (v + kStaticAlign - 1) / kStaticAlign * kStaticAlign; }
// layout: reaction sums | link words | solid normals | colour field | interface normals
constexpr size_t kOffAcc = 0;
constexpr size_t kOffLink = round_up(4 * sizeof(double));
constexpr size_t kOffNs = kOffLink + round_up(kStaticNodes * sizeof(uint32_t));
constexpr size_t kOffRhoN = kOffNs + round_up(kStaticNodes * sizeof(float4));
constexpr size_t kOffNrm = kOffRhoN + round_up(kStaticNodes * sizeof(float));
constexpr size_t kStaticBytes = kOffNrm + round_up(kStaticNodes * sizeof(float4));

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

// device address of g_static_scratch, looked up once per device
constexpr int kMaxDevices = 64;
unsigned char *g_static_ptr[kMaxDevices] = {};
std::mutex g_static_mutex;

int static_scratch(int dev, unsigned char **out) {
  if (dev < 0 || dev >= kMaxDevices) return LBM_EINVAL;
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (!g_static_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return LBM_ECUDA;
    }
    g_static_ptr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_static_ptr[dev];
  return LBM_OK;
}

// solid nodes next to the fluid, found from the link words (no node list)
__global__ void k_color_solid_all(Lattice L, const uint32_t *__restrict__ link, float *__restrict__ rhoN) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= L.nx || y >= L.ny) return;
  const long long s = nidx(L, x, y, z);
  if (!(link[s] & BIT_SOLID_BND)) return;
  Stencil S;
  S.init(L, x, y, z);
  float num = 0.f, den = 0.f;
#pragma unroll
  for (int i = 0; i < Q - 1; ++i) {
    const long long nb = S.nb(L, CX[i], CY[i], CZ[i]);
    if (!(link[nb] & BIT_SOLID)) {
      num += W[i] * rhoN[nb];
      den += W[i];
    }
  }
  rhoN[s] = den > 0.f ? num / den : 0.f;
}

__global__ void k_normal_solid_all(Lattice L, const uint32_t *__restrict__ link, float4 *__restrict__ nrm) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= L.nx || y >= L.ny) return;
  const long long s = nidx(L, x, y, z);
  if (!(link[s] & BIT_SOLID_BND)) return;
  Stencil S;
  S.init(L, x, y, z);
  float ax = 0.f, ay = 0.f, az = 0.f;
#pragma unroll
  for (int i = 0; i < Q - 1; ++i) {
    const long long nb = S.nb(L, CX[i], CY[i], CZ[i]);
    if (!(link[nb] & BIT_SOLID)) {
      const float4 v = nrm[nb];
      ax += W[i] * v.x;
      ay += W[i] * v.y;
      az += W[i] * v.z;
    }
  }
  const float m = sqrtf(ax * ax + ay * ay + az * az);
  nrm[s] = m >= GRAD_EPS ? make_float4(ax / m, ay / m, az / m, 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// The entries of f_out that k_main does not write: zero at solid nodes (they
// carry no populations), and in the paper's reaction mode the seven reactant
// populations of every fluid node, which that mode does not evolve (copied).
__global__ void k_static_rest(Lattice L, int reaction_mode, const uint32_t *__restrict__ link,
                              const float *__restrict__ fin, float *__restrict__ fout) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= L.nx || y >= L.ny) return;
  const unsigned ps = (unsigned)L.pstride;
  const unsigned off = (unsigned)((z + 1) * L.plane + (long long)y * L.nx + x);
  if (link[nidx(L, x, y, z)] & BIT_SOLID) {
#pragma unroll
    for (int p = 0; p < NPOP; ++p) fout[(unsigned)p * ps + off] = 0.f;
  } else if (reaction_mode == 1) {
#pragma unroll
    for (int j = 0; j < Q7; ++j) fout[(unsigned)(2 * Q + j) * ps + off] = fin[(unsigned)(2 * Q + j) * ps + off];
  }
}

}  // namespace

extern "C" {

const char *lbm_strerror(int code) {
  switch (code) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument (dimensions, parameters, sizes or null pointer)";
    case LBM_ENOMEM: return "device memory allocation failed";
    case LBM_ECUDA: return "CUDA launch or execution error";
    case LBM_ENAN: return "non-finite or non-positive density detected";
    default: return "unknown error code";
  }
}

int lbm_create(const lbm_geometry *geom, const lbm_params *params, lbm_ctx **out) {
  if (!out || check_geometry(geom) || check_params(params)) return LBM_EINVAL;
  // a mask without a fluid node (byte 0) is rejected before any device call; memchr stops at the first one
  const size_t n = (size_t)geom->nx * geom->ny * geom->nz;
  if (!std::memchr(geom->solid, 0, n)) return LBM_EINVAL;
  lbm_ctx *c = new (std::nothrow) lbm_ctx();
  if (!c) return LBM_ENOMEM;
  const int rc = batch_create(c->b, 1, geom, params, params->cuda_stream);
  if (rc) {
    free_all(c->b);
    delete c;
    return rc;
  }
  *out = c;
  return LBM_OK;
}

int lbm_step(lbm_ctx *c, int64_t nsteps) { return c ? step_n(c->b, nsteps) : LBM_EINVAL; }

int lbm_observables(lbm_ctx *c, lbm_obs *out) {
  if (!c || !out) return LBM_EINVAL;
  return fill_obs(c->b, out, 1);
}

int lbm_reaction(lbm_ctx *c, double *rate, double *consumed) {
  if (!c) return LBM_EINVAL;
  Batch &b = c->b;
  if (b.sticky) return b.sticky;
  cudaSetDevice(b.device);
  double a[4];
  CK(cudaMemcpyAsync(a, b.acc, sizeof(a), cudaMemcpyDeviceToHost, b.stream));
  CK(cudaStreamSynchronize(b.stream));
  const int s = (int)((b.step - 1) & 1);   // parity of the last step
  if (rate) *rate = b.step > 0 ? a[2 * s] : 0.0;
  if (consumed) *consumed = b.step > 0 ? a[2 * s + 1] : 0.0;
  return LBM_OK;
}

int lbm_reaction_async(lbm_ctx *c, double *dst) {
  if (!c || !dst) return LBM_EINVAL;
  Batch &b = c->b;
  if (b.sticky) return b.sticky;
  if (b.step < 1) return LBM_EINVAL;
  cudaSetDevice(b.device);
  // the last step's pair (its sum, the cumulative sum): one 16-byte copy
  CK(cudaMemcpyAsync(dst, b.acc + 2 * ((b.step - 1) & 1), 2 * sizeof(double), cudaMemcpyDeviceToHost, b.stream));
  return LBM_OK;
}

int lbm_init_fields(lbm_ctx *c, const float *rho_r, const float *rho_p, const float *conc, const float *u) {
  return c ? init_fields(c->b, 0, rho_r, rho_p, conc, u) : LBM_EINVAL;
}

int lbm_get_state(lbm_ctx *c, float *dst, size_t bytes) { return c ? get_state(c->b, 0, dst, bytes) : LBM_EINVAL; }

int lbm_set_state(lbm_ctx *c, const float *src, size_t bytes) {
  return c ? set_state(c->b, 0, src, bytes) : LBM_EINVAL;
}

int lbm_set_debug(lbm_ctx *c, int32_t enable) { return c ? set_debug(c->b, enable) : LBM_EINVAL; }

int lbm_get_field(lbm_ctx *c, int32_t which, float *dst, size_t bytes) {
  return c ? get_field(c->b, 0, which, dst, bytes) : LBM_EINVAL;
}

int lbm_profile(lbm_ctx *c, int32_t max_launches) { return c ? profile(c->b, max_launches) : LBM_EINVAL; }

int lbm_profile_read(lbm_ctx *c, double *ms, int64_t *launches, int32_t n) {
  return c ? profile_read(c->b, ms, launches, n) : LBM_EINVAL;
}

int lbm_tune(lbm_ctx *c, int32_t *blocks) { return c ? tune(c->b, blocks) : LBM_EINVAL; }

int lbm_set_launch(lbm_ctx *c, const int32_t *blocks) { return c ? set_launch(c->b, blocks) : LBM_EINVAL; }

int lbm_info(lbm_ctx *c, int64_t *n_fluid, int64_t *n_wall, int64_t *n_solid_bnd, int64_t *device_bytes) {
  if (!c) return LBM_EINVAL;
  if (n_fluid) *n_fluid = c->b.h[0].n_fluid;
  if (n_wall) *n_wall = c->b.h[0].n_wall;
  if (n_solid_bnd) *n_solid_bnd = c->b.h[0].n_bnd;
  if (device_bytes) *device_bytes = (int64_t)c->b.device_bytes;
  return LBM_OK;
}

int lbm_set_wetting(lbm_ctx *c, const float *theta_deg) { return c ? set_wetting(c->b, 0, theta_deg) : LBM_EINVAL; }

int lbm_set_inlet(lbm_ctx *c, double u_in, double c_in) { return c ? set_inlet(c->b, 0, u_in, c_in) : LBM_EINVAL; }

int lbm_adjoint_forward(lbm_ctx *c, int64_t nsteps, int64_t checkpoint_every, double *objective) {
  return c ? adjoint_forward(c->b, nsteps, checkpoint_every, objective) : LBM_EINVAL;
}

int lbm_adjoint_backward(lbm_ctx *c, double seed, double *dtheta_deg, double *du_in, float *dstate,
                         size_t state_bytes) {
  return c ? adjoint_backward(c->b, seed, dtheta_deg, du_in, dstate, state_bytes) : LBM_EINVAL;
}

void lbm_destroy(lbm_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->b.device);
  cudaStreamSynchronize(c->b.stream);
  free_all(c->b);
  delete c;
}

int lbm_batch_create(int32_t n, const lbm_geometry *geoms, const lbm_params *params, void *cuda_stream,
                     lbm_batch **out) {
  if (!out || n < 1 || !geoms || !params) return LBM_EINVAL;
  lbm_batch *bt = new (std::nothrow) lbm_batch();
  if (!bt) return LBM_ENOMEM;
  const int rc = batch_create(bt->b, n, geoms, params, cuda_stream);
  if (rc) {
    free_all(bt->b);
    delete bt;
    return rc;
  }
  *out = bt;
  return LBM_OK;
}

int lbm_batch_step(lbm_batch *bt, int64_t nsteps) { return bt ? step_n(bt->b, nsteps) : LBM_EINVAL; }

int lbm_batch_observables(lbm_batch *bt, lbm_obs *out, int32_t count) {
  if (!bt || !out || count != bt->b.n) return LBM_EINVAL;
  return fill_obs(bt->b, out, count);
}

int lbm_batch_get_state(lbm_batch *bt, int32_t k, float *dst, size_t bytes) {
  return bt ? get_state(bt->b, k, dst, bytes) : LBM_EINVAL;
}

int lbm_batch_set_state(lbm_batch *bt, int32_t k, const float *src, size_t bytes) {
  return bt ? set_state(bt->b, k, src, bytes) : LBM_EINVAL;
}

int lbm_batch_tune(lbm_batch *bt, int32_t *blocks) { return bt ? tune(bt->b, blocks) : LBM_EINVAL; }

int lbm_batch_set_launch(lbm_batch *bt, const int32_t *blocks) {
  return bt ? set_launch(bt->b, blocks) : LBM_EINVAL;
}

int lbm_batch_profile(lbm_batch *bt, int32_t max_launches) { return bt ? profile(bt->b, max_launches) : LBM_EINVAL; }

int lbm_batch_profile_read(lbm_batch *bt, double *ms, int64_t *launches, int32_t n) {
  return bt ? profile_read(bt->b, ms, launches, n) : LBM_EINVAL;
}

void lbm_batch_destroy(lbm_batch *bt) {
  if (!bt) return;
  cudaSetDevice(bt->b.device);
  cudaStreamSynchronize(bt->b.stream);
  free_all(bt->b);
  delete bt;
}

int lbm_step_static(int32_t nx, int32_t ny, int32_t nz, const uint8_t *solid, const uint8_t *reactive,
                    const float *f_in, float *f_out, double *delta_sum, const lbm_params *params) {
  if (!solid || !f_in || !f_out || !params) return LBM_EINVAL;
  if (nx < 1 || ny < 1 || nz < 1 || nz > 65535 || ny > 4 * 65535) return LBM_EINVAL;
  const long long n = (long long)nx * ny * nz;
  if (n > (long long)kStaticNodes) return LBM_EINVAL;
  if (check_params(params) != LBM_OK || params->storage != 0) return LBM_EINVAL;   // FP32 populations only
  const size_t pop_bytes = (size_t)NPOP * n * sizeof(float);
  const char *a = (const char *)f_in, *b = (const char *)f_out;
  if (a < b + pop_bytes && b < a + pop_bytes) return LBM_EINVAL;   // overlap
  // an error left pending by the caller's earlier work is reported, not consumed
  // (the check after the launches below can then only see this call's own)
  if (cudaPeekAtLastError() != cudaSuccess) return LBM_ECUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ECUDA;
  unsigned char *base = nullptr;
  int rc = static_scratch(dev, &base);
  if (rc) return rc;
  double *acc = reinterpret_cast<double *>(base + kOffAcc);
  uint32_t *link = reinterpret_cast<uint32_t *>(base + kOffLink);
  float4 *ns = reinterpret_cast<float4 *>(base + kOffNs);
  float *rhoN = reinterpret_cast<float *>(base + kOffRhoN);
  float4 *nrm = reinterpret_cast<float4 *>(base + kOffNrm);
  cudaStream_t st = (cudaStream_t)params->cuda_stream;
  // periodic box in the caller's layout p * N + node: the kernels address
  // population p, stored plane z + 1 at p * pstride + (z + 1) * plane, so the
  // base is moved back by one plane and pstride = N (no ghost planes needed)
  Lattice L{};
  L.nx = nx;
  L.ny = ny;
  L.nz = nz;
  L.bc_z = 0;
  L.n = n;
  L.plane = (long long)nx * ny;
  L.pstride = n;
  const StepParams sp = make_step_params(*params);
  const float *fin = f_in - L.plane;
  float *fout = f_out - L.plane;
  const dim3 nb = node_block(), ng = node_grid(L);
  if (cudaMemsetAsync(acc, 0, 4 * sizeof(double), st) != cudaSuccess) return LBM_ECUDA;
  k_geom<<<ng, nb, 0, st>>>(L, solid, reactive, theta_rad(*params), link, ns);
  k_density<<<ng, nb, 0, st>>>(L, fin, link, rhoN);
  k_color_solid_all<<<ng, nb, 0, st>>>(L, link, rhoN);
  k_normal<<<ng, nb, 0, st>>>(L, sp, rhoN, link, ns, nrm);
  k_normal_solid_all<<<ng, nb, 0, st>>>(L, link, nrm);
  k_main<<<ng, nb, 0, st>>>(L, sp, fin, fout, link, nrm, acc, 0, nullptr, nullptr);
  k_static_rest<<<ng, nb, 0, st>>>(L, sp.reaction_mode, link, fin, fout);
  if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
  if (delta_sum &&
      cudaMemcpyAsync(delta_sum, acc + 2, sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return LBM_ECUDA;
  return LBM_OK;
}


}  // extern "C"
