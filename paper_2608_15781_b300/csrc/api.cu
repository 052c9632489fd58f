// Host side of the C ABI declared in include/cglbm.h: context, device memory,
// launch sequence of one time step, observables, state transfer, profiling.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include "cglbm.h"
#include "compact.cuh"
#include "kernels.cuh"

using namespace cglbm;

struct lbm_ctx {
  int device = 0;
  Lattice L{};
  lbm_params prm{};
  StepParams sp{};
  cudaStream_t stream = nullptr;
  // device memory (library-owned)
  void *fa = nullptr, *fb = nullptr;    // current / next populations, compact layout [45][C.ns]
  bool half = false;                    // FP16 deviation storage (lbm_params.storage = 1)
  uint32_t *link = nullptr;
  float4 *ns = nullptr;
  float *rhoN = nullptr;
  float4 *nrm = nullptr;
  uint32_t *bnd_list = nullptr;         // solid nodes next to the fluid, packed (x, y, z)
  long long n_bnd = 0;
  double *acc = nullptr;                // [0] cumulative delta, [2 + s] per-step delta slots
  double *obs = nullptr;                // 8 observables accumulators
  int *err = nullptr;                   // device error flag (a bounded wait gave up)
  Compact C{};                          // fluid slots and slot stride
  int *gidx = nullptr;                  // stored lattice position -> slot, -1 = solid
  uint32_t *cnode = nullptr;            // slot -> packed (x, y, z), fluid slots only
  std::vector<uint32_t> h_slot_node;    // slot -> node index (host, for state transfer)
  float *dbg_H = nullptr, *dbg_delta = nullptr;
  bool debug = false;
  size_t device_bytes = 0;
  // host-side bookkeeping
  int64_t step = 0;
  double mc0 = 0.0;
  long long n_fluid = 0, n_wall = 0;
  bool have_fields = false;             // rhoN / nrm hold the last step's values
  int sticky = LBM_OK;
  // profiling
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_kind;
  size_t ev_used = 0;
  bool profiling = false;
};

namespace {

int cuda_fail(lbm_ctx *c, cudaError_t e) {
  if (e == cudaSuccess) return LBM_OK;
  if (c) c->sticky = LBM_ECUDA;
  return e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
}

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(c, e_); \
  } while (0)

int dalloc(lbm_ctx *c, void **p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    (void)cudaGetLastError();
    return LBM_ENOMEM;
  }
  c->device_bytes += bytes;
  return LBM_OK;
}

dim3 node_block() { return dim3(32, 4, 1); }
dim3 node_grid(const Lattice &L) { return dim3((L.nx + 31) / 32, (L.ny + 3) / 4, L.nz); }

void prof_begin(lbm_ctx *c, int kind) {
  if (!c->profiling || c->ev_used + 2 > c->ev.size()) return;
  cudaEventRecord(c->ev[c->ev_used], c->stream);
  c->ev_kind[c->ev_used / 2] = kind;
}
void prof_end(lbm_ctx *c) {
  if (!c->profiling || c->ev_used + 2 > c->ev.size()) return;
  cudaEventRecord(c->ev[c->ev_used + 1], c->stream);
  c->ev_used += 2;
}

void free_all(lbm_ctx *c) {
  cudaFree(c->fa);
  cudaFree(c->fb);
  cudaFree(c->link);
  cudaFree(c->ns);
  cudaFree(c->rhoN);
  cudaFree(c->nrm);
  cudaFree(c->bnd_list);
  cudaFree(c->acc);
  cudaFree(c->obs);
  cudaFree(c->err);
  cudaFree(c->gidx);
  cudaFree(c->cnode);
  cudaFree(c->dbg_H);
  cudaFree(c->dbg_delta);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  c->ev.clear();
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

void fill_step_params(lbm_ctx *c) {
  const lbm_params &p = c->prm;
  StepParams &s = c->sp;
  s.omega_cm = (float)(1.0 - 1.0 / p.tau);
  s.half_sigma = (float)(0.5 * p.sigma);
  s.beta = (float)p.beta;
  const double th = p.theta_deg * 3.14159265358979323846 / 180.0;
  s.cos_th = (float)std::cos(th);
  s.sin_th = (float)std::sin(th);
  s.ax = (float)p.accel[0];
  s.ay = (float)p.accel[1];
  s.az = (float)p.accel[2];
  s.inv_tau_g = (float)(1.0 / (4.0 * p.diffusivity + 0.5));
  s.k_rate = (float)p.k_rate;
  s.xi = (float)p.xi;
  s.rho_out = (float)p.rho_out;
  s.reaction_mode = p.reaction_mode;
}

// run f<float>() or f<__half>() for the context's population storage
template <class F>
void with_storage(const lbm_ctx *c, F &&f) {
  if (c->half)
    f((__half *)nullptr);
  else
    f((float *)nullptr);
}

// reduce observables of the current state into c->obs (async)
int launch_observables(lbm_ctx *c) {
  CK(cudaMemsetAsync(c->obs, 0, 8 * sizeof(double), c->stream));
  prof_begin(c, 5);
  with_storage(c, [&](auto *tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    k_observables_c<T><<<(unsigned)((c->C.nf + 255) / 256), 256, 0, c->stream>>>(c->L, c->C, (const T *)c->fa,
                                                                                c->cnode, c->obs);
  });
  prof_end(c);
  CK(cudaGetLastError());
  return LBM_OK;
}

// after the state changed: ghost planes, counters, m^C(0)
int reset_after_state(lbm_ctx *c) {
  const Lattice &L = c->L;
  if (L.bc_z == 1) {
    dim3 b(32, 4, 1), g((L.nx + 31) / 32, (L.ny + 3) / 4, 1);
    with_storage(c, [&](auto *tag) {
      using T = std::remove_pointer_t<decltype(tag)>;
      k_ghost_init_c<T><<<g, b, 0, c->stream>>>(L, c->C, c->gidx, (float)c->prm.u_in, (float)c->prm.c_in,
                                                (float)c->prm.rho_out, (T *)c->fa, (T *)c->fb);
    });
    CK(cudaGetLastError());
  }
  CK(cudaMemsetAsync(c->acc, 0, 4 * sizeof(double), c->stream));
  int rc = launch_observables(c);
  if (rc) return rc;
  double h[8];
  CK(cudaMemcpyAsync(h, c->obs, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->mc0 = h[2];
  c->step = 0;
  c->have_fields = false;
  return LBM_OK;
}

int launch_step(lbm_ctx *c) {
  const Lattice &L = c->L;
  const dim3 nb = node_block(), ng = node_grid(L);
  const int slot = (int)(c->step & 1);
  prof_begin(c, 0);
  const unsigned gf = (unsigned)((c->C.nf + 255) / 256);
  with_storage(c, [&](auto *tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    k_density_c<T><<<gf, 256, 0, c->stream>>>(L, c->C, (const T *)c->fa, c->gidx, c->cnode, c->rhoN);
  });
  prof_end(c);
  if (c->n_bnd > 0) {
    const unsigned gb = (unsigned)((c->n_bnd + 255) / 256);
    prof_begin(c, 1);
    k_color_solid<<<gb, 256, 0, c->stream>>>(L, c->bnd_list, c->n_bnd, c->link, c->rhoN);
    prof_end(c);
  }
  prof_begin(c, 2);
  k_normal_c<<<gf, 256, 0, c->stream>>>(L, c->sp, c->C, c->cnode, c->rhoN, c->link, c->ns, c->nrm);
  prof_end(c);
  if (c->n_bnd > 0) {
    const unsigned gb = (unsigned)((c->n_bnd + 255) / 256);
    prof_begin(c, 3);
    k_normal_solid<<<gb, 256, 0, c->stream>>>(L, c->bnd_list, c->n_bnd, c->link, c->nrm);
    prof_end(c);
  }
  prof_begin(c, 4);
  with_storage(c, [&](auto *tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    k_main_c<T><<<(unsigned)((c->C.nf + CGLBM_MAIN_BLOCK - 1) / CGLBM_MAIN_BLOCK), CGLBM_MAIN_BLOCK, 0,
                  c->stream>>>(L, c->C, c->sp, (const T *)c->fa, (T *)c->fb, c->gidx, c->cnode, c->link, c->nrm,
                               c->acc, slot, c->debug ? c->dbg_H : nullptr, c->debug ? c->dbg_delta : nullptr);
  });
  prof_end(c);
  CK(cudaGetLastError());
  void *t = c->fa;
  c->fa = c->fb;
  c->fb = t;
  c->step += 1;
  c->have_fields = true;
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
  if (!geom || !params || !out || !geom->solid) return LBM_EINVAL;
  if (geom->nx < 1 || geom->ny < 1 || geom->nz < 1) return LBM_EINVAL;
  if (geom->bc_z != 0 && geom->bc_z != 1) return LBM_EINVAL;
  if (geom->bc_z == 1 && geom->nz < 2) return LBM_EINVAL;
  // packed slot coordinates (10 + 10 + 11 bits)
  if (geom->nx > 1024 || geom->ny > 1024 || geom->nz > 2048) return LBM_EINVAL;
  int rc = check_params(params);
  if (rc) return rc;
  const long long n = (long long)geom->nx * geom->ny * geom->nz;
  if (n > (1ll << 31) - 1) return LBM_EINVAL;   // node lists are 32-bit
  // 32-bit population offsets: 45 populations x (nz + 2) planes must stay below 2^32
  if ((long long)NPOP * geom->nx * geom->ny * (geom->nz + 2) >= (1ll << 32)) return LBM_EINVAL;
  long long nfl = 0;
  for (long long i = 0; i < n; ++i) nfl += geom->solid[i] ? 0 : 1;
  if (nfl == 0) return LBM_EINVAL;

  lbm_ctx *c = new (std::nothrow) lbm_ctx();
  if (!c) return LBM_ENOMEM;
  cudaGetDevice(&c->device);
  c->prm = *params;
  c->stream = (cudaStream_t)params->cuda_stream;
  Lattice &L = c->L;
  L.nx = geom->nx;
  L.ny = geom->ny;
  L.nz = geom->nz;
  L.bc_z = geom->bc_z;
  L.n = n;
  L.plane = (long long)L.nx * L.ny;
  L.pstride = L.plane * (L.nz + 2);
  c->n_fluid = nfl;
  fill_step_params(c);


  uint8_t *d_solid = nullptr, *d_react = nullptr;
  rc = LBM_OK;
  rc = rc ? rc : dalloc(c, (void **)&c->link, n * sizeof(uint32_t));
  rc = rc ? rc : dalloc(c, (void **)&c->ns, n * sizeof(float4));
  rc = rc ? rc : dalloc(c, (void **)&c->rhoN, n * sizeof(float));
  rc = rc ? rc : dalloc(c, (void **)&c->nrm, n * sizeof(float4));
  rc = rc ? rc : dalloc(c, (void **)&c->acc, 8 * sizeof(double));
  rc = rc ? rc : dalloc(c, (void **)&c->obs, 8 * sizeof(double));
  rc = rc ? rc : dalloc(c, (void **)&c->err, sizeof(int));
  if (!rc && cudaMalloc((void **)&d_solid, n) != cudaSuccess) rc = LBM_ENOMEM;
  if (!rc && geom->reactive && cudaMalloc((void **)&d_react, n) != cudaSuccess) rc = LBM_ENOMEM;
  if (rc) {
    (void)cudaGetLastError();
    cudaFree(d_solid);
    cudaFree(d_react);
    free_all(c);
    delete c;
    return rc;
  }
  auto fail = [&](int code) {
    cudaFree(d_solid);
    cudaFree(d_react);
    free_all(c);
    delete c;
    return code;
  };
  if (cudaMemcpy(d_solid, geom->solid, n, cudaMemcpyHostToDevice) != cudaSuccess) return fail(LBM_ECUDA);
  if (d_react && cudaMemcpy(d_react, geom->reactive, n, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(LBM_ECUDA);
  if (cudaMemsetAsync(c->rhoN, 0, n * sizeof(float), c->stream) != cudaSuccess) return fail(LBM_ECUDA);
  if (cudaMemsetAsync(c->nrm, 0, n * sizeof(float4), c->stream) != cudaSuccess) return fail(LBM_ECUDA);
  if (cudaMemsetAsync(c->err, 0, sizeof(int), c->stream) != cudaSuccess) return fail(LBM_ECUDA);
  k_geom<<<node_grid(L), node_block(), 0, c->stream>>>(L, d_solid, d_react, c->link, c->ns);
  if (cudaGetLastError() != cudaSuccess) return fail(LBM_ECUDA);
  // boundary-solid list, built from the device flags in node order
  std::vector<uint32_t> hlink(n);
  if (cudaMemcpyAsync(hlink.data(), c->link, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return fail(LBM_ECUDA);
  cudaFree(d_solid);
  cudaFree(d_react);
  d_solid = d_react = nullptr;
  // boundary-solid list, compact slots (fluid nodes in lattice order, then the
  // inlet and outlet ghost planes in column mode) and the position -> slot map
  std::vector<uint32_t> blist, cnode;
  std::vector<int> gidx((size_t)L.plane * (L.nz + 2), -1);
  for (long long i = 0; i < n; ++i) {
    const uint32_t x = (uint32_t)(i % L.nx), y = (uint32_t)((i / L.nx) % L.ny), z = (uint32_t)(i / L.plane);
    if (hlink[i] & BIT_SOLID_BND) blist.push_back(x | (y << 10) | (z << 20));
    if (hlink[i] & BIT_WALL) c->n_wall++;
    if (!(hlink[i] & BIT_SOLID)) {
      gidx[(size_t)(i + L.plane)] = (int)cnode.size();
      c->h_slot_node.push_back((uint32_t)i);
      cnode.push_back(x | (y << 10) | (z << 20));
    }
  }
  c->C.nf = (int)cnode.size();
  const long long nghost = L.bc_z == 1 ? 2 * L.plane : 0;
  c->C.ns = (int)((c->C.nf + nghost + 63) / 64 * 64);
  if (L.bc_z == 1)
    for (long long q = 0; q < L.plane; ++q) {
      gidx[(size_t)q] = c->C.nf + (int)q;                                         // inlet plane
      gidx[(size_t)((L.nz + 1) * L.plane + q)] = c->C.nf + (int)(L.plane + q);    // outlet plane
    }
  c->half = params->storage == 1;
  const size_t pop_bytes = (size_t)NPOP * c->C.ns * (c->half ? sizeof(__half) : sizeof(float));
  if (dalloc(c, (void **)&c->fa, pop_bytes) || dalloc(c, (void **)&c->fb, pop_bytes) ||
      dalloc(c, (void **)&c->gidx, gidx.size() * sizeof(int)) ||
      dalloc(c, (void **)&c->cnode, cnode.size() * sizeof(uint32_t)))
    return fail(LBM_ENOMEM);
  if (cudaMemsetAsync(c->fa, 0, pop_bytes, c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->fb, 0, pop_bytes, c->stream) != cudaSuccess ||
      cudaMemcpy(c->gidx, gidx.data(), gidx.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->cnode, cnode.data(), cnode.size() * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(LBM_ECUDA);
  c->n_bnd = (long long)blist.size();
  if (c->n_bnd > 0) {
    if (dalloc(c, (void **)&c->bnd_list, blist.size() * sizeof(uint32_t))) return fail(LBM_ENOMEM);
    if (cudaMemcpy(c->bnd_list, blist.data(), blist.size() * sizeof(uint32_t), cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return fail(LBM_ECUDA);
  }
  with_storage(c, [&](auto *tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    k_init_c<T><<<(unsigned)((c->C.nf + 255) / 256), 256, 0, c->stream>>>(
        L, c->C, c->cnode, nullptr, nullptr, nullptr, nullptr, 1.0f, 0.0f, (float)params->c_init, (T *)c->fa,
        (T *)c->fb);
  });
  if (cudaGetLastError() != cudaSuccess) return fail(LBM_ECUDA);
  rc = reset_after_state(c);
  if (rc) return fail(rc);
  *out = c;
  return LBM_OK;
}

int lbm_step(lbm_ctx *c, int64_t nsteps) {
  if (!c || nsteps < 0) return LBM_EINVAL;
  if (c->sticky) return c->sticky;
  cudaSetDevice(c->device);
  for (int64_t s = 0; s < nsteps; ++s) {
    int rc = launch_step(c);
    if (rc) return rc;
  }
  return LBM_OK;
}

int lbm_observables(lbm_ctx *c, lbm_obs *out) {
  if (!c || !out) return LBM_EINVAL;
  if (c->sticky) return c->sticky;
  cudaSetDevice(c->device);
  int rc = launch_observables(c);
  if (rc) return rc;
  double h[8], a[4];
  int derr = 0;
  CK(cudaMemcpyAsync(h, c->obs, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(a, c->acc, sizeof(a), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&derr, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (derr) {
    c->sticky = LBM_ECUDA;
    return LBM_ECUDA;
  }
  std::memset(out, 0, sizeof(*out));
  out->mass_r = h[0];
  out->mass_p = h[1];
  out->mass_c = h[2];
  out->consumed = a[0];
  out->rate = c->step > 0 ? a[2 + ((c->step - 1) & 1)] : 0.0;
  out->gas_saturation = h[3] / (double)c->n_fluid;
  out->flux_in = h[4];
  out->flux_out = h[5];
  out->n_bad = (int64_t)h[6];
  out->step = c->step;
  out->n_fluid = c->n_fluid;
  if (c->L.bc_z == 1)
    out->conversion = out->flux_in != 0.0 ? 1.0 - out->flux_out / out->flux_in : 0.0;
  else
    out->conversion = c->mc0 != 0.0 ? out->consumed / c->mc0 : 0.0;
  return out->n_bad ? LBM_ENAN : LBM_OK;
}

int lbm_reaction(lbm_ctx *c, double *rate, double *consumed) {
  if (!c) return LBM_EINVAL;
  if (c->sticky) return c->sticky;
  cudaSetDevice(c->device);
  double a[4];
  CK(cudaMemcpyAsync(a, c->acc, sizeof(a), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (rate) *rate = c->step > 0 ? a[2 + ((c->step - 1) & 1)] : 0.0;
  if (consumed) *consumed = a[0];
  return LBM_OK;
}

int lbm_init_fields(lbm_ctx *c, const float *rho_r, const float *rho_p, const float *conc, const float *u) {
  if (!c || !rho_r || !rho_p || !conc) return LBM_EINVAL;
  if (c->sticky) return c->sticky;
  cudaSetDevice(c->device);
  const Lattice &L = c->L;
  const size_t nb = (size_t)L.n * sizeof(float);
  float *d = nullptr;
  const size_t tot = nb * (u ? 6 : 3);
  if (cudaMalloc((void **)&d, tot) != cudaSuccess) {
    (void)cudaGetLastError();
    return LBM_ENOMEM;
  }
  int rc = LBM_OK;
  if (cudaMemcpy(d, rho_r, nb, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy((char *)d + nb, rho_p, nb, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy((char *)d + 2 * nb, conc, nb, cudaMemcpyHostToDevice) != cudaSuccess ||
      (u && cudaMemcpy((char *)d + 3 * nb, u, 3 * nb, cudaMemcpyHostToDevice) != cudaSuccess))
    rc = cuda_fail(c, cudaErrorUnknown);
  if (!rc) {
    const float *fd = d;
    with_storage(c, [&](auto *tag) {
      using T = std::remove_pointer_t<decltype(tag)>;
      k_init_c<T><<<(unsigned)((c->C.nf + 255) / 256), 256, 0, c->stream>>>(
          L, c->C, c->cnode, fd, fd + L.n, fd + 2 * L.n, u ? fd + 3 * L.n : nullptr, 0.f, 0.f, 0.f, (T *)c->fa,
          (T *)c->fb);
    });
    if (cudaGetLastError() != cudaSuccess) rc = cuda_fail(c, cudaErrorLaunchFailure);
  }
  if (!rc) rc = reset_after_state(c);
  cudaStreamSynchronize(c->stream);
  cudaFree(d);
  return rc;
}

int lbm_get_state(lbm_ctx *c, float *dst, size_t bytes) {
  if (!c || !dst) return LBM_EINVAL;
  const Lattice &L = c->L;
  if (bytes != (size_t)NPOP * L.n * sizeof(float)) return LBM_EINVAL;
  if (c->sticky) return c->sticky;
  cudaSetDevice(c->device);
  const size_t nf = (size_t)c->C.nf;
  float *d = nullptr;
  if (cudaMalloc((void **)&d, (size_t)NPOP * nf * sizeof(float)) != cudaSuccess) {
    (void)cudaGetLastError();
    return LBM_ENOMEM;
  }
  with_storage(c, [&](auto *tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    k_slots_to_f32<T><<<(unsigned)((nf + 255) / 256), 256, 0, c->stream>>>(c->C, (const T *)c->fa, d);
  });
  std::vector<float> h((size_t)NPOP * nf);
  cudaError_t e = cudaMemcpyAsync(h.data(), d, h.size() * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(c, e);
  std::memset(dst, 0, bytes);   // solid nodes hold no populations
  for (int p = 0; p < NPOP; ++p) {
    float *o = dst + (size_t)p * L.n;
    const float *s = h.data() + (size_t)p * nf;
    for (size_t t = 0; t < nf; ++t) o[c->h_slot_node[t]] = s[t];
  }
  return LBM_OK;
}

int lbm_set_state(lbm_ctx *c, const float *src, size_t bytes) {
  if (!c || !src) return LBM_EINVAL;
  const Lattice &L = c->L;
  if (bytes != (size_t)NPOP * L.n * sizeof(float)) return LBM_EINVAL;
  if (c->sticky) return c->sticky;
  cudaSetDevice(c->device);
  const size_t nf = (size_t)c->C.nf;
  std::vector<float> h((size_t)NPOP * nf);
  for (int p = 0; p < NPOP; ++p) {
    const float *s = src + (size_t)p * L.n;
    float *o = h.data() + (size_t)p * nf;
    for (size_t t = 0; t < nf; ++t) o[t] = s[c->h_slot_node[t]];
  }
  float *d = nullptr;
  if (cudaMalloc((void **)&d, h.size() * sizeof(float)) != cudaSuccess) {
    (void)cudaGetLastError();
    return LBM_ENOMEM;
  }
  cudaError_t e = cudaMemcpyAsync(d, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) {
    with_storage(c, [&](auto *tag) {
      using T = std::remove_pointer_t<decltype(tag)>;
      k_f32_to_slots<T><<<(unsigned)((nf + 255) / 256), 256, 0, c->stream>>>(c->C, d, (T *)c->fa, (T *)c->fb);
    });
    e = cudaStreamSynchronize(c->stream);
  }
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(c, e);
  return reset_after_state(c);
}

int lbm_set_debug(lbm_ctx *c, int32_t enable) {
  if (!c) return LBM_EINVAL;
  cudaSetDevice(c->device);
  if (enable && !c->dbg_H) {
    const size_t nb = (size_t)c->L.n * sizeof(float);
    if (dalloc(c, (void **)&c->dbg_H, nb) || dalloc(c, (void **)&c->dbg_delta, nb)) return LBM_ENOMEM;
    if (cudaMemset(c->dbg_H, 0, nb) != cudaSuccess || cudaMemset(c->dbg_delta, 0, nb) != cudaSuccess)
      return cuda_fail(c, cudaErrorUnknown);
  }
  c->debug = enable != 0;
  return LBM_OK;
}

int lbm_get_field(lbm_ctx *c, int32_t which, float *dst, size_t bytes) {
  if (!c || !dst) return LBM_EINVAL;
  if (c->sticky) return c->sticky;
  cudaSetDevice(c->device);
  const Lattice &L = c->L;
  const size_t n = (size_t)L.n;
  const size_t one = n * sizeof(float);
  if (which == LBM_FIELD_RHON || which == LBM_FIELD_GRADMAG || which == LBM_FIELD_NN ||
      which == LBM_FIELD_CURV || which == LBM_FIELD_DELTA) {
    if (bytes != one) return LBM_EINVAL;
  } else if (which == LBM_FIELD_NORMAL || which == LBM_FIELD_NS) {
    if (bytes != 3 * one) return LBM_EINVAL;
  } else {
    return LBM_EINVAL;
  }
  CK(cudaStreamSynchronize(c->stream));
  if (which == LBM_FIELD_RHON) {
    CK(cudaMemcpy(dst, c->rhoN, one, cudaMemcpyDeviceToHost));
    return LBM_OK;
  }
  if (which == LBM_FIELD_CURV || which == LBM_FIELD_DELTA) {
    if (!c->dbg_H) return LBM_EINVAL;
    CK(cudaMemcpy(dst, which == LBM_FIELD_CURV ? c->dbg_H : c->dbg_delta, one, cudaMemcpyDeviceToHost));
    return LBM_OK;
  }
  if (which == LBM_FIELD_NN) {
    std::vector<uint32_t> h(n);
    CK(cudaMemcpy(h.data(), c->link, n * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < n; ++i) dst[i] = (float)((h[i] >> NN_SHIFT) & 7u);
    return LBM_OK;
  }
  std::vector<float4> h(n);
  CK(cudaMemcpy(h.data(), which == LBM_FIELD_NS ? c->ns : c->nrm, n * sizeof(float4), cudaMemcpyDeviceToHost));
  if (which == LBM_FIELD_GRADMAG) {
    for (size_t i = 0; i < n; ++i) dst[i] = h[i].w;
    return LBM_OK;
  }
  for (size_t i = 0; i < n; ++i) {
    dst[i] = h[i].x;
    dst[n + i] = h[i].y;
    dst[2 * n + i] = h[i].z;
  }
  return LBM_OK;
}

int lbm_profile(lbm_ctx *c, int32_t max_launches) {
  if (!c || max_launches < 0) return LBM_EINVAL;
  cudaSetDevice(c->device);
  const size_t need = (size_t)max_launches * 2;
  while (c->ev.size() < need) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    c->ev.push_back(e);
  }
  c->ev_kind.assign(c->ev.size() / 2 + 1, 0);
  c->ev_used = 0;
  c->profiling = max_launches > 0;
  return LBM_OK;
}

int lbm_profile_read(lbm_ctx *c, double *ms, int64_t *launches, int32_t n) {
  if (!c || !ms || !launches || n < 1 || n > LBM_NKERNELS) return LBM_EINVAL;
  cudaSetDevice(c->device);
  CK(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < n; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
  }
  for (size_t i = 0; i + 1 < c->ev_used; i += 2) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, c->ev[i], c->ev[i + 1]));
    const int k = c->ev_kind[i / 2];
    if (k < n) {
      ms[k] += t;
      launches[k] += 1;
    }
  }
  return LBM_OK;
}

int lbm_info(lbm_ctx *c, int64_t *n_fluid, int64_t *n_wall, int64_t *n_solid_bnd, int64_t *device_bytes) {
  if (!c) return LBM_EINVAL;
  if (n_fluid) *n_fluid = c->n_fluid;
  if (n_wall) *n_wall = c->n_wall;
  if (n_solid_bnd) *n_solid_bnd = c->n_bnd;
  if (device_bytes) *device_bytes = (int64_t)c->device_bytes;
  return LBM_OK;
}

int lbm_step_static(int32_t nx, int32_t ny, int32_t nz, const uint8_t *solid, const uint8_t *reactive,
                    const float *f_in, float *f_out, double *delta_sum, const lbm_params *params) {
  if (!solid || !f_in || !f_out || !params) return LBM_EINVAL;
  if (nx < 1 || ny < 1 || nz < 1 || nz > 65535 || ny > 4 * 65535) return LBM_EINVAL;
  const long long n = (long long)nx * ny * nz;
  if (n > (long long)kStaticNodes) return LBM_EINVAL;
  if (check_params(params) != LBM_OK) return LBM_EINVAL;
  const size_t pop_bytes = (size_t)NPOP * n * sizeof(float);
  const char *a = (const char *)f_in, *b = (const char *)f_out;
  if (a < b + pop_bytes && b < a + pop_bytes) return LBM_EINVAL;   // overlap
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
  lbm_ctx tmp;                      // parameter conversion only; owns no memory
  tmp.prm = *params;
  fill_step_params(&tmp);
  const float *fin = f_in - L.plane;
  float *fout = f_out - L.plane;
  const dim3 nb = node_block(), ng = node_grid(L);
  if (cudaMemsetAsync(acc, 0, 4 * sizeof(double), st) != cudaSuccess) return LBM_ECUDA;
  k_geom<<<ng, nb, 0, st>>>(L, solid, reactive, link, ns);
  k_density<<<ng, nb, 0, st>>>(L, fin, link, rhoN);
  k_color_solid_all<<<ng, nb, 0, st>>>(L, link, rhoN);
  k_normal<<<ng, nb, 0, st>>>(L, tmp.sp, rhoN, link, ns, nrm);
  k_normal_solid_all<<<ng, nb, 0, st>>>(L, link, nrm);
  k_main<<<ng, nb, 0, st>>>(L, tmp.sp, fin, fout, link, nrm, acc, 0, nullptr, nullptr);
  if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
  if (delta_sum &&
      cudaMemcpyAsync(delta_sum, acc + 2, sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return LBM_ECUDA;
  return LBM_OK;
}

void lbm_destroy(lbm_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
}

}  // extern "C"
