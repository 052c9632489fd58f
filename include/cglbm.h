/*
 * cglbm.h -- C ABI of the B300 colour-gradient lattice Boltzmann library.
 *
 * One context holds one lattice: two immiscible fluid components (liquid
 * reactant r, gas product p) on D3Q19 and a dissolved reactant C on D3Q7,
 * inside a static porous solid.  One call of lbm_step advances the lattice by
 * whole time steps of the method of Beunen & Harting, "Gas-generating reactive
 * flows in bicontinuous catalyst support structures":
 *
 *   pull streaming with halfway bounce-back        Sec. 2.2, Eq. bounce_back
 *   colour field, extrapolated into the solid      Eq. color_function,
 *                                                   Eq. color_lattice_weighted_average
 *   isotropic gradient, normal, wetting            Eq. finite_difference_scheme,
 *                                                   Eq. color_gradient_normal,
 *                                                   Eq. realigned_normal_vectors,
 *                                                   Eq. normal_vector_solid
 *   curvature, CSF force, exact-difference shift   Eq. interface_curvature,
 *                                                   Eq. continuum_surface_force,
 *                                                   Eq. operator_perturbation
 *   central-moment collision                       Appendix A, Eq. collision_operator,
 *                                                   Eq. back_transformation_vector
 *   recolouring                                    Eq. operator_recoloring
 *   surface reaction                               Eq. reactive_boundary_condition_*
 * and reports the observables of Sec. 5.1 (Eq. reactant_mass,
 * Eq. product_mass, Eq. production_rate).  The advection-diffusion lattice for
 * C and the inlet/outlet column boundaries are additions of this library (the
 * paper converts rho^r into rho^p directly and uses periodic boxes only);
 * reaction_mode = 1 selects the paper's direct conversion.
 *
 * Conventions
 *   - Lattice index of node (x, y, z): (z * ny + y) * nx + x, x fastest.
 *   - Populations: 45 per node, population-major ("structure of arrays"):
 *     f^r_0..18, f^p_0..18, g_0..6.  D3Q19 order is the column order of the
 *     paper's matrix M (Sec. 2.1), rest vector last; D3Q7 order is
 *     +x, -x, +y, -y, +z, -z, rest.  A state buffer for lbm_get_state /
 *     lbm_set_state holds 45 * nx * ny * nz floats, index p * N + node.
 *   - All host pointers are read or written synchronously inside the call and
 *     are not retained; the caller keeps ownership.  The library owns every
 *     device allocation of a context.  The CUDA stream passed in lbm_params is
 *     borrowed and must outlive the context.
 *   - Every function returns LBM_OK (0) or a negative code; none aborts.
 *     Kernel faults are asynchronous: lbm_step returns launch errors, and the
 *     next synchronising call (lbm_observables, lbm_get_*) returns the
 *     execution error.  A context that returned LBM_ECUDA should be destroyed.
 */
#ifndef CGLBM_H
#define CGLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_OK 0
#define LBM_EINVAL (-1)   /* bad dimensions, parameters, sizes or null pointers     */
#define LBM_ENOMEM (-2)   /* device allocation failed                               */
#define LBM_ECUDA (-3)    /* CUDA launch or execution error                         */
#define LBM_ENAN (-4)     /* observables found a non-finite or non-positive density */

typedef struct lbm_ctx lbm_ctx;   /* opaque, library-owned */

typedef struct {
  int32_t nx, ny, nz;        /* lattice size, each >= 1; nz >= 2 in column mode   */
  const uint8_t *solid;      /* host, nx*ny*nz bytes, nonzero = solid node s(x)=1   */
  const uint8_t *reactive;   /* host, optional r(x) (Sec. 2.2); NULL = every fluid
                                node with at least one solid nearest neighbour     */
  int32_t bc_z;              /* 0: periodic in z (paper, Sec. 2.2);
                                1: velocity inlet at z=0, pressure outlet at z=nz-1
                                (added by this library); x and y always periodic  */
  const float *theta_deg;    /* host, optional nx*ny*nz contact angles in degrees,
                                read at solid nodes; a wall node uses the D3Q19-
                                weighted mean over its solid neighbours (a spatial
                                wettability field, which the paper keeps uniform).
                                NULL = lbm_params.theta_deg everywhere             */
} lbm_geometry;

typedef struct {
  double tau;         /* relaxation time, > 0.5; nu = (tau - 1/2)/3 (Eq. kinematic_viscosity) */
  double sigma;       /* surface tension (Eq. continuum_surface_force)                        */
  double beta;        /* recolouring parameter (Eq. operator_recoloring)                      */
  double theta_deg;   /* contact angle in degrees, measured through the r phase               */
  double accel[3];    /* body acceleration a^k, same for both components                      */
  double diffusivity; /* D of the reactant C (D3Q7 BGK, tau_g = 4 D + 1/2), > 0               */
  double k_rate;      /* first-order surface rate k of the C-mode reaction                    */
  double c_init;      /* initial C for lbm_create's default start                             */
  double c_in;        /* inlet C (column mode)                                                */
  double u_in;        /* inlet velocity along +z (column mode)                                */
  double rho_out;     /* outlet density (column mode)                                         */
  double xi;          /* reaction rate of the paper's mode (Eq. reactive_boundary_condition_*) */
  int32_t reaction_mode; /* 0: delta = min(k NN r C psi, C, rho^r), C on D3Q7;
                            1: delta = min(xi NN r, 1) rho^r, C not evolved                  */
  int32_t storage;    /* population storage: 0 = FP32; 1 = FP16 deviations from the resting
                         reactant equilibrium (f^r - w, f^p, g - w, scaled by 2^12, so
                         deviations up to 16 in magnitude are representable), unbiased
                         stochastic rounding whose bits follow the step counter (reset with
                         it by lbm_init_fields / lbm_set_state), FP32 arithmetic              */
  void *cuda_stream;  /* cudaStream_t to launch on (borrowed); NULL = legacy default stream  */
} lbm_params;

typedef struct {
  double mass_r;          /* sum over fluid nodes of rho^r (Eq. reactant_mass)               */
  double mass_p;          /* sum of rho^p (Eq. product_mass)                                 */
  double mass_c;          /* sum of the reactant C                                           */
  double consumed;        /* cumulative sum of the reaction amounts delta since the start    */
  double rate;            /* sum of delta in the last step, = -dm^r/dt (Eq. production_rate) */
  double conversion;      /* periodic: consumed / m^C(0); column: 1 - flux_out / flux_in     */
  double gas_saturation;  /* mean over fluid nodes of (1 - rho^N)/2                          */
  double flux_in;         /* sum over fluid nodes of plane z=0 of u_z C                      */
  double flux_out;        /* same over plane z=nz-1                                          */
  int64_t step;           /* time steps taken since the state was last set                   */
  int64_t n_fluid;        /* number of fluid nodes                                           */
  int64_t n_bad;          /* fluid nodes with non-finite or non-positive rho^r + rho^p       */
} lbm_obs;

/* Intermediate fields of the last completed step (lbm_get_field), one float
 * per node unless noted.  Values at solid nodes are 0 except where noted. */
#define LBM_FIELD_RHON 0     /* rho^N, with the Eq. color_lattice_weighted_average values
                                at solid nodes next to the fluid                           */
#define LBM_FIELD_NORMAL 1   /* 3 floats per node (n_x, n_y, n_z), plane-major [3][N]:
                                wetted n at fluid nodes, averaged n at boundary solids      */
#define LBM_FIELD_GRADMAG 2  /* |grad rho^N| at fluid nodes                                */
#define LBM_FIELD_NS 3       /* 3 floats per node, [3][N]: solid normal n_s at wall nodes  */
#define LBM_FIELD_NN 4       /* NN(x) (Eq. nearest_solid_neighbors)                        */
#define LBM_FIELD_CURV 5     /* H (Eq. interface_curvature); needs lbm_set_debug(ctx, 1)   */
#define LBM_FIELD_DELTA 6    /* reaction amount delta of the last step; needs debug        */

/* Create a context: validates, copies the geometry to the device, builds the
 * static per-node data (bounce-back links, NN, r, wall flags, solid normals)
 * and the fluid-slot layout on the GPU (only three totals come back to the
 * host), and sets the equilibrium start rho^r = 1, rho^p = 0, u = 0,
 * C = c_init.  LBM_EINVAL also for a mask without fluid nodes (checked on
 * the host before any device call).  *out is set only on success. */
int lbm_create(const lbm_geometry *geom, const lbm_params *params, lbm_ctx **out);

/* Advance nsteps >= 0 time steps, asynchronously on the context's stream.
 * Unless profiling or debug output is on, each step is replayed from a CUDA
 * graph built at the first call (one graph launch per step). */
int lbm_step(lbm_ctx *ctx, int64_t nsteps);

/* Reduce the observables of the current (post-collision) state in FP64 on the
 * device, synchronise the stream and copy them to *out.  Returns LBM_ENAN
 * (with *out filled) if a fluid node holds a non-finite or non-positive density. */
int lbm_observables(lbm_ctx *ctx, lbm_obs *out);

/* Synchronise and copy the reaction sums kept by the step kernel (no extra
 * kernel): *rate = sum of delta in the last step, *consumed = cumulative sum.
 * Either pointer may be NULL.  This is the cheap per-step result read. */
int lbm_reaction(lbm_ctx *ctx, double *rate, double *consumed);

/* The same two values without synchronising: enqueues on the context's stream
 * one 16-byte copy of the last step's sum of delta into dst[0] and the cumulative
 * sum into dst[1] (host memory; page-locked memory keeps the copy asynchronous).  dst must
 * stay valid until the copies have run, i.e. until the next synchronising call on
 * the context or a synchronisation of its stream.  Call it before the next
 * lbm_step (the per-step slot is reused two steps later).  LBM_EINVAL before the
 * first step. */
int lbm_reaction_async(lbm_ctx *ctx, double *dst);

/* Equilibrium start from host fields of N floats each (u: 3*N, [3][N], or
 * NULL for rest): f^r = f^eq(rho_r, u), f^p = f^eq(rho_p, u), g = g^eq(conc, u).
 * Resets step, consumed and m^C(0). */
int lbm_init_fields(lbm_ctx *ctx, const float *rho_r, const float *rho_p,
                    const float *conc, const float *u);

/* Copy the current populations (45 * N floats, layout above) to / from host.
 * bytes must equal 45 * N * sizeof(float).  lbm_set_state resets step,
 * consumed and m^C(0), and rebuilds the column ghost planes from the state. */
int lbm_get_state(lbm_ctx *ctx, float *host_dst, size_t bytes);
int lbm_set_state(lbm_ctx *ctx, const float *host_src, size_t bytes);

/* Copy one LBM_FIELD_* of the last step to host; bytes must match exactly. */
int lbm_get_field(lbm_ctx *ctx, int32_t which, float *host_dst, size_t bytes);

/* 1: the step also stores H and delta per node (extra traffic; for checks). */
int lbm_set_debug(lbm_ctx *ctx, int32_t enable);

/* Per-kernel timing with CUDA events on the context's stream.  Kernel kinds:
 * 0 density, 1 solid colour, 2 normal, 3 solid normal, 4 main step,
 * 5 observables, 6 fused fields (solid colour, normals and solid normals in
 * one launch that marches through z with shared-memory planes, replacing
 * kinds 1-3).  lbm_profile(ctx, 1) resets and
 * starts; lbm_profile_read synchronises and returns total milliseconds and
 * launch counts (n <= 7). */
#define LBM_NKERNELS 7
int lbm_profile(lbm_ctx *ctx, int32_t enable);
int lbm_profile_read(lbm_ctx *ctx, double *ms, int64_t *launches, int32_t n);

/* Launch configuration of the step (not part of the paper): lbm_tune times each
 * candidate on the current state (main kernel 64/128/256 threads; colour-function
 * and normal kernels 128/256/512; then whole steps with the colour at solids,
 * the normals and the normals at solids as three kernels or as one kernel that
 * marches through z-chunks of 16, 32 or 64 planes with the colour field staged
 * in shared memory; then whole steps with the
 * kernels after the first launched as programmatic dependent launches, which
 * lets each one be scheduled while its predecessor's last blocks run, or as
 * plain launches) and keeps the fastest; blocks[5] (may be NULL) receives the
 * choice (main, density, normal, programmatic 1 / plain 0, fields: 0 three
 * kernels, 1 / 2 / 3 one marching kernel with chunks of 16 / 32 / 64 planes).
 * Every choice gives bit-identical results.  The state is not advanced.
 * Without a call: 128, 256, 256, 1, 0. */
int lbm_tune(lbm_ctx *ctx, int32_t *blocks);

/* Set the launch configuration directly (blocks[5] as filled by lbm_tune, e.g. a
 * tuning saved earlier).  LBM_EINVAL for a value outside the candidates.  The next step
 * rebuilds the step's CUDA graphs. */
int lbm_set_launch(lbm_ctx *ctx, const int32_t *blocks);

/* Static counts: fluid nodes, wall nodes, solid nodes next to the fluid,
 * device bytes held.  Any pointer may be NULL. */
int lbm_info(lbm_ctx *ctx, int64_t *n_fluid, int64_t *n_wall, int64_t *n_solid_bnd,
             int64_t *device_bytes);

/* Replace the contact-angle field (host, nx*ny*nz degrees read at solid nodes,
 * as lbm_geometry.theta_deg; NULL = the uniform params.theta_deg).  Synchronous;
 * LBM_EINVAL for a non-finite value. */
int lbm_set_wetting(lbm_ctx *ctx, const float *theta_deg);

/* Column mode: set the inlet velocity and concentration (rewrites the inlet
 * ghost plane, Eq. of the inlet reading: f^r = f^eq(1, u_in z), g = g^eq(c_in,
 * u_in z)).  LBM_EINVAL in a periodic box. */
int lbm_set_inlet(lbm_ctx *ctx, double u_in, double c_in);

/* ---------------------------------------------------------------------------
 * Reverse mode (discrete adjoint) of the outlet conversion of a column
 *
 *   J = 1 - Phi_out / Phi_in,  Phi = sum over the fluid nodes of plane z = 0
 *   (in) or z = nz - 1 (out) of u_z C,  u_z = j_z / rho of the stored state,
 *
 * after nsteps steps from the current state, differentiated with respect to the
 * per-solid-node contact angle (lbm_geometry.theta_deg) and the inlet velocity;
 * the start state is held fixed.  The paper's coating discussion (Sec. 5.2)
 * turns on how the wettability controls the conversion; this is its gradient.
 * Branch decisions of the forward (interface thresholds, the n_+/n_- choice,
 * the reaction clamps) are frozen.  Column mode, reaction_mode 0, FP32 storage
 * only (else LBM_EINVAL).
 *
 * lbm_adjoint_forward advances the state by nsteps exactly as lbm_step does,
 * storing a checkpoint every checkpoint_every steps (<= 0: ceil(sqrt(nsteps))),
 * and returns J in *objective (may be NULL).  Device memory for about
 * nsteps / K + K + 2 population states (K = checkpoint spacing), with the
 * density, normal and curvature fields of K states, is allocated on first use
 * and kept until lbm_destroy.  LBM_ENAN if Phi_in is zero or the fluxes are not
 * finite.
 *
 * lbm_adjoint_backward (valid until the state changes) recomputes each segment
 * from its checkpoint and runs the adjoint steps backwards.  Outputs, each
 * multiplied by seed (dL/dJ of an enclosing objective; 1 for dJ):
 *   dtheta_deg  host, nx*ny*nz doubles: dJ/dtheta per solid node, per degree
 *               (0 at fluid nodes and at solids without a wall neighbour)
 *   du_in       dJ/du_in
 *   dstate      host, 45*N floats in the lbm_get_state layout: dJ/df of the
 *               start state (state_bytes must equal 45 * N * sizeof(float))
 * Any output may be NULL.  The state and the LBM_FIELD_* buffers are left as the
 * forward left them. */
int lbm_adjoint_forward(lbm_ctx *ctx, int64_t nsteps, int64_t checkpoint_every, double *objective);
int lbm_adjoint_backward(lbm_ctx *ctx, double seed, double *dtheta_deg, double *du_in, float *dstate,
                         size_t state_bytes);

/* Release every device resource of the context; NULL is ignored. */
void lbm_destroy(lbm_ctx *ctx);

/* ---------------------------------------------------------------------------
 * Batches: many independent lattices of different sizes, masks and parameters
 * (e.g. a sweep over structures, contact angles or inlet velocities) advanced
 * together: every kernel of a time step is one launch over the fluid nodes of
 * all lattices, and a step is replayed as one CUDA graph.  Geometry k and
 * params k describe lattice k exactly as for lbm_create; all params must use
 * the same storage.  cuda_stream (borrowed) is used for every launch.
 * lbm_batch_set_state replaces lattice k's state and, as for lbm_set_state,
 * restarts the step counter and the reaction sums of the whole batch.
 * lbm_batch_observables fills count = n entries, one per lattice. */
typedef struct lbm_batch lbm_batch;   /* opaque, library-owned */
int lbm_batch_create(int32_t n, const lbm_geometry *geoms, const lbm_params *params, void *cuda_stream,
                     lbm_batch **out);
int lbm_batch_step(lbm_batch *batch, int64_t nsteps);
int lbm_batch_observables(lbm_batch *batch, lbm_obs *out, int32_t count);
int lbm_batch_get_state(lbm_batch *batch, int32_t k, float *host_dst, size_t bytes);
int lbm_batch_set_state(lbm_batch *batch, int32_t k, const float *host_src, size_t bytes);
int lbm_batch_tune(lbm_batch *batch, int32_t *blocks);
int lbm_batch_set_launch(lbm_batch *batch, const int32_t *blocks);
int lbm_batch_profile(lbm_batch *batch, int32_t max_launches);
int lbm_batch_profile_read(lbm_batch *batch, double *ms, int64_t *launches, int32_t n);
void lbm_batch_destroy(lbm_batch *batch);

/* ---------------------------------------------------------------------------
 * Allocation-free step.  The paper has no counterpart: this entry point exists
 * for callers that must not allocate device memory -- for example code that
 * runs while a memory pool or arena owns every allocation, a host process
 * whose allocator is locked down, or a stream that is being recorded and must
 * not see cudaMalloc / cudaFree.  It performs one time step of a periodic box
 * (bc_z = 0) on populations the caller already holds on the device, and keeps
 * every intermediate field (bounce-back links, solid normals, colour field,
 * interface normals, reaction sums) in one fixed scratch array compiled into
 * the library (about LBM_STATIC_MAX_NODES * 40 bytes, held on every GPU that
 * loads the library until the process exits).
 *
 *   nx, ny, nz    lattice size; nx * ny * nz <= LBM_STATIC_MAX_NODES, else
 *                 LBM_EINVAL (nothing is launched).
 *   solid         device, nx*ny*nz bytes, nonzero = solid (layout as lbm_geometry).
 *   reactive      device, optional r(x) mask, or NULL (fluid nodes with NN >= 1).
 *   f_in, f_out   device, 45 * nx*ny*nz floats each in the lbm_get_state layout
 *                 (index p * N + node); every entry of f_out is written: the
 *                 post-collision populations of the step at fluid nodes, zero
 *                 at solid nodes, and in the paper's reaction mode
 *                 (reaction_mode = 1, which does not evolve the reactant) the
 *                 seven reactant populations copied from f_in.  They must not
 *                 overlap.
 *   delta_sum     device, one double receiving the step's sum of reaction
 *                 amounts, or NULL.
 *   params        as for lbm_create (cuda_stream selects the stream; only
 *                 storage = 0 is accepted).
 *
 * Nothing is allocated or freed: no cudaMalloc, cudaFree or allocating library
 * call.  The first call on a device looks up the scratch array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  The static geometry is rebuilt on every
 * call (a few microseconds at the size limit).  All calls share the one
 * scratch array, which keeps the last call's contents (the reaction sums are
 * cleared at the start of each call): calls that may overlap on the GPU --
 * different streams, different host threads -- race and must be serialised by
 * the caller.  Returns LBM_OK, LBM_EINVAL or LBM_ECUDA (launch errors; kernel
 * faults surface at the caller's next synchronisation).  A CUDA error already
 * pending on the calling thread when the call starts is reported as
 * LBM_ECUDA before anything is launched and is left pending for the caller. */
#define LBM_STATIC_MAX_NODES 131072
int lbm_step_static(int32_t nx, int32_t ny, int32_t nz, const uint8_t *solid, const uint8_t *reactive,
                    const float *f_in, float *f_out, double *delta_sum, const lbm_params *params);

/* Static description of an error code. */
const char *lbm_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* CGLBM_H */
