"""Whole-lattice FP64 oracle of one colour-gradient LB time step.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Each stage is a separate
plain pass over the whole lattice, in the order the paper applies them:

  a1  pull streaming + halfway bounce-back      Eq. lattice_boltzmann_equation,
                                                Eq. bounce_back (Sec. 2.2)
  a2  moments, colour function                  Eq. moments_components,
                                                Eq. moments_mixture, Eq. color_function
  a3  colour at solid nodes                     Eq. color_lattice_weighted_average
  a4  isotropic gradient, interface normal      Eq. finite_difference_scheme,
                                                Eq. color_gradient_normal
  a5  wetting: realigned normals                Eq. realigned_normal_vectors,
                                                Eq. normal_vector_solid
  a6  curvature                                 Eq. interface_curvature
  a7  CSF force, exact-difference velocity shift Eq. continuum_surface_force,
                                                Eq. delta_u, Eq. operator_perturbation
  a8  central-moment collision                  Eq. collision_operator,
                                                Eq. forward_transformation_vector,
                                                Eq. relaxation_matrix
  a9  recolouring                               Eq. operator_recoloring
  a10 surface reaction (+ advection-diffusion)  Eq. reactive_boundary_condition_*
  a11 observables                               Eq. reactant_mass, Eq. product_mass,
                                                Eq. production_rate

Readings of the paper (where it is silent, ambiguous or self-inconsistent):
  * n = +grad(rho^N)/|grad(rho^N)| (points into the reactant r); the printed
    minus sign would make recolouring anti-segregating and flip the Laplace
    jump.  H and the recolouring formula are used as printed.
  * the solid normal n_s points into the solid (as printed), so the imposed
    contact angle theta is measured through the r phase.
  * |grad rho^N| < 1e-5: n = 0 and H = 0.  1 - (n_s.n)^2 < 1e-6, n = 0 or an
    undefined n_s: wetting leaves n unchanged.  The n_+ / n_- choice keeps n_+
    on ties.  Both thresholds sit well above the FP32 rounding noise of the
    gradient (~1e-7), so FP32 and FP64 evaluations take the same decisions: a
    noise-level gradient must not switch on the full-strength recolouring in a
    random direction.
  * n at a solid node next to the fluid (needed by the curvature stencil) is the
    lattice-weighted average of the (wetted) fluid-neighbour normals,
    renormalised; zero if that average is shorter than 1e-5.
  * recolouring acts on the colour-blind post-collision populations:
    f^r* = (rho^r/rho^m) f^m* + beta rho^r rho^p/rho^m w_i cos(phi_i)
    (Latva-Kokko, whose beta-term equals the printed one since f^eq(rho,0)=w rho).
  * the equilibria and the shifted velocities c - u use the unforced mixture
    velocity u^m; the physical velocity is u^m + du/2.
  * reaction (not fixed by the paper beyond first-order kinetics): explicit
    Euler from the post-streaming densities, applied after recolouring as a
    w_i-shaped transfer from f^r to f^p.  Paper mode: delta = min(xi NN r, 1)
    rho^r.  Advection-diffusion mode (not in the paper): D3Q7 BGK reactant C,
    delta = min(k NN r C psi, C, rho^r), psi = rho^r/rho^m; the same delta is
    removed from C.  delta is clipped below at 0.
  * reactive sites r(x): every fluid node with NN >= 1 unless a mask is given.
  * column mode (bc_z = 1, not in the paper): populations enter from a constant
    inlet ghost plane z = -1 (f^r = f^eq(1, u_in z), f^p = 0,
    g = g^eq(c_in, u_in z)) and from an outlet ghost plane z = nz built from the
    previous post-collision state of plane nz-1 by non-equilibrium extrapolation
    to density rho_out (split by that node's colour ratio; g copied).  Colour
    and geometry stencils clamp z into [0, nz-1] (zero-gradient extension).
"""
import math
from dataclasses import dataclass, field

import numpy as np

from .lattice import (
    C19, OPP19, Q19, CS2, C7, OPP7, Q7, CS2_7, NEAREST6, GRAD_EPS, SIN2_EPS,
    C19L, W19L, NORM19L, C7L, W7L, E92L, OMEGA92L,
)

NPOP = 2 * Q19 + Q7  # 45 populations per node: f^r[19], f^p[19], g[7]


@dataclass
class Params:
    tau: float = 1.0            # relaxation time, nu = c_s^2 (tau - 1/2)  (Eq. kinematic_viscosity)
    sigma: float = 0.01         # surface tension (Eq. continuum_surface_force)
    beta: float = 0.7           # recolouring parameter (Eq. operator_recoloring)
    theta_deg: float = 90.0     # imposed contact angle (Eq. realigned_normal_vectors)
    accel: tuple = (0.0, 0.0, 0.0)  # body acceleration a^k (same for both components)
    diffusivity: float = 0.05   # advection-diffusion D (ours)
    k_rate: float = 1e-3        # first-order surface rate k (ours)
    c_init: float = 1.0         # initial reactant concentration (ours)
    c_in: float = 1.0           # inlet concentration (column mode)
    u_in: float = 0.0           # inlet velocity along +z (column mode)
    rho_out: float = 1.0        # outlet density (column mode)
    xi: float = 1.0             # paper-mode reaction rate (Eq. reactive_boundary_condition_reactant)
    reaction_mode: int = 0      # 0: reactant C on D3Q7 (ours); 1: paper (rho^r -> rho^p)
    bc_z: int = 0               # 0: periodic in z; 1: inlet z=0 / outlet z=nz-1


# ---------------------------------------------------------------------------
# neighbour access
# ---------------------------------------------------------------------------
_NB_CACHE = {}


def _neighbor_index(shape, d, zmode):
    """Flat gather index giving, for every node x, the node x + d (see ``neighbor``)."""
    key = (shape, tuple(int(v) for v in d), zmode)
    idx = _NB_CACHE.get(key)
    if idx is None:
        nz, ny, nx = shape
        z = np.arange(nz) + int(d[2])
        z = z % nz if zmode == "periodic" else np.clip(z, 0, nz - 1)
        y = (np.arange(ny) + int(d[1])) % ny
        x = (np.arange(nx) + int(d[0])) % nx
        idx = ((z[:, None, None] * ny + y[None, :, None]) * nx + x[None, None, :]).ravel()
        _NB_CACHE[key] = idx
    return idx


def neighbor(a, d, zmode):
    """Value of ``a`` at x + d for every node x.

    ``a`` has the lattice in its last three axes (z, y, x).  x and y are
    periodic; z is periodic (``zmode='periodic'``) or clamped into [0, nz-1]
    (``zmode='clamp'``, zero-gradient extension used in column mode).
    """
    shape = a.shape[-3:]
    idx = _neighbor_index(shape, d, zmode)
    lead = a.shape[:-3]
    return a.reshape(lead + (-1,))[..., idx].reshape(a.shape)


def _zmode(bc_z):
    return "periodic" if bc_z == 0 else "clamp"


# ---------------------------------------------------------------------------
# static geometry (Sec. 2.2)
# ---------------------------------------------------------------------------
@dataclass
class Geometry:
    solid: np.ndarray                    # s(x) as bool, shape (nz, ny, nx)
    bc_z: int
    fluid: np.ndarray = field(init=False)       # l(x)
    nn: np.ndarray = field(init=False)          # NN(x), Eq. nearest_solid_neighbors
    reactive: np.ndarray = field(init=False)    # r(x)
    wall: np.ndarray = field(init=False)        # fluid node with a solid D3Q19 neighbour
    solid_bnd: np.ndarray = field(init=False)   # solid node with a fluid D3Q19 neighbour
    ns: np.ndarray = field(init=False)          # solid normal at wall nodes, shape (3, ...)
    ns_ok: np.ndarray = field(init=False)       # n_s defined (non-zero stencil sum)
    reactive_mask: np.ndarray = None            # optional user r(x)
    theta_deg: np.ndarray = None                # optional per-node contact angle, read at solid nodes
    theta_wall: np.ndarray = field(init=False)  # contact angle seen by each wall node (degrees) or None

    def __post_init__(self):
        s = self.solid.astype(bool)
        self.solid = s
        zm = _zmode(self.bc_z)
        self.fluid = ~s
        l = self.fluid.astype(np.float64)
        # Eq. nearest_solid_neighbors: NN = l(x) * sum over |c|^2 = 1 of s(x + c)
        nn = np.zeros(s.shape, dtype=np.int64)
        for i in NEAREST6:
            nn += neighbor(s, C19[i], zm).astype(np.int64)
        self.nn = nn * self.fluid
        if self.reactive_mask is None:
            self.reactive = self.fluid & (self.nn >= 1)
        else:
            self.reactive = self.reactive_mask.astype(bool) & self.fluid
        any_solid_nb = np.zeros(s.shape, dtype=bool)
        any_fluid_nb = np.zeros(s.shape, dtype=bool)
        for i in range(Q19 - 1):
            any_solid_nb |= neighbor(s, C19[i], zm)
            any_fluid_nb |= neighbor(self.fluid, C19[i], zm)
        self.wall = self.fluid & any_solid_nb
        self.solid_bnd = s & any_fluid_nb
        # Eq. normal_vector_solid with the weights of Eq. eigth_order_weight_function
        acc = np.zeros((3,) + s.shape)
        for e, om in zip(E92L, OMEGA92L):
            sv = neighbor(s, e, zm).astype(np.float64)
            for a in range(3):
                acc[a] += om * sv * e[a]
        mag = np.sqrt((acc * acc).sum(axis=0))
        self.ns_ok = self.wall & (mag > 0.0)
        self.ns = np.where(self.ns_ok, acc / np.where(mag > 0.0, mag, 1.0), 0.0)
        self.theta_wall = None if self.theta_deg is None else wall_contact_angle(self.theta_deg, s, self.bc_z)

    @property
    def shape(self):
        return self.solid.shape


def wall_contact_angle(theta_deg, solid, bc_z):
    """Contact angle at every fluid node from a per-solid-node field (our reading of a
    spatially varying wettability, which the paper keeps uniform): the D3Q19-weighted
    mean of theta over the solid neighbours x + c_i (geometry stencil), defined where
    there is at least one; 0 elsewhere.  Uniform theta gives that value."""
    s = np.asarray(solid, dtype=bool)
    th = np.asarray(theta_deg, dtype=np.float64)
    zm = _zmode(bc_z)
    num = np.zeros(s.shape)
    den = np.zeros(s.shape)
    for i in range(Q19 - 1):
        sn = neighbor(s, C19[i], zm).astype(np.float64)
        num += W19L[i] * sn * neighbor(th, C19[i], zm)
        den += W19L[i] * sn
    return np.where(den > 0.0, num / np.where(den > 0.0, den, 1.0), 0.0)


# ---------------------------------------------------------------------------
# equilibria
# ---------------------------------------------------------------------------
def feq(rho, u):
    """Eq. equilibrium_distribution, second-order truncated; rho (...), u (3, ...)."""
    uu = (u * u).sum(axis=0)
    out = np.empty((Q19,) + rho.shape, dtype=rho.dtype)
    for i in range(Q19):
        cx, cy, cz = C19L[i]
        cu = cx * u[0] + cy * u[1] + cz * u[2]
        out[i] = W19L[i] * rho * (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2))
    return out


def geq(conc, u):
    """Linear D3Q7 equilibrium of the advected reactant (ours): w_j C (1 + c_j.u / c_s^2)."""
    out = np.empty((Q7,) + conc.shape, dtype=conc.dtype)
    for j in range(Q7):
        cx, cy, cz = C7L[j]
        cu = cx * u[0] + cy * u[1] + cz * u[2]
        out[j] = W7L[j] * conc * (1.0 + cu / CS2_7)
    return out


# ---------------------------------------------------------------------------
# state
# ---------------------------------------------------------------------------
@dataclass
class State:
    f: np.ndarray          # (45, nz, ny, nx) post-collision populations of the last step
    step: int = 0
    consumed: float = 0.0  # cumulative sum of delta over all steps
    rate: float = 0.0      # sum of delta of the last step (= -dm^r/dt in paper mode)
    mc0: float = 0.0       # reactant (C) mass when the state was initialised


def init_state(geom, params, rho_r=None, rho_p=None, conc=None, u=None, dtype=np.float64):
    """Equilibrium start: f^k = f^eq(rho^k, u), g = g^eq(C, u) at fluid nodes, 0 at solids."""
    shp = geom.shape
    rho_r = np.ones(shp, dtype) if rho_r is None else np.asarray(rho_r, dtype)
    rho_p = np.zeros(shp, dtype) if rho_p is None else np.asarray(rho_p, dtype)
    conc = np.full(shp, params.c_init, dtype) if conc is None else np.asarray(conc, dtype)
    u = np.zeros((3,) + shp, dtype) if u is None else np.asarray(u, dtype)
    f = np.zeros((NPOP,) + shp, dtype=dtype)
    f[0:19] = feq(rho_r, u)
    f[19:38] = feq(rho_p, u)
    f[38:45] = geq(conc, u)
    f[:, geom.solid] = 0.0
    st = State(f=f)
    st.mc0 = float(f[38:45][:, geom.fluid].sum(dtype=np.float64))
    return st


# ---------------------------------------------------------------------------
# a1: streaming with bounce-back, column ghosts
# ---------------------------------------------------------------------------
def outlet_ghost(fstar_last, solid_last, params):
    """Outlet ghost plane z = nz from the post-collision plane z = nz-1 (column mode).

    Non-equilibrium extrapolation to density rho_out: ghost = f* + psi^k
    [f^eq(rho_out, v) - f^eq(rho*, v)] with rho*, v the density and velocity of
    f^m* at the last plane; g is copied (zero gradient).  Above a solid node the
    ghost is the resting reactant equilibrium w_i rho_out with no reactant C.
    """
    fr, fp, g = fstar_last[0:19], fstar_last[19:38], fstar_last[38:45]
    fm = fr + fp
    rho = fm.sum(axis=0)
    rho_safe = np.where(solid_last, 1.0, rho)
    v = np.stack([np.tensordot(C19[:, a].astype(fm.dtype), fm, axes=(0, 0)) for a in range(3)]) / rho_safe
    psi = fr.sum(axis=0) / rho_safe
    corr = feq(np.full_like(rho, params.rho_out), v) - feq(rho_safe, v)
    gr = fr + psi * corr
    gp = fp + (1.0 - psi) * corr
    ghost = np.concatenate([gr, gp, g.copy()], axis=0)
    rest = np.concatenate(
        [feq(np.full_like(rho, params.rho_out), np.zeros_like(v)),
         np.zeros_like(fp), np.zeros_like(g)], axis=0)
    return np.where(solid_last[None], rest, ghost)


def inlet_ghost(params, shape2d, dtype):
    """Inlet ghost plane z = -1 (column mode): f^r = f^eq(1, u_in z), f^p = 0, g = g^eq(c_in, u_in z)."""
    one = np.ones(shape2d, dtype)
    uin = np.zeros((3,) + shape2d, dtype)
    uin[2] = params.u_in
    return np.concatenate([feq(one, uin), np.zeros((Q19,) + shape2d, dtype),
                           geq(params.c_in * one, uin)], axis=0)


def _velocity_set(p):
    """(velocity, opposite index) of population p in the 45-population layout."""
    if p < 38:
        i = p % 19
        base = p - i
        return C19[i], base + OPP19[i]
    j = p - 38
    return C7[j], 38 + OPP7[j]


def stream(F, geom, params):
    """a1: f_i(x, t+1) = f*_i(x - c_i, t); bounce-back f*_{opp(i)}(x, t) if x - c_i is solid."""
    out = np.zeros_like(F)
    nz = geom.shape[0]
    column = params.bc_z == 1
    if column:
        ghost_in = inlet_ghost(params, geom.shape[1:], F.dtype)
        ghost_out = outlet_ghost(F[:, nz - 1], geom.solid[nz - 1], params)
    for p in range(NPOP):
        c, op = _velocity_set(p)
        if p >= 38 and params.reaction_mode == 1:
            out[p] = F[p]          # paper mode: the reactant populations are not evolved
            continue
        pulled = neighbor(F[p], -c, "periodic")
        src_solid = neighbor(geom.solid, -c, "periodic")
        if column and c[2] == 1:       # source plane z = -1
            pulled[0] = neighbor(ghost_in[p][None], -c * np.array([1, 1, 0]), "periodic")[0]
            src_solid[0] = False
        if column and c[2] == -1:      # source plane z = nz
            pulled[nz - 1] = neighbor(ghost_out[p][None], -c * np.array([1, 1, 0]), "periodic")[0]
            src_solid[nz - 1] = False
        out[p] = np.where(src_solid, F[op], pulled)
    out[:, geom.solid] = 0.0
    return out


# ---------------------------------------------------------------------------
# a3 - a6: colour field, normals, wetting, curvature
# ---------------------------------------------------------------------------
def color_at_solids(rhoN, geom):
    """a3, Eq. color_lattice_weighted_average at solid nodes with a fluid neighbour."""
    zm = _zmode(geom.bc_z)
    l = geom.fluid.astype(rhoN.dtype)
    num = np.zeros_like(rhoN)
    den = np.zeros_like(rhoN)
    for i in range(Q19):
        ln = neighbor(l, C19[i], zm)
        num += W19L[i] * neighbor(rhoN, C19[i], zm) * ln
        den += W19L[i] * ln
    out = rhoN.copy()
    sb = geom.solid_bnd
    out[sb] = num[sb] / den[sb]
    return out


def gradient(phi, geom):
    """Eq. finite_difference_scheme: grad phi = (1/c_s^2) sum_i w_i c_i phi(x + c_i)."""
    zm = _zmode(geom.bc_z)
    g = np.zeros((3,) + phi.shape, dtype=phi.dtype)
    for i in range(Q19):
        if not any(C19L[i]):
            continue
        v = neighbor(phi, C19[i], zm)
        for a in range(3):
            if C19L[i][a]:
                g[a] += (W19L[i] / CS2 * C19L[i][a]) * v
    return g


def wetting(n, geom, params):
    """a5, Eq. realigned_normal_vectors at wall nodes; keeps whichever of n_+/n_- is closer to n.

    theta is params.theta_deg, or per node geom.theta_wall when the geometry carries
    a per-solid-node contact angle.
    """
    if geom.theta_wall is None:
        th = math.radians(params.theta_deg)
        cos_th, sin_th = math.cos(th), math.sin(th)
    else:
        th = np.radians(geom.theta_wall)
        cos_th, sin_th = np.cos(th).astype(n.dtype), np.sin(th).astype(n.dtype)
    ns = geom.ns.astype(n.dtype)
    cos_tp = (ns * n).sum(axis=0)                       # cos(theta') = n_s . n
    nz_n = (n * n).sum(axis=0) > 0.0
    ok = geom.ns_ok & nz_n & (1.0 - cos_tp * cos_tp >= SIN2_EPS)
    cos_tp_s = np.where(ok, cos_tp, 0.0)
    sin_tp = np.sqrt(np.where(ok, 1.0 - cos_tp_s * cos_tp_s, 1.0))   # sin(arccos(.)) >= 0
    out = n.copy()
    cands = []
    for sgn in (+1.0, -1.0):
        # cos(+-theta) = cos(theta), sin(+-theta) = +-sin(theta)
        a_s = cos_th - sgn * sin_th * cos_tp_s / sin_tp
        a_n = sgn * sin_th / sin_tp
        cands.append(a_s * ns + a_n * n)
    d_plus = ((cands[0] - n) ** 2).sum(axis=0)
    d_minus = ((cands[1] - n) ** 2).sum(axis=0)
    pick = np.where(d_plus <= d_minus, 1, 0)
    chosen = np.where(pick[None] == 1, cands[0], cands[1])
    out = np.where(ok[None], chosen, n)
    return out


def normals_at_solids(n, geom):
    """n at solid nodes next to the fluid: weighted average of fluid-neighbour n, renormalised."""
    zm = _zmode(geom.bc_z)
    l = geom.fluid.astype(n.dtype)
    acc = np.zeros_like(n)
    for i in range(Q19):
        ln = neighbor(l, C19[i], zm)
        for a in range(3):
            acc[a] += W19L[i] * ln * neighbor(n[a], C19[i], zm)
    mag = np.sqrt((acc * acc).sum(axis=0))
    ok = geom.solid_bnd & (mag >= GRAD_EPS)
    out = np.where(geom.fluid[None], n, 0.0)
    out = np.where(ok[None], acc / np.where(mag > 0, mag, 1.0), out)
    return out


def curvature(n, geom):
    """Eq. interface_curvature: H = - sum_ab (delta_ab - n_a n_b) d_a n_b, d by Eq. finite_difference_scheme."""
    D = np.stack([gradient(n[b], geom) for b in range(3)], axis=1)  # D[a, b] = d_a n_b
    tr = D[0, 0] + D[1, 1] + D[2, 2]
    nDn = np.einsum("a...,ab...,b...->...", n, D, n)
    return -(tr - nDn)


# ---------------------------------------------------------------------------
# a8: central-moment collision (Appendix A)
# ---------------------------------------------------------------------------
def transform_matrix(u):
    """T with columns t_i of Eq. forward_transformation_vector at c_bar = c - u (Eq. local_fluid_velocity).

    u has shape (3, N); returns (N, 19, 19) with T[n, m, i] = t_i[m].
    """
    cb = C19.T[None, :, :].astype(u.dtype) - u.T[:, :, None]   # (N, 3, 19)
    x, y, z = cb[:, 0], cb[:, 1], cb[:, 2]
    T = np.empty((u.shape[1], Q19, Q19), dtype=u.dtype)
    T[:, 0] = 1.0
    T[:, 1], T[:, 2], T[:, 3] = x, y, z
    T[:, 4] = x * x + y * y + z * z
    T[:, 5] = x * x - y * y
    T[:, 6] = y * y - z * z
    T[:, 7], T[:, 8], T[:, 9] = x * y, x * z, y * z
    T[:, 10], T[:, 11] = x * x * y, x * y * y
    T[:, 12], T[:, 13] = x * x * z, x * z * z
    T[:, 14], T[:, 15] = y * y * z, y * z * z
    T[:, 16], T[:, 17], T[:, 18] = x * x * y * y, x * x * z * z, y * y * z * z
    return T


def cm_collision_backtransform(fm, u, tau, chunk=65536):
    """T^{-1} (I - R) T f^m (Eq. collision_operator, Eq. post_collision_moments_vector).

    fm (19, N), u (3, N).  The relaxation matrix R of Eq. relaxation_matrix is
    1 everywhere except 1/tau for moments 5..9, so k* is non-zero only there.
    T^{-1} k* is obtained with a linear solve (the definition), node by node.
    """
    dt = fm.dtype
    relax = np.ones(Q19, dtype=dt)
    relax[5:10] = 1.0 / tau
    one_minus_R = 1.0 - relax
    N = fm.shape[1]
    if not one_minus_R.any():
        # tau = 1: R = I, so k* = 0 and the solution of T y = 0 is y = 0
        return np.zeros((Q19, N), dtype=dt)
    out = np.empty((Q19, N), dtype=dt)
    for s in range(0, N, chunk):
        e = min(N, s + chunk)
        T = transform_matrix(u[:, s:e])
        k = np.einsum("nmi,in->nm", T, fm[:, s:e]) * one_minus_R[None, :]
        out[:, s:e] = np.linalg.solve(T, k[:, :, None])[:, :, 0].T
    return out


# ---------------------------------------------------------------------------
# the step
# ---------------------------------------------------------------------------
@dataclass
class StepFields:
    """Intermediate fields of the last step (post-streaming time level)."""
    rho_r: np.ndarray
    rho_p: np.ndarray
    conc: np.ndarray
    u: np.ndarray
    rhoN: np.ndarray      # with solid-node extrapolation (a3)
    grad_mag: np.ndarray
    n: np.ndarray         # wetted normal at fluid nodes, A6 average at boundary solids
    H: np.ndarray
    du: np.ndarray
    delta: np.ndarray


def step(state, geom, params, return_fields=False):
    """One time step a1..a10; returns the new State (and the intermediate fields)."""
    dt = state.f.dtype
    fl = geom.fluid
    # a1
    Fs = stream(state.f, geom, params)
    fr, fp, g = Fs[0:19], Fs[19:38], Fs[38:45]
    # a2: Eq. moments_components / moments_mixture (rho_0 = 1), Eq. color_function
    rho_r = fr.sum(axis=0)
    rho_p = fp.sum(axis=0)
    fm = fr + fp
    rho_m = rho_r + rho_p
    rho_m_safe = np.where(fl, rho_m, 1.0)
    u = np.stack([np.tensordot(C19[:, a].astype(dt), fm, axes=(0, 0)) for a in range(3)]) / rho_m_safe
    u = np.where(fl[None], u, 0.0)
    conc = g.sum(axis=0)
    rhoN = np.where(fl, (rho_r - rho_p) / rho_m_safe, 0.0)
    # a3
    rhoN = color_at_solids(rhoN, geom)
    # a4
    grad = gradient(rhoN, geom)
    gmag = np.sqrt((grad * grad).sum(axis=0))
    has_n = fl & (gmag >= GRAD_EPS)
    n = np.where(has_n[None], grad / np.where(has_n, gmag, 1.0), 0.0)
    # a5
    n = wetting(n, geom, params)
    n = np.where(fl[None], n, 0.0)
    # A6 reading: n at boundary solids for the curvature stencil
    n_all = normals_at_solids(n, geom)
    # a6
    H = np.where(has_n, curvature(n_all, geom), 0.0)
    # a7: du = F^k / rho^k = 0.5 sigma H grad(rho^N) / rho^m + a, grad(rho^N) = |grad| n_wet
    acc = np.asarray(params.accel, dtype=dt).reshape(3, 1, 1, 1)
    du = 0.5 * params.sigma * H * gmag * n / rho_m_safe + acc
    du = np.where(fl[None], du, 0.0)
    # a8: f^m* = f^m + Omega^(1) + Omega^CM = f^eq(rho^m, u + du) + T^{-1} k*
    idx = np.nonzero(fl.ravel())[0]
    fm_flat = fm.reshape(Q19, -1)[:, idx]
    u_flat = u.reshape(3, -1)[:, idx]
    bt = np.zeros((Q19, fl.size), dtype=dt)
    bt[:, idx] = cm_collision_backtransform(fm_flat, u_flat, params.tau)
    fm_star = feq(rho_m_safe, u + du) + bt.reshape((Q19,) + fl.shape)
    # a9: recolouring
    psi = rho_r / rho_m_safe
    fr_star = np.empty_like(fm_star)
    for i in range(Q19):
        cx, cy, cz = C19L[i]
        cn = cx * n[0] + cy * n[1] + cz * n[2]
        rec = params.beta * rho_r * rho_p / rho_m_safe * W19L[i] * (cn / NORM19L[i] if NORM19L[i] > 0 else 0.0)
        fr_star[i] = psi * fm_star[i] + rec
    fp_star = fm_star - fr_star
    # a10: reaction
    rmask = geom.reactive.astype(dt)
    nn = geom.nn.astype(dt)
    if params.reaction_mode == 1:
        delta = np.minimum(params.xi * nn * rmask, 1.0) * rho_r
    else:
        delta = np.minimum(np.minimum(params.k_rate * nn * rmask * conc * psi, conc), rho_r)
    delta = np.where(fl, np.maximum(delta, 0.0), 0.0)
    w19 = np.array(W19L, dtype=dt).reshape(-1, 1, 1, 1)
    fr_star = fr_star - w19 * delta
    fp_star = fp_star + w19 * delta
    if params.reaction_mode == 1:
        g_star = g
    else:
        tau_g = params.diffusivity / CS2_7 + 0.5
        u_phys = u + 0.5 * du
        g_star = g - (g - geq(conc, u_phys)) / tau_g - np.array(W7L, dtype=dt).reshape(-1, 1, 1, 1) * delta
    Fn = np.concatenate([fr_star, fp_star, g_star], axis=0).astype(dt)
    Fn[:, geom.solid] = 0.0
    dsum = float(delta.sum(dtype=np.float64))
    new = State(f=Fn, step=state.step + 1, consumed=state.consumed + dsum, rate=dsum, mc0=state.mc0)
    if return_fields:
        return new, StepFields(rho_r, rho_p, conc, u, rhoN, gmag, n_all, H, du, delta)
    return new


def run(state, geom, params, nsteps):
    for _ in range(nsteps):
        state = step(state, geom, params)
    return state


# ---------------------------------------------------------------------------
# a11: observables of the stored (post-collision) state
# ---------------------------------------------------------------------------
def observables(state, geom, params):
    """Masses (Eq. reactant_mass, Eq. product_mass), reactant mass, conversion, gas saturation, fluxes.

    Gas saturation S_g = sum over fluid nodes of (1 - rho^N)/2 divided by the
    number of fluid nodes.  Conversion: consumed / m^C(0) in a periodic box;
    1 - Phi_out/Phi_in in column mode with Phi = sum over a plane of u_z C.
    ``rate`` is the last step's sum of delta (the paper's -dm^r/dt).
    """
    F = state.f.astype(np.float64)
    fl = geom.fluid
    fr, fp, g = F[0:19], F[19:38], F[38:45]
    rr = fr.sum(axis=0)
    rp = fp.sum(axis=0)
    rm = rr + rp
    cc = g.sum(axis=0)
    rms = np.where(fl, rm, 1.0)
    rhoN = (rr - rp) / rms
    uz = np.tensordot(C19[:, 2].astype(np.float64), fr + fp, axes=(0, 0)) / rms
    nf = int(fl.sum())
    out = dict(
        mass_r=float(rr[fl].sum()),
        mass_p=float(rp[fl].sum()),
        mass_c=float(cc[fl].sum()),
        consumed=state.consumed,
        rate=state.rate,
        gas_saturation=float(((1.0 - rhoN) * 0.5)[fl].sum() / max(nf, 1)),
        flux_in=float((uz * cc)[0][fl[0]].sum()),
        flux_out=float((uz * cc)[-1][fl[-1]].sum()),
        step=state.step,
        n_fluid=nf,
    )
    if params.bc_z == 1:
        out["conversion"] = 1.0 - out["flux_out"] / out["flux_in"] if out["flux_in"] != 0 else 0.0
    else:
        out["conversion"] = state.consumed / state.mc0 if state.mc0 != 0 else 0.0
    return out
