"""Analysis of reactive-flow runs (host side): the paper's morphology statistics,
dimensionless numbers, nucleation-site rule, and effectiveness-factor model.

Nothing here is on the per-step hot path; these functions post-process
geometry masks and the observables time series of ``lbm_observables``.

Morphology (Sec. 3):
  surface area A = sum_x NN(x)                         (Eq. surface_area)
  porosity phi = sum_x l(x) / sum_x 1                  (Eq. porosity)
  reactor efficiency eta = kappa (A/V)^2
  permeability kappa = nu <u> / a                      (Eq. permeability)
Dimensionless numbers (Sec. 4.1, 4.2):
  Bo = drho g R^2 / sigma                              (Eq. bond_number)
  Bo_p = grad(p) R^2 / sigma                           (Eq. bond_number_pressure)
  Q = kappa V a / (nu L), t_f = nu L / (kappa a)       (Eq. volumetric_flow_rate, Eq. flow_timescale)
  t_xi = V / (xi A_r)                                  (Eq. reactive_timescale)
  Da = t_f / t_xi = xi A_r nu L / (kappa V a)          (Eq. damkohler_number)
  a = Bo_p sigma / (rho R^2)                           (parameter mapping, Sec. 4.2)
Reactive sites (Sec. 4.2): one site with exactly one solid nearest neighbour per
64^3 block, A_r = sum r NN (Eq. surface_area_reactive).
Effectiveness factor (Sec. 5.1):
  dm_th/dt = -xi A_r m^r / (phi V)                     (Eq. production_rate_theoretical)
  alpha = (dm^r/dt) / (dm_th/dt)                       (Eq. effectiveness_factor)
  alpha_bar(t) = (1/t) sum_{i<=t} alpha(i)             (Eq. effectiveness_factor_avg)
  m^r(t) = m^m exp(-xi A_r alpha t / (phi V))          (Eq. effectiveness_factor_solution)

Readings: <u> in the permeability is the superficial (volume-averaged) velocity
along the force, as in Darcy's law; the running average divides by the number
of samples.
"""
import math

import numpy as np

# the six nearest-neighbour offsets (|c|^2 = 1)
_NEAREST = ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1))


def nearest_solid_count(solid, periodic_z=True):
    """NN(x): solid nearest neighbours of each fluid node (0 at solid nodes), shape (nz, ny, nx)."""
    s = np.asarray(solid, dtype=bool)
    count = np.zeros(s.shape, dtype=np.int64)
    for dx, dy, dz in _NEAREST:
        sh = np.roll(s, shift=(-dz, -dy, -dx), axis=(0, 1, 2))
        if not periodic_z and dz != 0:
            # clamped z: outside the box continues the boundary plane
            if dz == 1:
                sh[-1] = s[-1]
            else:
                sh[0] = s[0]
        count += sh
    return np.where(s, 0, count)


def morphology(solid, periodic_z=True):
    """Surface area, porosity, volume and A/V of a mask (Sec. 3)."""
    s = np.asarray(solid, dtype=bool)
    nn = nearest_solid_count(s, periodic_z)
    V = s.size
    A = int(nn.sum())
    phi = float((~s).sum()) / V
    return {"surface_area": A, "porosity": phi, "volume": V, "area_to_volume": A / V}


def reactor_efficiency(kappa, area_to_volume):
    return kappa * area_to_volume ** 2


def permeability(nu, mean_velocity, accel):
    """Darcy permeability kappa = nu <u> / a (Eq. permeability), <u> superficial."""
    return nu * mean_velocity / accel


def kinematic_viscosity(tau):
    """nu = c_s^2 (tau - 1/2) (Eq. kinematic_viscosity)."""
    return (tau - 0.5) / 3.0


def bond_number(drho, g, R, sigma):
    return drho * g * R * R / sigma


def pressure_bond_number(grad_p, R, sigma):
    return grad_p * R * R / sigma


def pressure_gradient_for_bond(bo_p, R, sigma):
    """grad(p) that gives the pressure Bond number bo_p (inverse of Eq. bond_number_pressure)."""
    return bo_p * sigma / (R * R)


def acceleration_for_bond(bo_p, sigma, rho, R):
    """a = Bo_p sigma / (rho R^2): the body acceleration of the simulations (Sec. 4.2)."""
    return bo_p * sigma / (rho * R * R)


def laplace_pressure(sigma, R):
    """2 sigma / R across a spherical interface."""
    return 2.0 * sigma / R


def flow_timescale(nu, L, kappa, a):
    return nu * L / (kappa * a)


def reactive_timescale(V, xi, A_r):
    return V / (xi * A_r)


def damkohler(xi, A_r, nu, L, kappa, V, a):
    """Da = t_f / t_xi (Eq. damkohler_number)."""
    return xi * A_r * nu * L / (kappa * V * a)


def viscosity_for_damkohler(Da, xi, A_r, L, kappa, V, a):
    """nu giving the target Da at fixed geometry and forcing (the paper varies Da through nu)."""
    return Da * kappa * V * a / (xi * A_r * L)


def tau_for_viscosity(nu):
    return 3.0 * nu + 0.5


def nucleation_sites(solid, block=64, seed=0, periodic_z=True):
    """The paper's reactive-site rule: in every block^3 block, one fluid site with exactly one
    solid nearest neighbour (chosen with the given seed); blocks without such a site get none.
    Returns the boolean mask r(x)."""
    s = np.asarray(solid, dtype=bool)
    nn = nearest_solid_count(s, periodic_z)
    cand = (~s) & (nn == 1)
    rng = np.random.default_rng(seed)
    r = np.zeros(s.shape, dtype=bool)
    nz, ny, nx = s.shape
    for z0 in range(0, nz, block):
        for y0 in range(0, ny, block):
            for x0 in range(0, nx, block):
                sub = np.argwhere(cand[z0:z0 + block, y0:y0 + block, x0:x0 + block])
                if len(sub):
                    k = sub[rng.integers(len(sub))]
                    r[z0 + k[0], y0 + k[1], x0 + k[2]] = True
    return r


def reactive_surface_area(reactive, solid, periodic_z=True):
    """A_r = sum r(x) NN(x) (Eq. surface_area_reactive)."""
    nn = nearest_solid_count(solid, periodic_z)
    return int((np.asarray(reactive, dtype=bool) * nn).sum())


def theoretical_rate(m_r, xi, A_r, phi, V):
    """dm^r_th/dt = -xi A_r m^r / (phi V) (Eq. production_rate_theoretical)."""
    return -xi * A_r * np.asarray(m_r, dtype=np.float64) / (phi * V)


def effectiveness_factor(rate, m_r, xi, A_r, phi, V):
    """alpha = (dm^r/dt) / (dm^r_th/dt); ``rate`` is the consumed amount per step (= -dm^r/dt)."""
    return -np.asarray(rate, dtype=np.float64) / theoretical_rate(m_r, xi, A_r, phi, V)


def running_average(alpha):
    """alpha_bar(t): mean of alpha over the samples up to t (Eq. effectiveness_factor_avg)."""
    a = np.asarray(alpha, dtype=np.float64)
    return np.cumsum(a) / np.arange(1, a.size + 1)


def fit_effectiveness(t, m_r, m_m, xi, A_r, phi, V):
    """Least-squares alpha of m^r(t) = m^m exp(-xi A_r alpha t / (phi V)) (Eq. effectiveness_factor_solution).

    Fits log(m^r/m^m) = -k alpha t through the origin, k = xi A_r / (phi V).
    """
    t = np.asarray(t, dtype=np.float64)
    y = np.log(np.asarray(m_r, dtype=np.float64) / m_m)
    k = xi * A_r / (phi * V)
    return float(-(t @ y) / (k * (t @ t)))


def predicted_mass(t, m_m, alpha, xi, A_r, phi, V):
    return m_m * np.exp(-xi * A_r * alpha * np.asarray(t, dtype=np.float64) / (phi * V))
