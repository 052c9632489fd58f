"""Physics pins run on the CUDA path, at sizes the CPU oracle cannot reach in a test.

The GPU step is pinned to the oracle element by element (test_gpu_parity); these
tests check that the method itself reproduces the closed forms when the geometry
is resolved:

* Laplace law in 3-D (Eq. continuum_surface_force, Eq. interface_curvature):
  spherical droplets and bubbles of radius 8, 12 and 16 in a 64^3 periodic box at
  sigma = 0.01, started with the Laplace jump in density; dp = (rho_in - rho_out)/3
  time-averaged against 2 sigma / R.  Measured +7.1 / +3.2 / +1.7 %, droplet and
  bubble alike: the error of a finite interface width, falling as 1/R^2.
* Contact angle on a flat wall (Eq. realigned_normal_vectors, Eq. normal_vector_solid):
  quasi-2-D caps large enough that the contact region spans many interface widths,
  started 20 - 40 degrees away from the imposed angle, relax to it within 3 degrees
  at 30, 60, 90, 120 and 150 degrees (30: 31.3 from above and 30.3 from below; 150:
  152.6 from above and below at radius 30, 151.6 at radius 45).
"""
import math

import numpy as np
import pytest

from paper_2608_15781_b300 import build, lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbm.load_library()


# --------------------------------------------------------------------- Laplace law
def _laplace_sphere(R0, inverse, n=64, sigma=0.01, steps=3000, avg_from=1500, every=50):
    shape = (n, n, n)
    solid = np.zeros(shape, bool)
    z, y, x = np.mgrid[0:n, 0:n, 0:n]
    c = n / 2 - 0.5
    r = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    phi = np.tanh((R0 - r) / 2.0)
    rho = 1.0 + (3 * 2 * sigma / R0) * (1 + phi) / 2
    if inverse:
        phi = -phi
    ratios = []
    with lbm.Lattice(solid, lbm.Params(sigma=sigma, k_rate=0.0)) as L:
        L.init_fields((rho * (1 + phi) / 2).astype(np.float32), (rho * (1 - phi) / 2).astype(np.float32),
                      np.ones(shape, np.float32))
        for k in range(steps // every):
            L.step(every)
            if (k + 1) * every < avg_from:
                continue
            f = L.get_state().astype(np.float64)
            rr, rp = f[0:19].sum(axis=0), f[19:38].sum(axis=0)
            rm = rr + rp
            rN = (rr - rp) / rm
            inner = ((1 + rN) / 2 if not inverse else (1 - rN) / 2).sum()
            R = (inner * 3 / (4 * math.pi)) ** (1 / 3)
            dp = (rm[r < R - 4].mean() - rm[r > R + 4].mean()) / 3
            ratios.append(dp / (2 * sigma / R))
    return float(np.mean(ratios)), float(np.min(ratios))


@pytest.mark.parametrize("R0,tol", [(8, 0.08), (12, 0.05), (16, 0.025)])
@pytest.mark.parametrize("inverse", [False, True])
def test_laplace_law_spheres(R0, tol, inverse):
    mean, lowest = _laplace_sphere(R0, inverse)
    assert lowest > 0                 # higher pressure inside, droplet and bubble
    assert abs(mean - 1) < tol, mean


# --------------------------------------------------------------------- contact angle
def _fit_circle(px, pz):
    A = np.c_[2 * px, 2 * pz, np.ones_like(px)]
    b = px ** 2 + pz ** 2
    (xc, zc, c), *_ = np.linalg.lstsq(A, b, rcond=None)
    return xc, zc, math.sqrt(c + xc ** 2 + zc ** 2)


def _measured_angle(rN, solid):
    """Angle through r of the circle fitted to the rho^N = 0 line, with the wall plane z = 1/2."""
    nz, _, nx = solid.shape
    rN = np.where(~solid, rN, np.nan)[:, 0, :]
    pts = []
    for zz in range(3, nz - 2):
        for xx in range(nx):
            a, b = rN[zz, xx], rN[zz, (xx + 1) % nx]
            if a * b < 0:
                pts.append((xx + a / (a - b), zz))
    for xx in range(nx):
        for zz in range(3, nz - 3):
            a, b = rN[zz, xx], rN[zz + 1, xx]
            if a * b < 0:
                pts.append((xx, zz + a / (a - b)))
    pts = np.array(pts)
    xc, zc, R = _fit_circle(pts[:, 0], pts[:, 1])
    return math.degrees(math.acos((0.5 - zc) / R))


def _cap(nx, nz, theta0, area):
    th = math.radians(theta0)
    R = math.sqrt(area / (th - math.sin(th) * math.cos(th)))
    zc = 0.5 - R * math.cos(th)
    z, x = np.mgrid[0:nz, 0:nx].astype(float)
    return np.tanh((R - np.sqrt((x - nx / 2) ** 2 + (z - zc) ** 2)) / 2.0)[:, None, :]


@pytest.mark.parametrize("theta,start,nx,nz,area,steps", [
    (30.0, 50.0, 256, 40, 1500, 60000),
    (30.0, 10.0, 256, 40, 1500, 60000),
    (60.0, 90.0, 192, 48, 2000, 30000),
    (90.0, 60.0, 128, 48, 1000, 30000),
    (120.0, 90.0, 128, 64, 2000, 30000),
    (150.0, 130.0, 128, 80, 2000, 30000),
    (150.0, 170.0, 128, 80, 2000, 30000),
])
def test_contact_angle_large_caps(theta, start, nx, nz, area, steps):
    shape = (nz, 1, nx)
    solid = np.zeros(shape, bool)
    solid[0] = solid[-1] = True
    phi = _cap(nx, nz, start, area)
    with lbm.Lattice(solid, lbm.Params(sigma=0.02, theta_deg=theta, k_rate=0.0, tau=0.7)) as L:
        L.init_fields(((1 + phi) / 2).astype(np.float32), ((1 - phi) / 2).astype(np.float32),
                      np.ones(shape, np.float32))
        L.step(steps)
        measured = _measured_angle(L.field(lbm.FIELD_RHON), solid)
    print(f"theta {theta}: {measured:.2f} degrees after {steps} steps from {start}")
    assert abs(measured - theta) < 3.0, measured
