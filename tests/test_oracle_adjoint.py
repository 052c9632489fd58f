"""FP64 adjoint reference (oracle.adjoint) pinned against the NumPy oracle.

1. Its forward step is the oracle's step (random states, per-node contact
   angle, both z boundary modes, both reaction modes) to rounding.
2. Its autograd gradient of the column conversion agrees with FP64 central
   differences of the NumPy oracle along random directions in the per-node
   contact angle and in the inlet velocity.
"""
import numpy as np
import pytest
import torch

from oracle import adjoint as A
from oracle import cglbm as O


def _bubbly(shape, seed, bc, mode=0):
    """A liquid column with gas pockets touching the walls (interfaces at wall nodes)."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    solid = np.zeros(shape, dtype=bool)
    solid[:, 0, :] = True                          # a wall plane y = 0
    solid |= rng.random(shape) < 0.12
    solid[0] &= False
    solid[-1] &= False
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    gas = ((xx - nx / 2) ** 2 + (yy - 1.5) ** 2 + (zz - nz / 2) ** 2) < (min(nx, nz) / 3.2) ** 2
    rr = np.where(gas, 0.05, 1.0) + 0.02 * rng.random(shape)
    rp = np.where(gas, 0.95, 0.02)
    p = O.Params(sigma=0.02, theta_deg=60.0, k_rate=0.02, bc_z=bc, u_in=0.01, c_in=1.0, rho_out=1.0,
                 reaction_mode=mode, xi=0.3, accel=(0.0, 0.0, 1e-5 if bc == 0 else 0.0))
    theta = rng.uniform(30.0, 120.0, shape)
    g = O.Geometry(solid=solid, bc_z=bc, theta_deg=theta)
    u = np.zeros((3,) + shape)
    u[2] = p.u_in if bc == 1 else 0.0              # start from the inflow velocity
    st = O.init_state(g, p, rho_r=rr, rho_p=rp, u=u)
    st.f += 1e-4 * rng.standard_normal(st.f.shape)
    st.f[:, solid] = 0.0
    return p, g, st, theta


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_torch_step_equals_oracle_step(bc, mode):
    p, g, st, theta = _bubbly((9, 7, 8), 11 + bc, bc, mode)
    ts = A.TorchStep(g, p)
    tw = ts.wall_theta(torch.from_numpy(theta))
    assert torch.allclose(tw, torch.from_numpy(g.theta_wall), atol=1e-12, rtol=0)
    f = torch.from_numpy(st.f.copy())
    for _ in range(3):
        st = O.step(st, g, p)
        f = ts.step(f, tw, torch.tensor(p.u_in, dtype=torch.float64))
        assert np.abs(f.numpy() - st.f).max() < 1e-12
    if bc == 1:
        assert abs(float(ts.conversion(f)) - O.observables(st, g, p)["conversion"]) < 1e-12


def test_gradient_matches_central_differences():
    p, g, st, theta = _bubbly((10, 8, 8), 3, 1)
    nsteps = 4
    J, dth, du = A.conversion_gradient(g, p, st.f, theta, nsteps)
    assert abs(J - A.conversion_forward(g, p, st.f, theta, nsteps)) < 1e-12
    # only solid nodes next to a wall node can carry a theta sensitivity
    assert np.all(dth[g.fluid] == 0.0)
    assert np.abs(dth).max() > 0.0
    rng = np.random.default_rng(0)
    h = 1e-3
    for _ in range(3):
        v = rng.standard_normal(theta.shape) * g.solid
        jp = A.conversion_forward(g, p, st.f, theta + h * v, nsteps)
        jm = A.conversion_forward(g, p, st.f, theta - h * v, nsteps)
        fd = (jp - jm) / (2 * h)
        ad = float((dth * v).sum())
        assert abs(fd - ad) <= 1e-6 * abs(ad) + 1e-12, (fd, ad)
    hu = 1e-6
    import dataclasses
    jp = A.conversion_forward(g, dataclasses.replace(p, u_in=p.u_in + hu), st.f, theta, nsteps)
    jm = A.conversion_forward(g, dataclasses.replace(p, u_in=p.u_in - hu), st.f, theta, nsteps)
    fd = (jp - jm) / (2 * hu)
    assert abs(fd - du) <= 1e-6 * abs(du), (fd, du)
