"""Brute-force cross-check of the whole-lattice oracle on tiny boxes.

``oracle.pointwise`` evaluates one node at a time with pure Python loops,
recomputing every neighbour quantity, and writes the collision per component
as the operator split of Eq. operator_decomposition states it (with an
explicit inverse of T).  Agreement to rounding on random non-equilibrium
states, random masks, both z boundary modes and both reaction modes pins the
whole-lattice passes (indexing, ghost planes, bounce-back, the summed form of
the collision).
"""
import numpy as np
import pytest

from oracle import cglbm as O
from oracle.pointwise import PointwiseStep


def _case(bc, mode, seed, shape, solid_frac=0.25):
    rng = np.random.default_rng(seed)
    solid = rng.random(shape) < solid_frac
    p = O.Params(sigma=0.05, accel=(1e-4, 2e-5, -1e-5), theta_deg=60 + 10 * seed, k_rate=0.05,
                 bc_z=bc, u_in=0.01, rho_out=0.99, reaction_mode=mode, xi=0.4)
    g = O.Geometry(solid=solid, bc_z=bc)
    rr = rng.random(shape)
    rp = 1 - rr + 0.1 * rng.random(shape)
    st = O.init_state(g, p, rho_r=rr, rho_p=rp, conc=rng.random(shape),
                      u=0.02 * rng.standard_normal((3,) + shape))
    st.f += 1e-3 * rng.standard_normal(st.f.shape)
    st.f[:, g.solid] = 0.0
    return p, g, st


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("seed,shape", [(0, (7, 5, 6)), (1, (4, 4, 4))])
def test_pointwise_matches_lattice(bc, mode, seed, shape):
    p, g, st = _case(bc, mode, seed, shape)
    new, fl = O.step(st, g, p, return_fields=True)
    pw = PointwiseStep(st.f, g.solid, p)
    nz, ny, nx = shape
    worst = 0.0
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if g.solid[z, y, x]:
                    continue
                v, d = pw.update((x, y, z))
                worst = max(worst, np.abs(v - new.f[:, z, y, x]).max(), abs(d - fl.delta[z, y, x]))
    assert worst < 1e-13
    # the case exercises wetting and curvature
    assert g.wall.sum() > 0 and np.abs(fl.H).max() > 0.1


def test_pointwise_hand_mask_channel():
    """Hand-set 4x4x5 mask: a solid plane and a solid pillar; column boundaries."""
    solid = np.zeros((5, 4, 4), dtype=bool)
    solid[:, :, 0] = True          # wall plane x = 0
    solid[2, 2, 2] = True          # isolated solid node
    p = O.Params(sigma=0.1, theta_deg=45, k_rate=0.3, bc_z=1, u_in=0.02, rho_out=1.01, c_in=0.5)
    g = O.Geometry(solid=solid, bc_z=1)
    rng = np.random.default_rng(7)
    rr = np.clip(rng.random(solid.shape), 0.05, 1)
    st = O.init_state(g, p, rho_r=rr, rho_p=1.02 - rr)
    st.f += 1e-3 * rng.standard_normal(st.f.shape)
    st.f[:, g.solid] = 0.0
    new = O.step(st, g, p)
    pw = PointwiseStep(st.f, solid, p)
    for z, y, x in zip(*np.nonzero(g.fluid)):
        v, _ = pw.update((x, y, z))
        assert np.abs(v - new.f[:, z, y, x]).max() < 1e-13
