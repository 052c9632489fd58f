"""Per-solid-node contact angle in the oracle (the wetting parameter of the adjoint).

The paper imposes one contact angle (Eq. realigned_normal_vectors); a spatially
varying wettability is read as: each wall node uses the D3Q19-weighted mean of
theta over its solid neighbours.  Pins: a hand-computed mean on a flat wall,
reduction to the scalar path for a uniform field, and the naive per-node
cross-check with a random field.
"""
import numpy as np
import pytest

from oracle import cglbm as O
from oracle.pointwise import PointwiseStep


def test_wall_mean_on_flat_wall_by_hand():
    solid = np.zeros((6, 5, 5), dtype=bool)
    solid[0] = True                              # flat wall z = 0 (periodic z: also below z = 5)
    th = np.full(solid.shape, 90.0)
    th[0, 2, 2] = 30.0                           # the node right below (x, y) = (2, 2)
    tw = O.wall_contact_angle(th, solid, bc_z=1)
    # solid neighbours of (2, 2, 1): (0,0,-1) weight 1/18, four (+-1,0,-1), (0,+-1,-1) weight 1/36
    assert abs(tw[1, 2, 2] - (30 / 18 + 4 * 90 / 36) / (1 / 18 + 4 / 36)) < 1e-12   # = 70 degrees
    assert abs(tw[1, 2, 3] - (90 / 18 + 3 * 90 / 36 + 30 / 36) / (1 / 18 + 4 / 36)) < 1e-12
    assert tw[3, 2, 2] == 0.0                    # no solid neighbour


def _case(seed, bc, shape=(7, 6, 5)):
    rng = np.random.default_rng(seed)
    solid = rng.random(shape) < 0.3
    p = O.Params(sigma=0.05, theta_deg=60.0, k_rate=0.05, bc_z=bc, u_in=0.01)
    rr = rng.random(shape)
    return rng, solid, p, rr


@pytest.mark.parametrize("bc", [0, 1])
def test_uniform_field_reduces_to_scalar(bc):
    rng, solid, p, rr = _case(3, bc)
    g0 = O.Geometry(solid=solid, bc_z=bc)
    g1 = O.Geometry(solid=solid, bc_z=bc, theta_deg=np.full(solid.shape, p.theta_deg))
    st = O.init_state(g0, p, rho_r=rr, rho_p=1 - rr + 0.05)
    st.f += 1e-3 * rng.standard_normal(st.f.shape)
    st.f[:, solid] = 0.0
    a = O.step(st, g0, p)
    b = O.step(st, g1, p)
    assert np.abs(a.f - b.f).max() < 1e-14
    assert np.abs(g1.theta_wall[g1.wall] - p.theta_deg).max() < 1e-12


@pytest.mark.parametrize("bc", [0, 1])
def test_random_field_matches_pointwise(bc):
    rng, solid, p, rr = _case(5, bc)
    th = rng.uniform(20.0, 150.0, solid.shape)
    g = O.Geometry(solid=solid, bc_z=bc, theta_deg=th)
    st = O.init_state(g, p, rho_r=rr, rho_p=1 - rr + 0.05)
    st.f += 1e-3 * rng.standard_normal(st.f.shape)
    st.f[:, solid] = 0.0
    new, fl = O.step(st, g, p, return_fields=True)
    pw = PointwiseStep(st.f, solid, p, theta=th)
    for z, y, x in zip(*np.nonzero(g.fluid)):
        v, _ = pw.update((x, y, z))
        assert np.abs(v - new.f[:, z, y, x]).max() < 1e-13
    # the field changes the result (the case has wetting nodes on an interface)
    other = O.step(st, O.Geometry(solid=solid, bc_z=bc), p)
    assert np.abs(other.f - new.f).max() > 1e-6
