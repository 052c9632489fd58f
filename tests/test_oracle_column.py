"""Pins of the oracle's column boundaries (inlet ghost, outlet ghost, column conversion).

The paper uses periodic boxes with a body force (Sec. 2.2, boundary conditions);
the inlet/outlet column of the reactive flow-through workload is this library's
addition, so its pins come from the mathematics, not from a printed number:

* the uniform state rho = 1, u = u_in z is an exact fixed point of an empty duct
  with rho_out = 1, and a duct started at rest converges to it: every z-plane then
  carries the mass flux u_in A, the outlet plane sits at rho_out and the column
  conversion 1 - Phi_out / Phi_in vanishes;
* the outlet ghost by non-equilibrium extrapolation reduces, for an equilibrium
  plane, to the equilibria at the prescribed density with the plane's velocity,
  split by the plane's colour ratio; for any plane the full ghost node has density
  rho_out, the plane's velocity and the plane's colour ratio;
* mass balance of one step: the change of the r, p and reactant masses equals
  what crosses the two end faces minus (plus) the reacted amount, with the inlet
  supplying the closed-form (1 + 3u + 3u^2)/6 of mixture and c_in (1 + 4u)/8 of
  reactant per inlet node;
* at steady state the mass crossing every inter-plane face is the same.
"""
import numpy as np
import pytest

from oracle import cglbm as O
from oracle.lattice import C19, C7

CZ19 = C19[:, 2]
CZ7 = C7[:, 2]


def _uniform(shape, u_in, dtype=np.float64):
    u = np.zeros((3,) + shape, dtype)
    u[2] = u_in
    return u


# --------------------------------------------------------------------- uniform duct
def test_uniform_duct_is_an_exact_fixed_point():
    shape = (8, 3, 2)
    g = O.Geometry(solid=np.zeros(shape, bool), bc_z=1)
    p = O.Params(k_rate=0.0, u_in=0.02, c_in=0.8, c_init=0.8, rho_out=1.0, bc_z=1)
    st = O.init_state(g, p, conc=np.full(shape, 0.8), u=_uniform(shape, p.u_in))
    nxt = O.step(st, g, p)
    assert np.abs(nxt.f - st.f).max() < 1e-15


@pytest.mark.parametrize("u_in", [0.02, -0.01])
def test_uniform_duct_converges_from_rest(u_in):
    """Started at rest, the empty duct reaches rho = 1, u = u_in z: plane fluxes u_in A, conversion 0.

    With u_in < 0 the flow leaves through the inlet and enters through the outlet,
    whose reactant ghost is a zero-gradient copy: under inflow that leaves the
    level of C free (every uniform C is a fixed point), so only the mixture
    populations are checked there."""
    shape = (8, 1, 1)
    g = O.Geometry(solid=np.zeros(shape, bool), bc_z=1)
    p = O.Params(k_rate=0.0, u_in=u_in, c_in=1.0, c_init=1.0, rho_out=1.0, bc_z=1)
    st = O.run(O.init_state(g, p), g, p, 2000)
    ref = O.init_state(g, p, u=_uniform(shape, u_in)).f
    npop = 45 if u_in > 0 else 38
    assert np.abs(st.f - ref)[:npop].max() < 2e-8
    F = st.f
    rho = (F[0:19] + F[19:38]).sum(0)
    jz = np.tensordot(CZ19.astype(float), F[0:19] + F[19:38], axes=(0, 0))
    assert np.abs(jz - u_in).max() < 2e-8                      # every plane: mass flux u_in A (A = 1)
    assert abs(rho[-1, 0, 0] - p.rho_out) < 2e-8               # outlet plane at the prescribed density
    if u_in > 0:
        ob = O.observables(st, g, p)
        assert abs(ob["conversion"]) < 1e-6
        assert abs(ob["flux_in"] - u_in) < 2e-8 and abs(ob["flux_out"] - u_in) < 2e-8


# --------------------------------------------------------------------- outlet ghost
def _random_plane(rng, shape2, nonequilibrium):
    rr = 0.2 + rng.random(shape2)
    rp = 0.2 + rng.random(shape2)
    v = 0.05 * rng.standard_normal((3,) + shape2)
    F = np.concatenate([O.feq(rr, v), O.feq(rp, v), O.geq(rng.random(shape2), v)], axis=0)
    if nonequilibrium:
        F = F + 1e-2 * rng.standard_normal(F.shape)
    solid = rng.random(shape2) < 0.25
    F[:, solid] = 0.0
    return F, rr, rp, v, solid


def test_outlet_ghost_of_an_equilibrium_plane():
    """Equilibrium input: ghost^r = f^eq(psi rho_out, v), ghost^p = f^eq((1 - psi) rho_out, v)."""
    rng = np.random.default_rng(3)
    F, rr, rp, v, solid = _random_plane(rng, (5, 7), nonequilibrium=False)
    p = O.Params(rho_out=1.03, bc_z=1)
    G = O.outlet_ghost(F, solid, p)
    psi = rr / (rr + rp)
    want_r = O.feq(psi * p.rho_out, v)
    want_p = O.feq((1.0 - psi) * p.rho_out, v)
    fl = ~solid
    assert np.abs(G[0:19] - want_r)[:, fl].max() < 1e-14
    assert np.abs(G[19:38] - want_p)[:, fl].max() < 1e-14
    assert np.abs(G[38:45] - F[38:45])[:, fl].max() == 0.0            # reactant: zero gradient
    # above a solid node: the resting reactant liquid at rho_out
    rest = O.feq(np.full(solid.shape, p.rho_out), np.zeros_like(v))
    assert np.abs(G[0:19] - rest)[:, solid].max() < 1e-15
    assert np.abs(G[19:45])[:, solid].max() == 0.0


def test_outlet_ghost_node_has_outlet_density_plane_velocity_and_colour():
    """Any input: the ghost node's density is rho_out, its velocity and colour ratio are the plane's."""
    rng = np.random.default_rng(4)
    F, _, _, _, solid = _random_plane(rng, (6, 5), nonequilibrium=True)
    p = O.Params(rho_out=0.97, bc_z=1)
    G = O.outlet_ghost(F, solid, p)
    fl = ~solid
    fm, gm = F[0:19] + F[19:38], G[0:19] + G[19:38]
    rho, rho_g = fm.sum(0), gm.sum(0)
    assert np.abs(rho_g - p.rho_out)[fl].max() < 1e-14
    for a in range(3):
        va = np.tensordot(C19[:, a].astype(float), fm, axes=(0, 0)) / np.where(fl, rho, 1.0)
        vg = np.tensordot(C19[:, a].astype(float), gm, axes=(0, 0)) / rho_g
        assert np.abs(va - vg)[fl].max() < 1e-14
    psi = F[0:19].sum(0) / np.where(fl, rho, 1.0)
    assert np.abs(G[0:19].sum(0) / rho_g - psi)[fl].max() < 1e-14


# --------------------------------------------------------------------- mass balance of one step
def _face_terms(F, G, solid, fluid, comp, cz):
    """(leaving through the inlet face, entering through the outlet face, leaving through it) of one component.

    comp: slice of the component's populations in F; cz: their z velocities."""
    out_in = sum(F[comp][i][0][fluid[0]].sum() for i in range(len(cz)) if cz[i] == -1)
    leave_out = sum(F[comp][i][-1][fluid[-1]].sum() for i in range(len(cz)) if cz[i] == 1)
    return out_in, leave_out


def _outlet_inflow(G, fluid_last, comp, vel):
    """Mass pulled from the outlet ghost plane G by the fluid nodes of the last plane."""
    tot = 0.0
    for i in range(len(vel)):
        if vel[i][2] != -1:
            continue
        src = np.roll(G[comp][i], shift=(int(vel[i][1]), int(vel[i][0])), axis=(0, 1))   # value at x - c
        tot += src[fluid_last].sum()
    return tot


@pytest.mark.parametrize("mode", [0, 1])
def test_column_mass_balance_of_one_step(mode):
    rng = np.random.default_rng(10 + mode)
    shape = (9, 6, 7)
    solid = rng.random(shape) < 0.3
    g = O.Geometry(solid=solid, bc_z=1)
    p = O.Params(sigma=0.03, theta_deg=60.0, k_rate=0.05, xi=0.3, u_in=0.015, c_in=0.7, rho_out=1.02,
                 reaction_mode=mode, bc_z=1)
    rr = rng.random(shape)
    st = O.init_state(g, p, rho_r=rr, rho_p=1.05 - rr, conc=rng.random(shape),
                      u=0.02 * rng.standard_normal((3,) + shape))
    st.f += 1e-3 * rng.standard_normal(st.f.shape)
    st.f[:, solid] = 0.0
    nxt = O.step(st, g, p)
    fl = g.fluid
    F = st.f
    G = O.outlet_ghost(F[:, -1], solid[-1], p)
    n0 = int(fl[0].sum())
    u = p.u_in
    m = {}
    for name, comp, vel, inflow in (("r", slice(0, 19), C19, n0 * (1 + 3 * u + 3 * u * u) / 6.0),
                                    ("p", slice(19, 38), C19, 0.0),
                                    ("c", slice(38, 45), C7, n0 * p.c_in * (1 + 4 * u) / 8.0)):
        cz = vel[:, 2]
        out_in, leave_out = _face_terms(F, G, solid, fl, comp, cz)
        enter_out = _outlet_inflow(G, fl[-1], comp, vel)
        before = F[comp][:, fl].sum()
        after = nxt.f[comp][:, fl].sum()
        m[name] = (after - before, inflow - out_in + enter_out - leave_out)
    d = nxt.rate
    assert d > 0
    scale = F[0:38][:, fl].sum()
    assert abs(m["r"][0] - (m["r"][1] - d)) < 1e-12 * scale
    assert abs(m["p"][0] - (m["p"][1] + d)) < 1e-12 * scale
    if mode == 0:
        assert abs(m["c"][0] - (m["c"][1] - d)) < 1e-12 * scale
    else:   # paper mode: the reactant populations are not evolved
        assert np.abs(nxt.f[38:45] - F[38:45])[:, fl].max() == 0.0


# --------------------------------------------------------------------- steady channel
def _face_flux(F, G, fluid, u_in):
    """Mixture mass crossing each face between planes z and z + 1 in one step, from the stored state F.

    Index 0 is the inlet face (z = -1/2), index nz the outlet face.  A population
    whose destination is solid bounces back and crosses nothing."""
    nz = F.shape[1]
    fm = F[0:19] + F[19:38]
    J = np.zeros(nz + 1)
    for i in range(19):
        c = C19[i]
        if c[2] == 0:
            continue
        # destination of each node's population i: x + c; keep it when that node is fluid
        dest_fluid = np.roll(fluid, shift=(-int(c[1]), -int(c[0])), axis=(1, 2))
        if c[2] == 1:
            for z in range(nz - 1):
                J[z + 1] += fm[i, z][fluid[z] & dest_fluid[z + 1]].sum()
            J[nz] += fm[i, nz - 1][fluid[nz - 1]].sum()                     # leaves through the outlet
        else:
            for z in range(1, nz):
                J[z] -= fm[i, z][fluid[z] & dest_fluid[z - 1]].sum()
            J[0] -= fm[i, 0][fluid[0]].sum()                                  # leaves through the inlet
            src = np.roll(G[i] + G[19 + i], shift=(int(c[1]), int(c[0])), axis=(0, 1))
            J[nz] -= src[fluid[nz - 1]].sum()                                 # enters from the outlet ghost
    J[0] += fluid[0].sum() * (1 + 3 * u_in + 3 * u_in * u_in) / 6.0          # enters from the inlet ghost
    return J


def test_channel_steady_state_carries_one_flux_through_every_plane():
    """Plate channel (solid plane x = 0, periodic y) driven by the inlet: at steady state the same
    mass crosses every face, and the outlet plane holds the prescribed density on average."""
    shape = (10, 1, 7)
    solid = np.zeros(shape, bool)
    solid[:, :, 0] = True
    g = O.Geometry(solid=solid, bc_z=1)
    p = O.Params(tau=0.9, k_rate=0.0, u_in=0.01, c_in=1.0, rho_out=1.0, bc_z=1)
    st = O.run(O.init_state(g, p), g, p, 2000)
    prev = st.f.copy()
    st = O.step(st, g, p)
    assert np.abs(st.f - prev)[0:38].max() < 1e-9             # steady mixture (C still diffuses slowly)
    G = O.outlet_ghost(st.f[:, -1], solid[-1], p)
    J = _face_flux(st.f, G, g.fluid, p.u_in)
    assert J[0] > 0
    assert np.abs(J / J[0] - 1).max() < 1e-9
    rho_last = (st.f[0:38].sum(0))[-1][g.fluid[-1]]
    assert abs(rho_last.mean() - p.rho_out) < 1e-3


def test_column_conversion_of_a_hand_built_state():
    """Uniform flow u_z = 0.01 carrying C = 1 through the first plane and C = 1/4 through the last:
    the last plane carries a quarter of the reactant flux, so the conversion is 3/4; the
    reactant's flux Phi = sum over a plane of u_z C is 0.01 A at the inlet and 0.0025 A at the outlet."""
    shape = (6, 2, 3)
    g = O.Geometry(solid=np.zeros(shape, bool), bc_z=1)
    p = O.Params(u_in=0.01, bc_z=1)
    conc = np.ones(shape)
    conc[-1] = 0.25
    st = O.init_state(g, p, conc=conc, u=_uniform(shape, 0.01))
    ob = O.observables(st, g, p)
    assert abs(ob["flux_in"] - 0.01 * 6) < 1e-15
    assert abs(ob["flux_out"] - 0.0025 * 6) < 1e-15
    assert abs(ob["conversion"] - 0.75) < 1e-13
