"""Oracle pins for the lattice constants and the central-moment collision.

Checked against what the paper and the mathematics fix, not against the
oracle itself:
  * D3Q19 weights and isotropy (Sec. 2.1, Eq. d3q19_weight_function), the
    92-vector eighth-order stencil (Eq. eigth_order_weight_function);
  * the paper's printed closed-form rows of T^{-1} k* (Appendix A,
    Eq. back_transformation_vector, typed into tests/golden/) against the
    oracle's linear solve of the definition (Eq. collision_operator);
  * collision invariants: mass, momentum (plus the exact-difference momentum
    rho du), shear central moments scaled by (1 - 1/tau), the bulk central
    moment relaxed to equilibrium;
  * per-node conservation of each component through recolouring and of the
    colour-blind populations through the reaction.
"""
import os

import numpy as np
import pytest
import sympy

from oracle import cglbm as O
from oracle.lattice import C19, W19, OPP19, E92, OMEGA92, CS2, C7, W7

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_d3q19_weights_and_isotropy():
    assert abs(W19.sum() - 1.0) < 1e-15
    # second-order isotropy: sum_i w_i c_ia c_ib = c_s^2 delta_ab
    M2 = np.einsum("i,ia,ib->ab", W19, C19, C19)
    assert np.allclose(M2, CS2 * np.eye(3), atol=1e-15)
    # fourth-order isotropy needed by the second-order equilibrium
    M4 = np.einsum("i,ia,ib,ic,id->abcd", W19, C19, C19, C19, C19)
    d = np.eye(3)
    ref = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(M4, ref, atol=1e-15)
    assert all((C19[OPP19[i]] == -C19[i]).all() for i in range(19))
    # the rest vector is last (Sec. 2.1, matrix M)
    assert (C19[18] == 0).all()


def test_d3q7_isotropy():
    assert abs(W7.sum() - 1.0) < 1e-15
    M2 = np.einsum("i,ia,ib->ab", W7, C7, C7)
    assert np.allclose(M2, 0.25 * np.eye(3), atol=1e-15)


def test_eighth_order_stencil():
    assert len(E92) == 92
    sq = set(int(v) for v in (E92 * E92).sum(axis=1))
    assert sq == {1, 2, 3, 4, 5, 6, 8}
    M2 = np.einsum("i,ia,ib->ab", OMEGA92, E92, E92)
    assert np.allclose(M2, np.eye(3), atol=1e-14)


def _printed_rows():
    ux, uy, uz, k5, k6, k7, k8, k9 = sympy.symbols("ux uy uz k5 k6 k7 k8 k9")
    rows = {}
    with open(os.path.join(GOLDEN, "back_transformation_rows.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            i, expr = line.split(":", 1)
            rows[int(i)] = sympy.lambdify((ux, uy, uz, k5, k6, k7, k8, k9), sympy.sympify(expr), "numpy")
    assert sorted(rows) == list(range(19))
    return rows


def test_printed_back_transformation_matches_definition():
    rows = _printed_rows()
    rng = np.random.default_rng(3)
    N = 64
    u = 0.2 * rng.standard_normal((3, N))
    fm = rng.random((19, N))
    tau = 0.83
    bt = O.cm_collision_backtransform(fm, u, tau)
    T = O.transform_matrix(u)
    k = np.einsum("nmi,in->nm", T, fm) * (1.0 - 1.0 / tau)
    printed = np.array([rows[i](u[0], u[1], u[2], k[:, 5], k[:, 6], k[:, 7], k[:, 8], k[:, 9])
                        for i in range(19)])
    assert np.abs(printed - bt).max() < 1e-13


def _collide(fm, u, du, tau):
    rho = fm.sum(axis=0)
    return O.feq(rho, u + du) + O.cm_collision_backtransform(fm, u, tau)


def test_collision_invariants():
    rng = np.random.default_rng(5)
    N = 200
    rho = 0.5 + rng.random(N)
    u0 = 0.05 * rng.standard_normal((3, N))
    fm = O.feq(rho, u0) + 0.01 * rng.standard_normal((19, N))
    rho = fm.sum(axis=0)
    u = np.einsum("ia,in->an", C19.astype(float), fm) / rho
    du = 0.01 * rng.standard_normal((3, N))
    tau = 0.71
    post = _collide(fm, u, du, tau)
    # mass, and momentum rho (u + du) (exact-difference forcing adds rho du)
    assert np.abs(post.sum(axis=0) - rho).max() < 1e-14
    mom = np.einsum("ia,in->an", C19.astype(float), post)
    assert np.abs(mom - rho * (u + du)).max() < 1e-14
    # without force: shear central moments scaled by (1 - 1/tau), Eq. post_collision_moments
    post0 = _collide(fm, u, 0 * du, tau)
    T = O.transform_matrix(u)
    pre_cm = np.einsum("nmi,in->nm", T, fm)
    post_cm = np.einsum("nmi,in->nm", T, post0)
    assert np.abs(post_cm[:, 5:10] - (1 - 1 / tau) * pre_cm[:, 5:10]).max() < 1e-14
    # momentum conserved, central momentum zero
    assert np.abs(post_cm[:, 1:4]).max() < 1e-14
    # moments relaxed with rate 1 equal those of the equilibrium
    eq_cm = np.einsum("nmi,in->nm", T, O.feq(rho, u))
    relaxed = [0, 4] + list(range(10, 19))
    assert np.abs(post_cm[:, relaxed] - eq_cm[:, relaxed]).max() < 1e-13
    # second-order truncated equilibrium: central second moments rho c_s^2 delta
    assert np.abs(eq_cm[:, 4] - 3 * CS2 * rho).max() < 1e-14
    assert np.abs(eq_cm[:, 5:10]).max() < 1e-14


def test_bgk_limit_tau_one():
    """tau = 1 relaxes everything to equilibrium: f^m* = f^eq(rho, u + du)."""
    rng = np.random.default_rng(1)
    fm = O.feq(np.ones(10), 0.03 * rng.standard_normal((3, 10))) + 0.01 * rng.random((19, 10))
    rho = fm.sum(axis=0)
    u = np.einsum("ia,in->an", C19.astype(float), fm) / rho
    du = 1e-3 * np.ones((3, 10))
    assert np.abs(_collide(fm, u, du, 1.0) - O.feq(rho, u + du)).max() < 1e-15


def _random_state(shape, solid_frac, seed, params, noise=1e-3):
    rng = np.random.default_rng(seed)
    solid = rng.random(shape) < solid_frac
    g = O.Geometry(solid=solid, bc_z=params.bc_z)
    rr = rng.random(shape)
    rp = 1.0 - rr + 0.05 * rng.random(shape)
    st = O.init_state(g, params, rho_r=rr, rho_p=rp, conc=rng.random(shape),
                      u=0.02 * rng.standard_normal((3,) + shape))
    st.f += noise * rng.standard_normal(st.f.shape)
    st.f[:, g.solid] = 0.0
    return g, st


@pytest.mark.parametrize("mode", [0, 1])
def test_component_and_reaction_balance(mode):
    """Recolouring keeps rho^r and rho^p per node; the reaction moves exactly delta from r to p.

    Per node: sum(f^r*) = rho^r - delta, sum(f^p*) = rho^p + delta, f^m momentum
    = rho^m (u + du), and the reactant C loses delta (advection-diffusion mode).
    """
    p = O.Params(sigma=0.05, theta_deg=70, k_rate=0.2, accel=(1e-4, 0, 0), reaction_mode=mode, xi=0.3)
    g, st = _random_state((6, 7, 5), 0.25, 11, p)
    new, fl = O.step(st, g, p, return_fields=True)
    f = new.f
    fluid = g.fluid
    assert np.abs((f[0:19].sum(0) - (fl.rho_r - fl.delta))[fluid]).max() < 1e-14
    assert np.abs((f[19:38].sum(0) - (fl.rho_p + fl.delta))[fluid]).max() < 1e-14
    rho_m = fl.rho_r + fl.rho_p
    mom = np.einsum("ia,i...->a...", C19.astype(float), f[0:19] + f[19:38])
    assert np.abs((mom - rho_m * (fl.u + fl.du))[:, fluid]).max() < 1e-14
    if mode == 0:
        assert np.abs((f[38:45].sum(0) - (fl.conc - fl.delta))[fluid]).max() < 1e-14
        assert (fl.delta > 0).sum() > 0
    else:
        # paper mode: delta = min(xi NN r, 1) rho^r (Eq. reactive_boundary_condition_reactant, explicit Euler)
        ref = np.minimum(0.3 * g.nn * g.reactive, 1.0) * fl.rho_r
        assert np.abs((fl.delta - np.maximum(ref, 0))[fluid]).max() < 1e-15
