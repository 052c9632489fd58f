"""Batches of independent lattices: every kernel of a step is one launch over
all of them (and a step is replayed as one CUDA graph).  Each lattice of a batch
must evolve exactly as it does alone, and one batched step must match the
oracle's step for every lattice."""
import numpy as np
import pytest

from oracle import cglbm as O
from paper_2608_15781_b300 import build, lbm, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbm.load_library()


def _cases():
    shapes = [(20, 16, 24), (16, 20, 20), (24, 12, 16), (10, 10, 12)]
    bcs = [1, 0, 1, 0]
    params = [
        lbm.Params(theta_deg=40.0, u_in=0.004, k_rate=5e-3, sigma=0.02),
        lbm.Params(theta_deg=100.0, k_rate=2e-3, accel=(2e-5, 0, 0)),
        lbm.Params(theta_deg=70.0, u_in=0.008, reaction_mode=1, xi=0.5),
        lbm.Params(theta_deg=20.0, k_rate=1e-2, sigma=0.05),
    ]
    solids = [synth.grf_mask(s, 3, 0.45 + 0.05 * k, 30 + k, periodic_z=(bcs[k] == 0)) for k, s in enumerate(shapes)]
    return solids, params, bcs


def _oparams(p, bc):
    return O.Params(tau=p.tau, sigma=p.sigma, beta=p.beta, theta_deg=p.theta_deg, accel=tuple(p.accel),
                    diffusivity=p.diffusivity, k_rate=p.k_rate, c_init=p.c_init, c_in=p.c_in, u_in=p.u_in,
                    rho_out=p.rho_out, xi=p.xi, reaction_mode=p.reaction_mode, bc_z=bc)


def test_batch_matches_single_lattices():
    solids, params, bcs = _cases()
    with lbm.Batch(solids, params, bc_z=bcs) as B:
        B.step(30)
        states = [B.get_state(k) for k in range(len(solids))]
        obs = B.observables()
    for k, (s, p, bc) in enumerate(zip(solids, params, bcs)):
        with lbm.Lattice(s, p, bc_z=bc) as L:
            L.step(30)
            ref = L.get_state()
            ob = L.observables()
        assert np.abs(states[k] - ref).max() <= 1e-6, k
        for key in ("mass_r", "mass_p", "mass_c", "consumed", "gas_saturation", "flux_in", "flux_out"):
            assert abs(obs[k][key] - ob[key]) <= 1e-9 * max(1.0, abs(ob[key])), (k, key)
        assert obs[k]["step"] == 30 and obs[k]["n_fluid"] == ob["n_fluid"]


def test_batch_step_matches_oracle_for_every_lattice():
    solids, params, bcs = _cases()
    with lbm.Batch(solids, params, bc_z=bcs) as B:
        B.step(12)
        pre = [B.get_state(k) for k in range(len(solids))]
        B.step(1)
        post = [B.get_state(k) for k in range(len(solids))]
    for k, (s, p, bc) in enumerate(zip(solids, params, bcs)):
        g = O.Geometry(solid=s, bc_z=bc)
        ref = O.step(O.State(f=pre[k].astype(np.float64)), g, _oparams(p, bc)).f
        err = np.abs(post[k].astype(np.float64) - ref)[:, g.fluid].max()
        assert err < 5e-7, (k, err)


def test_tune_keeps_state_and_picks_candidates():
    solids, params, bcs = _cases()
    with lbm.Batch(solids, params, bc_z=bcs) as A, lbm.Batch(solids, params, bc_z=bcs) as B:
        A.step(5)
        B.step(5)
        blocks = B.tune()
        assert blocks["main"] in (64, 128, 256) and blocks["density"] in (128, 256, 512)
        A.step(10)
        B.step(10)
        for k in range(len(solids)):
            assert np.abs(A.get_state(k) - B.get_state(k)).max() <= 1e-6


def test_set_state_of_one_lattice_keeps_the_others():
    solids, params, bcs = _cases()
    with lbm.Batch(solids, params, bc_z=bcs) as B:
        B.step(7)   # odd: the current state sits in the second buffer
        keep = [B.get_state(k) for k in range(len(solids))]
        f = keep[1].copy()
        B.set_state(1, f)
        for k in range(len(solids)):
            assert np.abs(B.get_state(k) - keep[k]).max() == 0.0, k
