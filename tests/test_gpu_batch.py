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
        for key in ("mass_r", "mass_p", "mass_c", "consumed", "rate", "gas_saturation", "flux_in", "flux_out"):
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


def test_lattices_of_a_few_nodes():
    """Lattices so small that lattice creation cannot stage its inputs (mask, layout
    counts) in the colour and normal fields and takes buffers of its own: a 3x3x3
    periodic box alone, and a batch of six 2x2x2 boxes and a 3x2x2 column.  One step
    after 6 against the oracle; every lattice of the batch as it evolves alone."""
    rng = np.random.default_rng(9)
    shapes = [(2, 2, 2)] * 6 + [(3, 2, 2)]
    bcs = [0] * 6 + [1]
    solids = []
    for s in shapes:
        m = np.zeros(s, bool)
        m.flat[rng.integers(0, m.size)] = True   # one solid node, the rest fluid
        solids.append(m)
    params = [lbm.Params(theta_deg=50.0 + 10 * k, k_rate=5e-3, sigma=0.02, u_in=0.004) for k in range(len(shapes))]
    box = np.zeros((3, 3, 3), bool)
    box[1, 1, 1] = True
    cases = [([box], [lbm.Params(theta_deg=60.0, k_rate=5e-3, accel=(1e-5, 0, 0))], [0]), (solids, params, bcs)]
    for sol, prm, bc in cases:
        with lbm.Batch(sol, prm, bc_z=bc) as B:
            B.step(6)
            pre = [B.get_state(k) for k in range(len(sol))]
            B.step(1)
            post = [B.get_state(k) for k in range(len(sol))]
        for k, (s, p, b) in enumerate(zip(sol, prm, bc)):
            g = O.Geometry(solid=s, bc_z=b)
            ref = O.step(O.State(f=pre[k].astype(np.float64)), g, _oparams(p, b)).f
            err = np.abs(post[k].astype(np.float64) - ref)[:, g.fluid].max()
            assert err < 5e-7, (k, err)
            with lbm.Lattice(s, p, bc_z=b) as L:
                L.step(7)
                assert np.abs(L.get_state() - post[k]).max() <= 1e-6, k


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


def test_full_batch_workload_sampled_nodes():
    """The bench's batch of 64 columns (edges 48-96, 26 M nodes) in its launch
    configuration: after 10 steps, one more step checked node by node against the
    per-node oracle on the downloaded pre-step state of every eighth lattice (wall
    nodes, bulk, inlet and outlet planes; 5e-7)."""
    from oracle.pointwise import PointwiseStep
    from paper_2608_15781_b300.configs import batched_workload

    masks, params, bcs, edges = batched_workload()
    rng = np.random.default_rng(5)
    with lbm.Batch(masks, params, bc_z=bcs) as B:
        B.set_launch(dict(main=128, density=128, normal=128, pdl=1, fields=0))
        B.step(10)
        ks = list(range(0, len(masks), 8))
        pre = {k: B.get_state(k) for k in ks}
        B.step(1)
        post = {k: B.get_state(k) for k in ks}
    worst = 0.0
    for k in ks:
        solid = masks[k]
        pw = PointwiseStep(pre[k], solid, _oparams(params[k], bcs[k]))
        fluid = ~solid
        wall = np.zeros(solid.shape, bool)
        for c in O.C19[:18]:
            wall |= O.neighbor(solid, c, "clamp")
        zs = np.argwhere(fluid)
        groups = [np.argwhere(fluid & wall), np.argwhere(fluid & ~wall), zs[zs[:, 0] == 0],
                  zs[zs[:, 0] == solid.shape[0] - 1]]
        for grp in groups:
            for i in rng.choice(len(grp), size=min(4, len(grp)), replace=False):
                z, y, x = (int(v) for v in grp[i])
                ref, _ = pw.update((x, y, z))
                worst = max(worst, float(np.abs(post[k][:, z, y, x].astype(np.float64) - ref).max()))
    assert worst < 5e-7, worst
