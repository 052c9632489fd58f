"""Entry points around the step: asynchronous per-step reads, changing the inlet
and the wettability of an existing context (each must equal a fresh context)."""
import dataclasses

import numpy as np
import pytest
import torch

from paper_2608_15781_b300 import build, lbm, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbm.load_library()


def _column():
    shape = (24, 20, 18)
    solid = synth.grf_mask(shape, 3, 0.5, 21, periodic_z=False)
    p = lbm.Params(theta_deg=50.0, u_in=0.006, k_rate=5e-3, c_in=1.0)
    return solid, p


def test_reaction_async_matches_synchronous_read():
    solid, p = _column()
    ring = torch.zeros(2 * 30, dtype=torch.float64, pin_memory=True)
    sync = []
    with lbm.Lattice(solid, p, bc_z=1) as L:
        with pytest.raises(lbm.LbmError):
            L.reaction_async(ring.data_ptr())          # before the first step
        for k in range(30):
            L.step(1)
            L.reaction_async(ring.data_ptr() + 16 * k)
            if k % 7 == 0:
                sync.append((k, L.reaction()))
        L.observables()
    r = ring.numpy().reshape(-1, 2)
    for k, (rate, consumed) in sync:
        assert r[k, 0] == rate and r[k, 1] == consumed
    assert np.all(np.diff(r[:, 1]) >= 0) and r[-1, 1] > 0


@pytest.mark.parametrize("storage", [0, 1])
def test_set_inlet_and_wetting_equal_a_fresh_context(storage):
    """Also with FP16 storage: its rounding bits restart with the step counter, so a
    re-initialised context rounds exactly as a fresh one."""
    solid, p = _column()
    p = dataclasses.replace(p, storage=storage)
    rng = np.random.default_rng(1)
    theta = rng.uniform(30, 110, solid.shape).astype(np.float32)
    q = dataclasses.replace(p, u_in=0.009, c_in=0.6)
    with lbm.Lattice(solid, q, bc_z=1, theta=theta) as ref:
        ref.step(25)
        want = ref.get_state()
    with lbm.Lattice(solid, p, bc_z=1) as L:
        L.step(5)
        L.set_wetting(theta)
        L.set_inlet(q.u_in, q.c_in)
        L.init_fields(np.ones(solid.shape, np.float32), np.zeros(solid.shape, np.float32),
                      np.full(solid.shape, q.c_init, np.float32))
        L.step(25)
        got = L.get_state()
    assert np.array_equal(got, want)
