"""Launch configurations of the step: every choice lbm_tune can make (block
sizes, programmatic dependent launch or plain launches, the colour at solids,
normals and normals at solids as three kernels or as one tiled kernel) gives
the same populations bit for bit, for one lattice and for a batch, FP32 and
FP16 storage, on boxes whose sizes are not multiples of the field tile; bad
configurations are rejected; the tuner keeps the state."""
import dataclasses

import numpy as np
import pytest

from paper_2608_15781_b300 import build, lbm, synth

pytestmark = pytest.mark.gpu

DEFAULT = dict(main=128, density=256, normal=256, pdl=1, fields=0)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbm.load_library()


def _case(bc, storage):
    shape = (26, 22, 19)
    solid = synth.grf_mask(shape, 3, 0.5, 31 + bc, periodic_z=(bc == 0))
    p = lbm.Params(sigma=0.02, theta_deg=55.0, k_rate=0.01, storage=storage)
    if bc == 1:
        p = dataclasses.replace(p, u_in=0.008, c_in=1.0)
    else:
        p = dataclasses.replace(p, accel=(1e-5, 0.0, 0.0))
    rr, rp = synth.droplet_fields(shape, (9, 11, 13), 5.0, inside_r=False)
    return solid, p, rr, rp


def _run(solid, p, bc, rr, rp, launch, nsteps=15):
    with lbm.Lattice(solid, p, bc_z=bc) as L:
        L.set_launch(launch)
        L.init_fields(rr, rp, np.ones(solid.shape, np.float32))
        L.step(nsteps)
        return L.get_state(), L.observables()


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("storage", [0, 1])
def test_launch_choices_are_bit_identical(bc, storage):
    solid, p, rr, rp = _case(bc, storage)
    f0, ob0 = _run(solid, p, bc, rr, rp, DEFAULT)
    assert ob0["n_bad"] == 0
    for launch in (dict(DEFAULT, pdl=0), dict(DEFAULT, fields=2), dict(main=64, density=128, normal=512, pdl=1, fields=1),
                   dict(main=256, density=512, normal=128, pdl=0, fields=3)):
        f1, ob1 = _run(solid, p, bc, rr, rp, launch)
        assert np.array_equal(f0, f1), launch
        assert ob1["mass_r"] == ob0["mass_r"] and ob1["gas_saturation"] == ob0["gas_saturation"]


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("shape", [(26, 22, 19), (9, 17, 40), (3, 5, 2)])
def test_fused_fields_equal_three_kernels(bc, shape):
    """rho^N (fluid and boundary solids) and the normals (fluid and boundary solids) of one step."""
    solid = synth.grf_mask(shape, 2, 0.5, 7 + bc, periodic_z=(bc == 0))
    p = lbm.Params(sigma=0.02, theta_deg=55.0, k_rate=0.01, u_in=0.008 * bc)
    rng = np.random.default_rng(5)
    rr = rng.random(shape).astype(np.float32)
    out = []
    for fields in (0, 1, 2, 3):
        with lbm.Lattice(solid, p, bc_z=bc) as L:
            L.set_launch(dict(DEFAULT, fields=fields))
            L.init_fields(rr, 1.0 - rr, np.ones(shape, np.float32))
            L.step(3)
            out.append((L.field(lbm.FIELD_RHON), L.field(lbm.FIELD_NORMAL), L.field(lbm.FIELD_GRADMAG),
                        L.get_state()))
    for other in out[1:]:
        for a, b in zip(out[0], other):
            assert np.array_equal(a, b)


def test_batch_launch_shapes():
    masks = [synth.grf_mask((14, 12, 16), 2, 0.5, s, periodic_z=False) for s in (3, 4, 5)]
    ps = [lbm.Params(theta_deg=t, u_in=0.005, c_in=1.0, k_rate=0.01) for t in (40.0, 80.0, 110.0)]
    states = []
    for launch in (DEFAULT, dict(main=64, density=512, normal=128, pdl=0, fields=2), dict(DEFAULT, fields=1),
                   dict(DEFAULT, fields=3)):
        with lbm.Batch(masks, ps, bc_z=[1, 1, 1]) as B:
            B.set_launch(launch)
            B.step(7)
            states.append([B.get_state(k) for k in range(3)])
    for other in states[1:]:
        for a, b in zip(states[0], other):
            assert np.array_equal(a, b)


def test_set_launch_rejects_and_tune_reports():
    solid, p, rr, rp = _case(0, 0)
    with lbm.Lattice(solid, p) as L:
        for bad in (dict(DEFAULT, main=96), dict(DEFAULT, density=64), dict(DEFAULT, normal=1024),
                    dict(DEFAULT, pdl=2), dict(DEFAULT, fields=4)):
            with pytest.raises(lbm.LbmError):
                L.set_launch(bad)
        L.step(2)
        st = L.get_state()
        chosen = L.tune()
        assert np.array_equal(L.get_state(), st)
        assert chosen["main"] in (64, 128, 256) and chosen["normal"] in (128, 256, 512) and chosen["pdl"] in (0, 1)
        assert chosen["fields"] in (0, 1, 2, 3)
        L.set_launch(chosen)
        L.step(2)
        L.observables()
