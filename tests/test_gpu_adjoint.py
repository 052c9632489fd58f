"""GPU reverse mode (hand-written adjoint kernels, through the C ABI) against the
FP64 autograd reference of the oracle, plus finite differences on the GPU.

* dJ/df_0 after one step, element by element: every reverse kernel (collision,
  curvature, solid normals, wetting, gradient, solid colour, streaming, outlet
  ghost) contributes to it.
* dJ/dtheta (per solid node) and dJ/du_in over a checkpointed multi-step run on
  a 24^3 crop of a column, against the FP64 reference.
* checkpoint spacing does not change the gradient; the autograd Function
  returns the same numbers.
* central differences of the GPU forward along random directions.

Tolerances: the reference differentiates the FP64 forward; the GPU adjoint runs
in FP32 around FP32 forward states, so errors are relative to the largest
gradient entry (the stencil transposes use FP32 atomics).
"""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import adjoint as A
from oracle import cglbm as O
from paper_2608_15781_b300 import adjoint as ADJ
from paper_2608_15781_b300 import build, lbm, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbm.load_library()


def _oparams(p):
    return O.Params(tau=p.tau, sigma=p.sigma, beta=p.beta, theta_deg=p.theta_deg, accel=tuple(p.accel),
                    diffusivity=p.diffusivity, k_rate=p.k_rate, c_init=p.c_init, c_in=p.c_in, u_in=p.u_in,
                    rho_out=p.rho_out, xi=p.xi, reaction_mode=p.reaction_mode, bc_z=1)


def _case(shape, seed, grf=False):
    """Column with gas pockets on the walls, random contact-angle field, inflow start."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    if grf:
        solid = synth.grf_mask(shape, max(2, nx // 8), 0.5, seed, periodic_z=False)
    else:
        solid = rng.random(shape) < 0.15
        solid[:, 0, :] = True
    solid[0] = False
    solid[-1] = False
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    gas = np.zeros(shape, bool)
    for c in rng.integers(0, [nz, ny, nx], size=(3, 3)):
        gas |= ((xx - c[2]) ** 2 + (yy - c[1]) ** 2 + (zz - c[0]) ** 2) < (min(shape) / 5) ** 2
    gas &= ~solid
    p = lbm.Params(sigma=0.02, theta_deg=60.0, k_rate=0.02, diffusivity=0.05, u_in=0.01, c_in=1.0,
                   c_init=0.5, rho_out=1.0)
    theta = rng.uniform(30.0, 120.0, shape)
    op = _oparams(p)
    g = O.Geometry(solid=solid, bc_z=1, theta_deg=theta.astype(np.float32).astype(np.float64))
    u = np.zeros((3,) + shape)
    u[2] = p.u_in
    st = O.init_state(g, op, rho_r=np.where(gas, 0.05, 1.0), rho_p=np.where(gas, 0.95, 0.02),
                      conc=np.full(shape, 0.5), u=u)
    st.f += 1e-4 * rng.standard_normal(st.f.shape)
    st.f[:, solid] = 0.0
    f0 = st.f.astype(np.float32)
    return solid, p, op, g, theta.astype(np.float32), f0


def _reference(g, op, f0, theta, nsteps, want_state=False):
    ts = A.TorchStep(g, op)
    th = torch.tensor(theta.astype(np.float64), requires_grad=True)
    u_in = torch.tensor(op.u_in, dtype=torch.float64, requires_grad=True)
    f = torch.tensor(f0.astype(np.float64), requires_grad=want_state)
    x = f
    tw = ts.wall_theta(th)
    for _ in range(nsteps):
        x = ts.step(x, tw, u_in)
    J = ts.conversion(x)
    J.backward()
    return float(J.detach()), th.grad.numpy(), float(u_in.grad), (f.grad.numpy() if want_state else None)


def test_state_gradient_one_step():
    shape = (12, 10, 11)
    solid, p, op, g, theta, f0 = _case(shape, 1)
    with lbm.Lattice(solid, p, bc_z=1, theta=theta) as L:
        L.set_state(f0)
        J = L.adjoint_forward(1, 1)
        dth, du, ds = L.adjoint_backward(want_state=True)
    Jr, dthr, dur, dsr = _reference(g, op, f0, theta, 1, want_state=True)
    assert abs(J - Jr) < 1e-5 * max(1.0, abs(Jr))
    fl = g.fluid
    scale = np.abs(dsr[:, fl]).max()
    err = np.abs(ds.astype(np.float64) - dsr)[:, fl]
    assert err.max() < 2e-4 * scale, (err.max(), scale, np.unravel_index(err.argmax(), err.shape))
    sc = np.abs(dthr).max()
    assert sc > 0
    assert np.abs(dth - dthr).max() < 2e-4 * sc, (np.abs(dth - dthr).max(), sc)
    assert abs(du - dur) < 2e-4 * abs(dur), (du, dur)
    assert np.all(dth[fl] == 0.0)


@pytest.mark.parametrize("shape", [(2, 7, 9), (3, 8, 6), (4, 5, 7)])
def test_thin_columns_three_steps(shape):
    """Columns two to four planes deep (the least a column takes), where every node sits
    next to a ghost plane and populations leave at both ends: three steps with
    checkpoints every two, dJ/df_0, dJ/dtheta and dJ/du_in against the FP64 autograd
    reference (2e-4 of the largest entry)."""
    solid, p, op, g, theta, f0 = _case(shape, 11 + shape[0])
    with lbm.Lattice(solid, p, bc_z=1, theta=theta) as L:
        L.set_state(f0)
        J = L.adjoint_forward(3, 2)
        dth, du, ds = L.adjoint_backward(want_state=True)
    Jr, dthr, dur, dsr = _reference(g, op, f0, theta, 3, want_state=True)
    assert abs(J - Jr) < 1e-5 * max(1.0, abs(Jr))
    fl = g.fluid
    scale = np.abs(dsr[:, fl]).max()
    err = np.abs(ds.astype(np.float64) - dsr)[:, fl]
    assert err.max() < 2e-4 * scale, (err.max(), scale)
    sc = np.abs(dthr).max()
    if sc > 0:
        assert np.abs(dth - dthr).max() < 2e-4 * sc, (np.abs(dth - dthr).max(), sc)
    assert abs(du - dur) < 2e-4 * abs(dur), (du, dur)


def _reference_along(g, op, states, theta, nsteps):
    """FP64 adjoint linearised along a given trajectory (the GPU's own FP32 states)."""
    ts = A.TorchStep(g, op)
    th = torch.tensor(theta.astype(np.float64), requires_grad=True)
    u = torch.tensor(op.u_in, dtype=torch.float64, requires_grad=True)
    fT = torch.tensor(states[nsteps].astype(np.float64), requires_grad=True)
    ts.conversion(fT).backward()
    lam = fT.grad.clone()
    for t in range(nsteps - 1, -1, -1):
        x = torch.tensor(states[t].astype(np.float64), requires_grad=True)
        ts.step(x, ts.wall_theta(th), u).backward(lam)
        lam = x.grad.clone()
    return th.grad.numpy(), float(u.grad)


def _rel_stats(a, r):
    sc = np.abs(r).max()
    e = np.abs(a - r)
    nz = r != 0
    return sc, e.max() / sc, np.percentile(e[nz], 99) / sc, np.median(e[nz]) / sc


def test_crop24_multi_step_against_fp64_reference():
    """24^3 crop, 24 steps, checkpoints every 5 steps.

    Along the GPU's own trajectory the FP64 adjoint and the FP32 kernels agree to
    rounding.  Against the FP64 trajectory a few nodes differ by up to ~1e-2 of
    the largest entry: the FP32 and FP64 forwards part at nodes where the
    interface threshold |grad rho^N| = 1e-5 is crossed, and the gradient there is
    large (n = grad/|grad|); the bulk agrees to ~1e-6.
    """
    shape = (24, 24, 24)
    nsteps = 24
    solid, p, op, g, theta, f0 = _case(shape, 5, grf=True)
    with lbm.Lattice(solid, p, bc_z=1, theta=theta) as L:
        L.set_state(f0)
        states = [L.get_state()]
        for _ in range(nsteps):
            L.step(1)
            states.append(L.get_state())
        L.set_state(f0)
        J = L.adjoint_forward(nsteps, 5)
        dth, du, _ = L.adjoint_backward()
    dta, dua = _reference_along(g, op, states, theta, nsteps)
    sc, emax, e99, emed = _rel_stats(dth, dta)
    assert emax < 1e-4 and e99 < 1e-5, (emax, e99, emed)
    assert abs(du - dua) < 1e-5 * abs(dua), (du, dua)
    Jr, dthr, dur, _ = _reference(g, op, f0, theta, nsteps)
    assert abs(J - Jr) < 1e-4 * max(1.0, abs(Jr))
    sc, emax, e99, emed = _rel_stats(dth, dthr)
    assert emed < 1e-5 and e99 < 5e-3 and emax < 0.1, (emax, e99, emed)
    assert abs(du - dur) < 1e-3 * abs(dur), (du, dur)


def test_directional_derivatives_against_fp64_central_differences():
    """16 random directions in the contact-angle field and the inlet velocity (24^3 GRF
    column with smooth gas pockets, 12 steps): the GPU adjoint against FP64 central
    differences of the NumPy oracle, Richardson-extrapolated from steps h and h/2 (error
    O(h^4); |D(h) - D(h/2)| stays small, so no threshold or branch of the discrete map is
    crossed inside +-h), and against the FP64 adjoint linearised along the GPU's own FP32
    trajectory (reported).

    Bounds: the 16 derivatives as one vector within 1e-3 in the relative 2-norm
    (measured 2.0e-4), median 5e-4, every direction 2e-3 (15 of 16 within 1e-3, the
    worst 1.08e-3), u_in 1e-5.  The directional derivatives
    of this discrete map are sensitive to rounding-level changes of the state: a random
    1e-7 perturbation of the start moves the FP64 central differences themselves by
    2e-4 - 5e-3 per direction (interfaces whose normal n = grad / |grad| rounds
    differently), so an adjoint of the FP32 forward, which is rounded at that level every
    step, cannot agree with the FP64 differences much more closely in every direction.
    The inlet velocity, a smooth parameter, agrees to ~3e-7."""
    shape = (24, 24, 24)
    nsteps = 12
    solid, rr, rp = _clean_case(shape, 7)
    p = lbm.Params(sigma=0.02, theta_deg=60.0, k_rate=0.02, diffusivity=0.05, u_in=0.01, c_in=1.0)
    op = _oparams(p)
    rng = np.random.default_rng(4)
    theta = rng.uniform(30.0, 120.0, shape).astype(np.float32)
    g = O.Geometry(solid=solid, bc_z=1, theta_deg=theta.astype(np.float64))
    with lbm.Lattice(solid, p, bc_z=1, theta=theta) as L:
        u = np.zeros((3,) + shape, np.float32)
        u[2] = p.u_in
        L.init_fields(rr, rp, np.ones(shape, np.float32), u)
        f0 = L.get_state()
        states = [f0]
        for _ in range(nsteps):
            L.step(1)
            states.append(L.get_state())
        L.set_state(f0)
        L.adjoint_forward(nsteps)
        dth, du, _ = L.adjoint_backward()
    dth_along, du_along = _reference_along(g, op, states, theta, nsteps)
    th64 = theta.astype(np.float64)

    def central(fun, h):
        return (fun(h) - fun(-h)) / (2 * h)

    def richardson(fun, h):
        d1, d2 = central(fun, h), central(fun, h / 2)
        return (4 * d2 - d1) / 3, abs(d1 - d2)

    rel, rel_own, rel_traj, spread, pairs = [], [], [], [], []
    for _ in range(16):
        v = rng.standard_normal(shape) * solid
        fd, sp = richardson(lambda e: A.conversion_forward(g, op, f0, th64 + e * v, nsteps), 1e-2)
        gpu, along = float((dth * v).sum()), float((dth_along * v).sum())
        pairs.append((gpu, fd))
        rel.append(abs(gpu - fd) / abs(fd))
        rel_own.append(abs(gpu - along) / abs(along))
        rel_traj.append(abs(along - fd) / abs(fd))
        spread.append(sp / abs(fd))
    fdu, spu = richardson(lambda e: A.conversion_forward(g, dataclasses.replace(op, u_in=op.u_in + e), f0, th64,
                                                         nsteps), 1e-5)
    rel, rel_own, rel_traj, spread = (np.array(x) for x in (rel, rel_own, rel_traj, spread))
    fmt = lambda x: np.array2string(x, precision=2)
    print("\nGPU adjoint vs FP64 differences:", fmt(rel), "\nGPU adjoint vs FP64 adjoint along the GPU trajectory:",
          fmt(rel_own), "\nFP64 adjoint along the GPU trajectory vs FP64 differences:", fmt(rel_traj),
          "\n|D(h) - D(h/2)|:", fmt(spread), "\nu_in:", abs(du - fdu) / abs(fdu), abs(du - du_along) / abs(du_along))
    # the 16 directional derivatives as one vector (the gradient's projection on the
    # random directions): its relative error in the 2-norm
    gv, fv = np.array(pairs).T
    agg = np.linalg.norm(gv - fv) / np.linalg.norm(fv)
    print("projected gradient, relative 2-norm error:", agg)
    assert spread.max() < 1e-3, spread
    assert agg < 1e-3, agg
    assert np.median(rel) < 5e-4 and rel.max() < 2e-3, rel
    assert abs(du - fdu) < 1e-5 * abs(fdu), (du, fdu)


def test_checkpoint_spacing_and_autograd_function():
    shape = (16, 14, 12)
    solid, p, op, g, theta, f0 = _case(shape, 9)
    grads = []
    with lbm.Lattice(solid, p, bc_z=1, theta=theta) as L:
        for every in (1, 4, 0, 12):
            L.set_state(f0)
            L.adjoint_forward(12, every)
            dth, du, _ = L.adjoint_backward()
            grads.append((dth, du))
        th = torch.tensor(theta.astype(np.float64), requires_grad=True)
        u = torch.tensor(p.u_in, dtype=torch.float64, requires_grad=True)
        J = ADJ.conversion(th, u, L, f0, 12, 4)
        (2.0 * J).backward()
    ref = grads[0]
    for dth, du in grads[1:]:
        assert np.abs(dth - ref[0]).max() <= 1e-5 * np.abs(ref[0]).max()
        assert abs(du - ref[1]) <= 1e-5 * abs(ref[1])
    assert np.abs(th.grad.numpy() - 2.0 * ref[0]).max() <= 1e-5 * np.abs(ref[0]).max()
    assert abs(float(u.grad) - 2.0 * ref[1]) <= 1e-5 * abs(ref[1])


def _clean_case(shape, seed):
    """GRF column, liquid with smooth (tanh) gas pockets and no noise: the bulk has
    no colour gradient, as in a physical run."""
    nz, ny, nx = shape
    solid = synth.grf_mask(shape, max(2, nx // 8), 0.5, seed, periodic_z=False)
    solid[0] = False
    solid[-1] = False
    rng = np.random.default_rng(seed)
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    phi = np.ones(shape)
    for c in rng.integers(0, [nz, ny, nx], size=(4, 3)):
        r = np.sqrt((xx - c[2]) ** 2 + (yy - c[1]) ** 2 + (zz - c[0]) ** 2)
        phi = np.minimum(phi, np.tanh((r - min(shape) / 6) / 2.0))
    return solid, (0.5 * (1 + phi)).astype(np.float32), (0.5 * (1 - phi)).astype(np.float32)


def test_central_differences_of_the_gpu_forward():
    """Central differences of the FP32 GPU forward itself (10 steps, 16 directions).

    The FP32 forward's rounding is re-randomised by any perturbation, so below
    about 1 degree the differences are noise-limited and above it the response is
    nonlinear; at h = 1 degree they agree with the adjoint to about 1e-2 (median).
    The inlet velocity is smoother and agrees to 1e-3.
    """
    shape = (40, 32, 32)
    nsteps = 10
    solid, rr, rp = _clean_case(shape, 13)
    p = lbm.Params(sigma=0.01, theta_deg=60.0, k_rate=2e-3, diffusivity=0.05, u_in=0.004, c_in=1.0)
    rng = np.random.default_rng(3)
    theta = rng.uniform(40.0, 100.0, shape).astype(np.float32)
    with lbm.Lattice(solid, p, bc_z=1, theta=theta) as L:
        u = np.zeros((3,) + shape, np.float32)
        u[2] = p.u_in
        L.init_fields(rr, rp, np.ones(shape, np.float32), u)
        f0 = L.get_state()
        L.adjoint_forward(nsteps)
        dth, du, _ = L.adjoint_backward()

        def J_of(th, uin):
            L.set_wetting(th)
            L.set_inlet(uin, p.c_in)
            L.set_state(f0)
            return L.adjoint_forward(nsteps, nsteps)

        h = 1.0
        rel = []
        for _ in range(16):
            v = (rng.standard_normal(shape) * solid).astype(np.float32)
            fd = (J_of(theta + h * v, p.u_in) - J_of(theta - h * v, p.u_in)) / (2 * h)
            rel.append(abs(fd - float((dth * v).sum())) / abs(fd))
        hu = 1e-4
        fdu = (J_of(theta, p.u_in + hu) - J_of(theta, p.u_in - hu)) / (2 * hu)
    rel = np.array(rel)
    assert np.median(rel) < 3e-2, rel
    assert abs(fdu - du) < 2e-3 * abs(du), (fdu, du)
