"""The allocation-free entry point lbm_step_static.

lbm_step_static serves callers that must not allocate device memory (an arena
or pool owns every allocation, or the stream is being recorded): it keeps its
intermediate fields in a fixed scratch array inside the library.  Here the
caller's buffers come from PyTorch, the second one left uninitialised; two calls
in a row (ping-pong between the two buffers) must reproduce two steps of the
FP64 oracle and of the regular context-based path, over the whole output array
(solid entries zero; in the paper's reaction mode the reactant block copied).
This file is collected last on purpose.
"""
import numpy as np
import pytest

from oracle import cglbm as O
from paper_2608_15781_b300 import build, lbm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", [0, 1])
def test_static_step_matches_oracle_and_context_path_two_calls(mode):
    import torch

    build.build()
    lbm.load_library()
    torch.cuda.init()
    shape = (16, 20, 24)
    rng = np.random.default_rng(21 + mode)
    solid = rng.random(shape) < 0.3
    p = lbm.Params(sigma=0.05, theta_deg=50.0, accel=(1e-4, 0.0, -2e-5), k_rate=0.05, xi=0.3, reaction_mode=mode)
    n = int(np.prod(shape))
    assert n <= lbm.STATIC_MAX_NODES
    with lbm.Lattice(solid, p) as L:
        rr = rng.random(shape).astype(np.float32)
        L.init_fields(rr, 1.02 - rr, rng.random(shape).astype(np.float32),
                      (0.02 * rng.standard_normal((3,) + shape)).astype(np.float32))
        f0 = L.get_state()
        refs, rates = [], []
        for _ in range(2):
            L.step(1)
            refs.append(L.get_state())
            rates.append(L.reaction()[0])
    g = O.Geometry(solid=solid, bc_z=0)
    op = O.Params(sigma=p.sigma, theta_deg=p.theta_deg, accel=p.accel, k_rate=p.k_rate, xi=p.xi,
                  reaction_mode=mode)
    dev = torch.device("cuda:0")
    solid_d = torch.from_numpy(solid.astype(np.uint8)).to(dev)
    bufs = [torch.from_numpy(f0.reshape(-1)).to(dev), torch.empty(45 * n, dtype=torch.float32, device=dev)]
    bufs[1].fill_(float("nan"))      # anything the call leaves unwritten shows
    dsum = torch.zeros(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    fluid = ~solid
    for k in range(2):
        src, dst = bufs[k % 2], bufs[(k + 1) % 2]
        inp = src.cpu().numpy().reshape((45,) + shape)
        lbm.lbm_step_static(shape, solid_d.data_ptr(), src.data_ptr(), dst.data_ptr(), p,
                            delta_sum_dev=dsum.data_ptr(), stream=stream)
        torch.cuda.synchronize()
        out = dst.cpu().numpy().reshape((45,) + shape).astype(np.float64)
        assert np.isfinite(out).all(), k
        assert (out[:, solid] == 0.0).all(), k
        # one FP64 oracle step from the same FP32 input
        ora = O.step(O.State(f=inp.astype(np.float64)), g, op)
        err = np.abs(out - ora.f)[:, fluid].max()
        assert err < 5e-7, (k, err)
        assert abs(float(dsum.item()) - ora.rate) < 1e-5 * max(1.0, ora.rate), (k, dsum.item(), ora.rate)
        if mode == 1:
            assert (out[38:45] == inp[38:45].astype(np.float64)).all(), k
        # the context-based path (same arithmetic on another layout; from the second call on
        # the inputs differ by the first call's FP32 rounding, so the sums agree to FP32 level)
        err_ctx = np.abs(out - refs[k].astype(np.float64))[:, fluid].max()
        assert err_ctx < 5e-7, (k, err_ctx)
        assert abs(float(dsum.item()) - rates[k]) < 1e-6 * max(1.0, rates[k]), (k, dsum.item(), rates[k])


def test_static_step_rejects_oversize():
    build.build()
    lib = lbm.load_library()
    p = lbm.Params().to_c()
    big = 64
    assert big ** 3 > lbm.STATIC_MAX_NODES
    rc = lib.lbm_step_static(big, big, big, 1, None, 1, 2, None, p)
    assert rc == lbm.LBM_EINVAL
