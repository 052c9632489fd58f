"""The allocation-free entry point lbm_step_static against the regular path.

lbm_step_static serves callers that must not allocate device memory (an arena
or pool owns every allocation, or the stream is being recorded): it keeps its
intermediate fields in a fixed scratch array inside the library.  Here the
caller's buffers come from PyTorch; two calls in a row (ping-pong between two
buffers) must reproduce two steps of the regular context-based path.  This
file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2608_15781_b300 import build, lbm

pytestmark = pytest.mark.gpu


def test_static_step_matches_context_path_two_calls():
    import torch

    build.build()
    lbm.load_library()
    torch.cuda.init()
    shape = (16, 20, 24)
    rng = np.random.default_rng(21)
    solid = rng.random(shape) < 0.3
    p = lbm.Params(sigma=0.05, theta_deg=50.0, accel=(1e-4, 0.0, -2e-5), k_rate=0.05)
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
    dev = torch.device("cuda:0")
    solid_d = torch.from_numpy(solid.astype(np.uint8)).to(dev)
    bufs = [torch.from_numpy(f0.reshape(-1)).to(dev), torch.empty(45 * n, dtype=torch.float32, device=dev)]
    dsum = torch.zeros(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    for k in range(2):
        src, dst = bufs[k % 2], bufs[(k + 1) % 2]
        lbm.lbm_step_static(shape, solid_d.data_ptr(), src.data_ptr(), dst.data_ptr(), p,
                            delta_sum_dev=dsum.data_ptr(), stream=stream)
        torch.cuda.synchronize()
        out = dst.cpu().numpy().reshape((45,) + shape)
        fluid = ~solid
        err = np.abs(out.astype(np.float64) - refs[k].astype(np.float64))[:, fluid].max()
        assert err < 5e-7, (k, err)
        assert abs(float(dsum.item()) - rates[k]) < 1e-9 * max(1.0, rates[k]), (k, dsum.item(), rates[k])


def test_static_step_rejects_oversize():
    build.build()
    lib = lbm.load_library()
    p = lbm.Params().to_c()
    big = 64
    assert big ** 3 > lbm.STATIC_MAX_NODES
    rc = lib.lbm_step_static(big, big, big, 1, None, 1, 2, None, p)
    assert rc == lbm.LBM_EINVAL
