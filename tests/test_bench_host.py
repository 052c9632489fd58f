"""Host-side logic of bench.py (no GPU): the byte models behind the roofline, the
rule that reports ncu traffic only for unchanged kernel sources, the reader of the
FP64 crop reference and the velocity difference of two states."""
import importlib.util
import os
from types import SimpleNamespace

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_host_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_byte_models(bench):
    """45 (38 in paper mode) populations read and written per fluid node, 4 B (FP32) or
    2 B (FP16) each, plus one byte of flags; the density pass re-reads the 19 f^r / f^p
    pairs and writes one float."""
    p = lambda mode, storage: SimpleNamespace(reaction_mode=mode, storage=storage)
    assert bench.bytes_per_fluid_node(p(0, 0)) == 2 * 45 * 4 + 1 == 361
    assert bench.bytes_per_fluid_node(p(1, 0)) == 2 * 38 * 4 + 1 == 305
    assert bench.bytes_per_fluid_node(p(0, 1)) == 181
    assert bench.bytes_per_fluid_node(p(1, 1)) == 153
    assert bench.density_pass_bytes_per_fluid_node(p(0, 0)) == 19 * 2 * 4 + 4 == 156
    assert bench.density_pass_bytes_per_fluid_node(p(0, 1)) == 80


def test_traffic_reported_only_for_unchanged_kernels(bench, tmp_path, monkeypatch):
    f = tmp_path / "traffic.txt"
    f.write_text("# comment = ignored\nkernel_sources_sha256_16 = %s\ndram_bytes_per_fluid_node = 406.2\n"
                 % bench.kernel_source_hash())
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.ncu_traffic_per_fluid_node() == pytest.approx(406.2)
    f.write_text("kernel_sources_sha256_16 = 0000000000000000\ndram_bytes_per_fluid_node = 406.2\n")
    assert bench.ncu_traffic_per_fluid_node() is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.txt"))
    assert bench.ncu_traffic_per_fluid_node() is None


def test_committed_traffic_record_is_well_formed(bench):
    """The committed record carries a 16-hex-digit source hash and a per-node figure
    above the 361 B algorithmic model (the slot map and the curvature's normals add
    reads; a figure below it would mean a wrong capture)."""
    kv = {}
    for line in open(bench.TRAFFIC_FILE):
        if "=" in line and not line.startswith("#"):
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    assert len(kv["kernel_sources_sha256_16"]) == 16
    int(kv["kernel_sources_sha256_16"], 16)
    assert 361.0 < float(kv["dram_bytes_per_fluid_node"]) < 2 * 361.0


def test_precision_crop_reference_reader(bench):
    obs, vel = bench.read_precision_crop()
    assert [r[0] for r in obs] == list(range(500, 5001, 500))
    assert all(len(r) == 6 for r in obs) and all(len(r) == 6 for r in vel)
    assert len(vel) == 4096
    for step, conv, sat, mr, mp, mc in obs:
        assert 0.0 < conv < 1.0 and 0.0 < sat < 1.0
        # periodic crop with the reaction turning red mass into product: the total
        # stays the fluid node count, and the red mass tracks the reactant's
        assert mr + mp == pytest.approx(132009.0, rel=1e-10)
        assert mr == pytest.approx(mc, rel=1e-10)
    z, y, x = (np.array([r[k] for r in vel]) for k in range(3))
    assert z.min() >= 0 and max(z.max(), y.max(), x.max()) < 64


def test_velocity_difference(bench):
    """u = sum_i c_i (f^r_i + f^p_i) / rho at fluid nodes; solid nodes are ignored."""
    rng = np.random.default_rng(4)
    shape = (3, 4, 5)
    solid = np.zeros(shape, np.uint8)
    solid[0, 0, 0] = 1
    w = np.array([1 / 18] * 6 + [1 / 36] * 12 + [1 / 3])
    fa = np.zeros((45,) + shape, np.float32)
    fa[0:19] = w[:, None, None, None] * (1 + 0.01 * rng.standard_normal((19,) + shape))
    fb = fa.copy()
    fb[19:38] += 1e-3 * rng.standard_normal((19,) + shape).astype(np.float32)
    fb[:, 0, 0, 0] = 1e3                     # a solid node's values do not count
    d, umax = bench.velocity_difference(fa, fb, solid, chunk=2)

    def u(f):
        m = f[0:19].astype(np.float64) + f[19:38]
        return np.einsum("ia,i...->a...", bench._C19.astype(np.float64), m) / m.sum(0)

    fl = solid == 0
    assert d == pytest.approx(np.abs(u(fa) - u(fb))[:, fl].max(), rel=1e-6)
    assert umax == pytest.approx(np.abs(u(fb))[:, fl].max(), rel=1e-6)
