"""Input generators: SplitMix64 reference outputs, GRF mask porosity and connectivity."""
import numpy as np
from scipy import ndimage

from paper_2608_15781_b300 import synth


def test_splitmix64_reference_values():
    # published reference outputs of SplitMix64 for seeds 0 and 1234567
    assert [int(v) for v in synth.splitmix64(0, 2)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4]
    assert int(synth.splitmix64(1234567, 1)[0]) == 6457827717110365317


def test_gaussian_noise_moments():
    z = synth.gaussian_noise(5, (64, 64, 16))
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01


def test_grf_mask_porosity_and_bicontinuity():
    m = synth.grf_mask((32, 32, 32), 4, 0.55, 1)
    assert abs((1 - m.mean()) - 0.55) < 0.02
    for phase in (~m, m):
        lab, n = ndimage.label(phase)
        assert n >= 1
    # deterministic for a given seed
    assert (synth.grf_mask((32, 32, 32), 4, 0.55, 1) == m).all()
    assert not (synth.grf_mask((32, 32, 32), 4, 0.55, 2) == m).all()
