"""Seeded input generators: SplitMix64 against its published outputs, phantom recipe."""
import numpy as np

from paper_1708_01663_gb300 import synth


def test_splitmix64_published_outputs():
    # First outputs of SplitMix64 from state 0 and from seed 1234567
    # (the generator's reference implementation, Steele et al. 2014).
    assert [int(v) for v in synth.splitmix64(0, 0, 3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert int(synth.splitmix64(1234567, 0, 1)[0]) == 6457827717110365317


def test_uniform_and_normal_moments():
    r = synth.Rng(7)
    u = r.uniform(count=200000)
    assert 0.0 <= u.min() and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5e-3
    z = synth.Rng(8).normal(200000)
    assert abs(z.mean()) < 1e-2 and abs(z.std() - 1.0) < 1e-2


def test_phantom_recipe():
    cfg = synth.CONFIGS["c2"]
    f = synth.ellipse_phantom(cfg["n"], cfg["shapes"], cfg["contrast"], cfg["seed"], cfg["imag"])
    assert f.shape == (256, 256)
    assert f.real.max() <= 1.0 and f.real.min() >= 0.0
    nz = np.abs(f) > 0
    assert np.allclose(f.imag[nz], 0.05)
    # deterministic
    g = synth.ellipse_phantom(cfg["n"], cfg["shapes"], cfg["contrast"], cfg["seed"], cfg["imag"])
    assert np.array_equal(f, g)


def test_noise_unit_variance():
    e = synth.complex_noise(3, (64, 256))
    assert abs(np.mean(np.abs(e) ** 2) - 1.0) < 0.02
