"""The seeded synthetic inputs against their recipe: the MPM protocol of the
paper's data (Sec. 3.2: PDw / T1w / MTw at 6 / 21 / 6 degrees, TR 25 ms,
8 / 8 / 6 echoes 2.3 ms apart), piecewise-smooth maps in the stated ranges,
smooth B1 fields, first-echo SNR 20, and Rician magnitude noise, which at zero
signal is the Rayleigh distribution."""
import math

import numpy as np
import pytest

from paper_2102_01604_gb300 import phantom


def test_protocol_is_the_mpm_protocol():
    p = phantom.protocol()
    assert p["names"] == ["PDw", "T1w", "MTw"]
    assert np.allclose(np.degrees(p["alpha"]), [6.0, 21.0, 6.0])
    assert p["tr"] == [0.025] * 3
    assert p["mt"] == [0, 0, 1]
    assert p["n_echoes"] == [8, 8, 6]
    te = np.array(p["te"])
    assert len(te) == 22
    expect = np.concatenate([0.0023 * np.arange(1, n + 1) for n in (8, 8, 6)])
    assert np.allclose(te, expect)


def test_phantom_regions_ranges_and_fields():
    shape = (40, 36, 24)
    ph = phantom.phantom(shape, seed=3)
    y, lab = ph["y"], ph["label"]
    assert y.shape == (4, int(np.prod(shape)))
    assert len(np.unique(lab)) == 12                      # 12 Voronoi regions
    pd, r1, r2 = np.exp(y[0]), np.exp(y[1]), np.exp(y[2])
    mt = 1.0 / (1.0 + np.exp(-y[3]))
    for v, (lo, hi) in zip((pd, r1, r2, mt), [(2000, 4000), (0.5, 1.5), (10, 40), (0.002, 0.02)]):
        # region value in [lo, hi] times a smooth factor in [0.95, 1.05]
        assert v.min() >= lo * 0.95 - 1e-9 and v.max() <= hi * 1.05 + 1e-9
        # within a region the map varies only by the smooth factor
        for r in range(12):
            m = v[lab == r]
            assert m.max() / m.min() <= 1.05 / 0.95 + 1e-9
    assert 0.8 - 1e-12 <= ph["b1p"].min() and ph["b1p"].max() <= 1.2 + 1e-12
    assert abs(np.abs(ph["b1p"] - 1.0).max() - 0.2) < 0.05   # the field spans its range
    assert ph["b1m"].shape == (3, y.shape[1])
    assert 0.9 - 1e-12 <= ph["b1m"].min() and ph["b1m"].max() <= 1.1 + 1e-12


def test_phantom_is_seeded():
    a = phantom.phantom((12, 10, 6), seed=5)
    b = phantom.phantom((12, 10, 6), seed=5)
    c = phantom.phantom((12, 10, 6), seed=6)
    assert np.array_equal(a["y"], b["y"]) and np.array_equal(a["b1p"], b["b1p"])
    assert not np.array_equal(a["y"], c["y"])


def test_noise_sigma_is_first_echo_mean_over_snr():
    prot = phantom.protocol()
    rng = np.random.default_rng(0)
    s = rng.uniform(100.0, 300.0, size=(22, 1000))
    sig2 = phantom.noise_sigma2(s, prot, snr=20.0)
    for c, i0 in enumerate((0, 8, 16)):
        assert math.isclose(math.sqrt(sig2[c]), s[i0].mean() / 20.0, rel_tol=1e-12)


@pytest.mark.parametrize("use_torch", [False, True])
def test_rician_noise_at_zero_signal_is_rayleigh(use_torch):
    """|0 + sigma (n1 + i n2)| is Rayleigh(sigma): mean sigma sqrt(pi/2), second
    moment 2 sigma^2."""
    prot = {"n_echoes": [1, 1], "sigma2": [4.0, 0.25]}
    n = 400_000
    s = np.zeros((2, n))
    if use_torch:
        import torch
        x = phantom.rician_torch(torch.zeros((2, n), dtype=torch.float64), prot, seed=11).numpy()
    else:
        x = phantom.rician(s, prot, seed=11)
    for c, sigma in enumerate((2.0, 0.5)):
        assert abs(x[c].mean() / (sigma * math.sqrt(math.pi / 2)) - 1.0) < 5e-3
        assert abs((x[c] ** 2).mean() / (2 * sigma * sigma) - 1.0) < 1e-2


def test_rician_noise_at_high_snr_is_nearly_gaussian():
    """Far above the noise, |s + sigma n| is s + sigma n1 to first order, so the
    mean is s + sigma^2 / (2 s) and the spread sigma."""
    prot = {"n_echoes": [1], "sigma2": [1.0]}
    s = np.full((1, 400_000), 50.0)
    x = phantom.rician(s, prot, seed=2)[0]
    assert abs(x.mean() - (50.0 + 1.0 / 100.0)) < 5e-3
    assert abs(x.std() - 1.0) < 5e-3
