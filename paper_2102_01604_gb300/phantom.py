"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds no arithmetic of the fit itself (no signal equation, no
likelihood, no prior): it only draws the acquisition protocol, piecewise-smooth
ground-truth parameter maps, smooth B1 fields and noise.  Noise-free images
are made by whoever calls it (the oracle in the tests, the library's own
forward model in the bench) and passed back to :func:`rician`.

The recipe stands in for the paper's 0.8 mm MPM data (Sec. 3.2), which are
not available: PDw / T1w / MTw SPGR contrasts at 6 / 21 / 6 degrees, TR 25 ms,
8 / 8 / 6 echoes 2.3 ms apart, first-echo SNR 20, Rician magnitude noise.
"""
from __future__ import annotations

import math

import numpy as np

# Contrast presets: (nominal flip angle in degrees, TR in s, MT pulse).
CONTRASTS = {
    "PDw": (6.0, 0.025, 0),
    "T1w": (21.0, 0.025, 0),
    "MTw": (6.0, 0.025, 1),
    "VFA15": (15.0, 0.025, 0),
}

ECHO_SPACING = 0.0023  # s; TE_k = ECHO_SPACING * (k + 1)


def protocol(contrasts=("PDw", "T1w", "MTw"), n_echoes=(8, 8, 6), sigma2=None) -> dict:
    """Acquisition protocol as a plain dict: ``alpha`` (rad), ``tr`` (s),
    ``mt`` (0/1), ``n_echoes``, ``te`` (s, contrast-major, flat), ``sigma2``
    (noise variance per contrast; filled in by :func:`noise_sigma2`)."""
    assert len(contrasts) == len(n_echoes)
    alpha, tr, mt, te = [], [], [], []
    for name, ne in zip(contrasts, n_echoes):
        a, t, m = CONTRASTS[name]
        alpha.append(math.radians(a))
        tr.append(t)
        mt.append(m)
        te.extend(ECHO_SPACING * (k + 1) for k in range(ne))
    if sigma2 is None:
        sigma2 = [1.0] * len(contrasts)
    return {"names": list(contrasts), "alpha": alpha, "tr": tr, "mt": mt,
            "n_echoes": list(n_echoes), "te": te, "sigma2": list(sigma2)}


def _axes(shape):
    """Normalised coordinates along x, y, z (each in [0, 1))."""
    return [np.arange(n, dtype=np.float64) / n for n in shape]


def _separable(shape, fx, fy, fz):
    """Volume f(x) g(y) h(z) flattened with x fastest."""
    nx, ny, nz = shape
    return (fz[:, None, None] * fy[None, :, None] * fx[None, None, :]).reshape(-1)


def _smooth_field(rng, axes, shape):
    """Product of one low-frequency cosine per axis, scaled to [-1, 1]."""
    f = []
    for a in axes:
        freq = rng.integers(1, 3)
        phase = rng.uniform(0.0, 2.0 * math.pi)
        f.append(np.cos(math.pi * freq * a + phase))
    m = np.max(np.abs(f[0])) * np.max(np.abs(f[1])) * np.max(np.abs(f[2]))
    out = _separable(shape, *f)
    return out / m if m > 0 else out


def phantom(shape, seed: int = 0, n_regions: int = 12, n_contrasts: int = 3,
            with_b1m: bool = True, with_mt: bool = True) -> dict:
    """Piecewise-smooth ground truth on a grid ``(nx, ny, nz)`` (x fastest).

    Returns ``y`` [K][N] float64 log-parameters (log PD, log R1, log R2*,
    logit MTsat; K = 4 if ``with_mt`` else 3), ``b1p`` [N] in [0.8, 1.2] and
    ``b1m`` [C][N] in [0.9, 1.1] (or None).  Regions are the Voronoi cells of
    ``n_regions`` seeded centres with PD in [2000, 4000], R1 in [0.5, 1.5] /s,
    R2* in [10, 40] /s and MTsat in [0.002, 0.02], each modulated by a smooth
    factor ``1 + 0.05 prod_d cos(pi f_d x_d + phi_d)``.  The phantom fills the
    whole volume (no air background)."""
    rng = np.random.default_rng(seed)
    shape = tuple(int(v) for v in shape)
    axes = _axes(shape)
    N = int(np.prod(shape))
    centres = rng.uniform(0.0, 1.0, size=(n_regions, 3))
    best = np.full(N, np.inf)
    label = np.zeros(N, dtype=np.int64)
    for r in range(n_regions):
        d = (((axes[2] - centres[r, 2]) ** 2)[:, None, None]
             + ((axes[1] - centres[r, 1]) ** 2)[None, :, None]
             + ((axes[0] - centres[r, 0]) ** 2)[None, None, :]).reshape(-1)
        closer = d < best
        best[closer] = d[closer]
        label[closer] = r
    ranges = [(2000.0, 4000.0), (0.5, 1.5), (10.0, 40.0), (0.002, 0.02)]
    K = 4 if with_mt else 3
    y = np.empty((K, N))
    for k in range(K):
        lo, hi = ranges[k]
        vals = rng.uniform(lo, hi, size=n_regions)[label]
        vals *= 1.0 + 0.05 * _smooth_field(rng, axes, shape)
        y[k] = np.log(vals / (1.0 - vals)) if k == 3 else np.log(vals)
    b1p = 1.0 + 0.2 * _smooth_field(rng, axes, shape)
    b1m = None
    if with_b1m:
        b1m = np.stack([1.0 + 0.1 * _smooth_field(rng, axes, shape) for _ in range(n_contrasts)])
    return {"y": y, "b1p": b1p, "b1m": b1m, "label": label}


def noise_sigma2(s: np.ndarray, prot: dict, snr: float = 20.0) -> list:
    """Per-contrast noise variance: sigma_c = mean over voxels of the first-echo
    noise-free image of contrast c, divided by ``snr``."""
    out, i = [], 0
    for ne in prot["n_echoes"]:
        sig = float(np.mean(s[i])) / snr
        out.append(sig * sig)
        i += ne
    return out


def normals(shape, seed: int):
    """Two seeded standard-normal arrays (real and imaginary noise)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape), rng.standard_normal(shape)


def rician(s: np.ndarray, prot: dict, seed: int) -> np.ndarray:
    """Rician magnitude data |s + sigma_c (n1 + i n2)| per image (numpy, float64)."""
    n1, n2 = normals(s.shape, seed)
    sig = np.empty(s.shape[0])
    i = 0
    for c, ne in enumerate(prot["n_echoes"]):
        sig[i:i + ne] = math.sqrt(prot["sigma2"][c])
        i += ne
    sig = sig[:, None]
    return np.sqrt((s + sig * n1) ** 2 + (sig * n2) ** 2)


def rician_torch(s, prot: dict, seed: int):
    """Same noise model on a torch tensor (any device), seeded torch generator.
    Used where the volume is too large to draw noise on the host quickly."""
    import torch
    gen = torch.Generator(device=s.device)
    gen.manual_seed(seed)
    out = torch.empty_like(s)
    i = 0
    for c, ne in enumerate(prot["n_echoes"]):
        sig = math.sqrt(prot["sigma2"][c])
        for e in range(ne):
            n1 = torch.randn(s.shape[1:], generator=gen, device=s.device, dtype=s.dtype)
            n2 = torch.randn(s.shape[1:], generator=gen, device=s.device, dtype=s.dtype)
            out[i] = torch.sqrt((s[i] + sig * n1) ** 2 + (sig * n2) ** 2)
            i += 1
    return out


def single_voxel_protocols(n: int, seed: int, n_echoes: int = 5):
    """The convergence experiment's sampler (Sec. 3.1): per voxel, three
    contrasts (the last with an MT pulse) with five echoes each; log A, log R1,
    log R2*, logit MTsat, log TR and log TE uniform in [-5, 5]; flip angles
    uniform in [0, pi/4]; noise variance 1.  Yields (protocol, truth y[4])."""
    rng = np.random.default_rng(seed)
    for _ in range(n):
        y = rng.uniform(-5.0, 5.0, size=4)
        alpha = rng.uniform(0.0, math.pi / 4, size=3)
        tr = np.exp(rng.uniform(-5.0, 5.0, size=3))
        te = np.exp(rng.uniform(-5.0, 5.0, size=3 * n_echoes))
        prot = {"names": ["c0", "c1", "c2"], "alpha": list(alpha), "tr": list(tr),
                "mt": [0, 0, 1], "n_echoes": [n_echoes] * 3, "te": list(te),
                "sigma2": [1.0, 1.0, 1.0]}
        yield prot, y
