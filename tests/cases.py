"""Seeded test inputs shared by the GPU parity tests.

Every input comes from the seeded phantom generator and the FP64 oracle
(noise-free images), rounded once to float32 (or bfloat16) so that the CUDA
library and the oracle see exactly the same numbers.  Nothing here is computed
by the CUDA path.
"""
from __future__ import annotations

import numpy as np

import oracle as orc
from paper_2102_01604_gb300 import phantom


def f32(a):
    return None if a is None else np.asarray(a, dtype=np.float32)


def round_protocol(prot: dict) -> dict:
    """Protocol with every number rounded to float32 (the library computes in
    float32), so both sides use identical constants."""
    out = dict(prot)
    for k in ("alpha", "tr", "te", "sigma2"):
        out[k] = [float(np.float32(v)) for v in prot[k]]
    return out


def dataset(shape, seed=0, contrasts=("PDw", "T1w", "MTw"), n_echoes=(8, 8, 6), b1p=True,
            b1m=True, snr=20.0, noise=True):
    """Phantom maps, B1 fields and Rician images (float32) on ``shape``."""
    prot = phantom.protocol(contrasts, n_echoes)
    with_mt = any(prot["mt"])
    ph = phantom.phantom(shape, seed=seed, n_contrasts=len(contrasts), with_b1m=b1m,
                         with_mt=with_mt)
    prot = round_protocol(prot)
    bp = f32(ph["b1p"]) if b1p else None
    bm = f32(ph["b1m"]) if b1m else None
    p0 = orc.make_problem(prot, shape)
    s = orc.forward(p0, ph["y"], bp, bm)
    prot["sigma2"] = [float(np.float32(v)) for v in phantom.noise_sigma2(s, prot, snr)]
    prot = round_protocol(prot)
    x = phantom.rician(s, prot, seed=seed + 1) if noise else s
    return {"prot": prot, "shape": tuple(shape), "y_true": ph["y"], "b1p": bp, "b1m": bm,
            "x": f32(x), "s": s}


def to_dev(a, device="cuda"):
    import torch
    if a is None:
        return None
    return torch.from_numpy(np.ascontiguousarray(a)).to(device)


def to_np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def assert_close_scaled(got, ref, rtol, what=""):
    """|got - ref| <= rtol (|ref| + rms of the row): element-wise relative
    error with a floor at the row's typical magnitude, per row (map, image or
    Hessian entry)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    ref2 = ref.reshape(ref.shape[0], -1) if ref.ndim > 1 else ref[None]
    got2 = got.reshape(ref2.shape)
    for i in range(ref2.shape[0]):
        floor = np.sqrt(np.mean(ref2[i] ** 2)) if ref2[i].size else 0.0
        err = np.abs(got2[i] - ref2[i])
        bound = rtol * (np.abs(ref2[i]) + floor)
        bad = err > bound
        assert not bad.any(), (f"{what} row {i}: {bad.sum()} of {bad.size} elements out of "
                               f"tolerance; worst err {err.max():.3e} "
                               f"at ref {ref2[i][np.argmax(err)]:.4e}, floor {floor:.3e}")


def map_error(y_got, y_ref):
    """Per-voxel error in log space relative to max(1, |y|)."""
    return np.abs(y_got - y_ref) / np.maximum(1.0, np.abs(y_ref))


# ------------------------------------------------------------ spatial projection

def sub_protocol(prot, c):
    """The protocol of contrast c alone."""
    i0 = sum(prot["n_echoes"][:c])
    out = {k: (v[c:c + 1] if isinstance(v, list) else v) for k, v in prot.items()}
    out["te"] = list(prot["te"][i0:i0 + prot["n_echoes"][c]])
    return out


def moved_dataset(shape, grids, affines, seed=0, contrasts=("PDw", "T1w", "MTw"),
                  n_echoes=(6, 6, 5), snr=20.0):
    """Phantom maps on the reconstruction grid ``shape``; contrast c acquired
    on ``grids[c]`` with ``affines[c]`` (acquisition voxel -> reconstruction
    voxel coordinates).  The images of each contrast are the oracle's forward
    model of the pulled (interpolated) maps, with Rician noise at first-echo
    SNR ``snr``, rounded to float32; B1 fields are drawn on each acquisition
    grid."""
    prot = phantom.protocol(contrasts, n_echoes)
    with_mt = any(prot["mt"])
    ph = phantom.phantom(shape, seed=seed, n_contrasts=len(contrasts), with_mt=with_mt)
    prot = round_protocol(prot)
    K = 4 if with_mt else 3
    p0 = orc.make_problem(prot, shape)
    s_list, bps, bms = [], [], []
    for c in range(len(contrasts)):
        yc, _ = orc.pull(p0, grids[c], affines[c], ph["y"])
        fc = phantom.phantom(grids[c], seed=seed + 101 + c, n_contrasts=1, with_mt=with_mt)
        bp, bm = f32(fc["b1p"]), f32(fc["b1m"][0])
        sub = orc.make_problem(sub_protocol(prot, c), grids[c], n_maps=K)
        s_list.append(orc.forward(sub, yc, bp, bm[None]))
        bps.append(bp)
        bms.append(bm)
    sig2 = []
    for c, s in enumerate(s_list):
        m = float(np.mean(s[0])) / snr
        sig2.append(float(np.float32(m * m)))
    prot["sigma2"] = sig2
    prot = round_protocol(prot)
    xs = []
    for c, s in enumerate(s_list):
        sp = sub_protocol(prot, c)
        xs.append(f32(phantom.rician(s, sp, seed=seed + 7 + c)))
    return {"prot": prot, "shape": tuple(shape), "y_true": ph["y"], "xs": xs, "b1ps": bps,
            "b1ms": bms, "grids": [tuple(g) for g in grids],
            "affines": [np.asarray(a, dtype=np.float64) for a in affines]}


# ------------------------------------------------------------ full-size fits

FULLSIZE = {
    # config: (shape, voxel size in mm)
    "1mm": ((176, 240, 256), (1.0, 1.0, 1.0)),
    "0.8mm": ((208, 300, 320), (0.8, 0.8, 0.8)),
}
FULLSIZE_FIT = {"gn_iters": 20, "cg_iters": 30, "lam": 10.0, "eps": 1e-3, "seed": 0}


def bf16_round(x32):
    """float32 -> nearest bfloat16 (ties to even), returned as float32: the
    values a bfloat16 copy of the images holds."""
    u = np.ascontiguousarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def fullsize_case(config="1mm", echo="f32"):
    """The headline workload's inputs at full size: the bench protocol and
    phantom statistics, seeded host noise (so the oracle sees the same data),
    float32 images (rounded once more to bfloat16 values with echo="bf16")."""
    shape, vx = FULLSIZE[config]
    d = dataset(shape, seed=FULLSIZE_FIT["seed"])
    d.pop("s")
    if echo == "bf16":
        d["x"] = bf16_round(d["x"])
    d["vx"] = vx
    return d


def sample_voxels(shape, n_inner=8192, n_face=4096, seed=12345):
    """Seeded voxel indices for sampled comparisons: uniform over the volume,
    plus voxels on its six faces (where the prior's boundary rule acts)."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    inner = rng.choice(nx * ny * nz, size=n_inner, replace=False)
    c = np.stack([rng.integers(0, n, size=n_face) for n in shape])
    axis = rng.integers(0, 3, size=n_face)
    side = rng.integers(0, 2, size=n_face)
    for a in range(3):
        sel = axis == a
        c[a, sel] = side[sel] * (shape[a] - 1)
    face = c[0] + nx * (c[1] + ny * c[2])
    return np.unique(np.concatenate([inner, face]))


def block_means(v, shape, b=16):
    """Means of each map over b x b x b blocks (partial blocks at the far
    edges): a whole-volume summary of [K][N] maps."""
    nx, ny, nz = shape
    K = v.shape[0]
    a = np.asarray(v, dtype=np.float64).reshape(K, nz, ny, nx)
    out = []
    for z0 in range(0, nz, b):
        for y0 in range(0, ny, b):
            for x0 in range(0, nx, b):
                out.append(a[:, z0:z0 + b, y0:y0 + b, x0:x0 + b].reshape(K, -1).mean(axis=1))
    return np.stack(out, axis=1)
