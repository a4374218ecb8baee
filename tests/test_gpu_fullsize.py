"""Parity at the benchmark's full size (176 x 240 x 256, the launch
configuration bench.py times) and at a size whose stencil launches march
several z planes per block.

The oracle cannot run the whole fit at full size in seconds, so each call is
checked on its own: the voxel pass on sampled voxels (it is voxel-wise), the
JTV weights and energy over the whole volume, and the PCG solve over the
whole volume for a few iterations, all from inputs the oracle computed.
"""
import numpy as np
import pytest

import oracle as orc
from cases import assert_close_scaled, dataset, map_error, to_dev, to_np

pytestmark = pytest.mark.gpu

FULL = (176, 240, 256)


@pytest.fixture(scope="module")
def mpm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2102_01604_gb300 as m
    m._lib.load()
    return m


@pytest.fixture(scope="module")
def full():
    return dataset(FULL, seed=0)


def _sample_problem(d, idx):
    """The voxels `idx` as a 1-D volume (the voxel pass does not couple voxels)."""
    sub = {"prot": d["prot"], "shape": (len(idx), 1, 1)}
    x = np.ascontiguousarray(d["x"][:, idx])
    b1p = np.ascontiguousarray(d["b1p"][idx])
    b1m = np.ascontiguousarray(d["b1m"][:, idx])
    return sub, x, b1p, b1m


def test_grad_hess_full_size_sampled(mpm, full):
    d = full
    N = int(np.prod(FULL))
    rng = np.random.default_rng(1)
    y = (d["y_true"] + 0.05 * rng.standard_normal(d["y_true"].shape)).astype(np.float32)
    pg = mpm.make_problem(d["prot"], FULL)
    g, h, nll = mpm.mpm_grad_hess(pg, to_dev(d["x"]), to_dev(y), to_dev(d["b1p"]),
                                  to_dev(d["b1m"]))
    idx = np.unique(np.concatenate([rng.integers(0, N, 4000), [0, N - 1, 175, 176 * 240]]))
    sub, xs, bps, bms = _sample_problem(d, idx)
    po = orc.make_problem(d["prot"], sub["shape"])
    _, g_o, h_o = orc.grad_hess(po, xs, np.ascontiguousarray(y[:, idx]), bps, bms)
    assert_close_scaled(to_np(g)[:, idx], g_o, 1e-4, "g")
    assert_close_scaled(to_np(h)[:, idx], h_o, 1e-4, "h")
    # likelihood over the whole volume from the oracle's forward model
    s = orc.forward(orc.make_problem(d["prot"], FULL), y, d["b1p"], d["b1m"])
    ref, i = 0.0, 0
    for c, ne in enumerate(d["prot"]["n_echoes"]):
        ref += np.sum((d["x"][i:i + ne].astype(np.float64) - s[i:i + ne]) ** 2) / (2 * d["prot"]["sigma2"][c])
        i += ne
    assert abs(nll.item() - ref) <= 2e-6 * ref


def test_jtv_full_size(mpm, full):
    d = full
    rng = np.random.default_rng(2)
    y = (d["y_true"] + 0.02 * rng.standard_normal(d["y_true"].shape)).astype(np.float32)
    pg = mpm.make_problem(d["prot"], FULL)
    w, jtv = mpm.mpm_jtv_weights(pg, to_dev(y))
    e_o, w_o = orc.jtv(orc.make_problem(d["prot"], FULL), y)
    np.testing.assert_allclose(to_np(w), w_o, rtol=1e-5)
    assert abs(jtv.item() - e_o) <= 2e-6 * e_o


@pytest.mark.parametrize("shape,cg_iters", [(FULL, 4), ((176, 240, 24), 30)])
def test_solve_full_volume(mpm, full, shape, cg_iters):
    """Whole-volume PCG parity; the 176x240x24 case gives stencil blocks that
    march two z planes each."""
    if shape == FULL:
        d = full
    else:
        d = dataset(shape, seed=3)
    po = orc.make_problem(d["prot"], shape)
    rng = np.random.default_rng(4)
    y = (d["y_true"] + 0.05 * rng.standard_normal(d["y_true"].shape)).astype(np.float32)
    _, g, h = orc.grad_hess(po, d["x"], y, d["b1p"], d["b1m"])
    _, w = orc.jtv(po, y)
    h, w, g = h.astype(np.float32), w.astype(np.float32), g.astype(np.float32)
    pg = mpm.make_problem(d["prot"], shape)
    opts = mpm.make_opts(cg_iters=cg_iters)
    delta, resid = mpm.mpm_solve(pg, opts, to_dev(h), to_dev(w), to_dev(g), to_dev(y))
    d_o, it, r_o = orc.solve(po, h, w, g, y, cg_iters)
    assert it == cg_iters
    assert_close_scaled(to_np(delta), d_o, 2e-4, "delta")
    np.testing.assert_allclose(to_np(resid), r_o, rtol=1e-3, atol=1e-6 * r_o[0])


def test_fit_multi_plane_blocks(mpm):
    """Whole fit where stencil blocks march several z planes (176x240x24)."""
    import torch
    shape = (176, 240, 24)
    d = dataset(shape, seed=5)
    pg = mpm.make_problem(d["prot"], shape)
    po = orc.make_problem(d["prot"], shape)
    K, N = pg.n_maps, int(np.prod(shape))
    y = torch.zeros((K, N), dtype=torch.float32, device="cuda")
    st, rep = mpm.mpm_fit(pg, mpm.make_opts(gn_iters=3, cg_iters=30), to_dev(d["x"]), y,
                          to_dev(d["b1p"]), to_dev(d["b1m"]))
    ref = orc.fit(po, d["x"], None, d["b1p"], d["b1m"], gn_iters=3, cg_iters=30)
    assert rep.iters == 3
    np.testing.assert_allclose(np.array(rep.F[:4]), ref["F"], rtol=1e-5)
    assert map_error(to_np(y), ref["y"]).max() <= 1e-3
