"""Edge cases through the C ABI on the GPU: empty and one-voxel volumes,
degenerate grids, error paths, numeric failure reporting, determinism and
resume."""
import ctypes

import numpy as np
import pytest

import oracle as orc
from cases import dataset, map_error, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mpm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2102_01604_gb300 as m
    m._lib.load()
    return m


def test_empty_volume(mpm):
    import torch
    d = dataset((3, 3, 1), seed=1)
    p = mpm.make_problem(d["prot"], (0, 5, 5))
    y = torch.zeros((4, 1), device="cuda")
    x = torch.zeros((22, 1), device="cuda")
    st, rep = mpm.mpm_fit(p, mpm.make_opts(), x, y)
    assert st == 0 and rep.iters == 0
    g, h, nll = mpm.mpm_grad_hess(p, x, y, ws=torch.zeros(1 << 20, dtype=torch.uint8, device="cuda"))
    assert nll.item() == 0.0


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 5), (2, 1, 1), (1, 7, 1), (31, 1, 9)])
def test_degenerate_grids(mpm, shape):
    import torch
    d = dataset(shape, seed=2)
    pg = mpm.make_problem(d["prot"], shape)
    po = orc.make_problem(d["prot"], shape)
    K, N = 4, int(np.prod(shape))
    y = torch.zeros((K, N), device="cuda")
    st, rep = mpm.mpm_fit(pg, mpm.make_opts(gn_iters=4), to_dev(d["x"]), y, to_dev(d["b1p"]),
                          to_dev(d["b1m"]))
    ref = orc.fit(po, d["x"], None, d["b1p"], d["b1m"], gn_iters=4, cg_iters=30)
    assert rep.iters == ref["iters"]
    np.testing.assert_allclose(np.array(rep.F[:rep.iters + 1]), ref["F"], rtol=1e-5)
    assert map_error(to_np(y), ref["y"]).max() <= 1e-3


def test_invalid_arguments(mpm):
    import torch
    lib = mpm._lib.load()
    d = dataset((8, 8, 4), seed=3)
    p = mpm.make_problem(d["prot"], (8, 8, 4))
    o = mpm.make_opts()
    x = to_dev(d["x"])
    y = torch.zeros((4, 256), device="cuda")
    ws = mpm.workspace(p, o)
    rep = mpm.Report()
    # workspace too small
    st = lib.mpm_fit(ctypes.byref(p), ctypes.byref(o), ctypes.c_void_p(x.data_ptr()), None, None,
                     ctypes.c_void_p(y.data_ptr()), None, ctypes.c_void_p(ws.data_ptr()),
                     ws.numel() - 1024, ctypes.byref(rep), None)
    assert st == mpm._lib.ERR_WORKSPACE_TOO_SMALL
    # host pointer for the images
    xh = d["x"]
    st = lib.mpm_fit(ctypes.byref(p), ctypes.byref(o), ctypes.c_void_p(xh.ctypes.data), None, None,
                     ctypes.c_void_p(y.data_ptr()), None, ctypes.c_void_p(ws.data_ptr()),
                     ws.numel(), ctypes.byref(rep), None)
    assert st == mpm._lib.ERR_INVALID_ARG
    # misaligned map pointer
    st = lib.mpm_fit(ctypes.byref(p), ctypes.byref(o), ctypes.c_void_p(x.data_ptr()), None, None,
                     ctypes.c_void_p(y.data_ptr() + 2), None, ctypes.c_void_p(ws.data_ptr()),
                     ws.numel(), ctypes.byref(rep), None)
    assert st == mpm._lib.ERR_INVALID_ARG
    # the device is still healthy
    st, rep = mpm.mpm_fit(p, mpm.make_opts(gn_iters=1), x, y, ws=ws)
    assert st == 0


def test_nan_input_reported(mpm):
    import torch
    d = dataset((8, 8, 4), seed=4)
    x = d["x"].copy()
    x[3, 17] = np.nan
    p = mpm.make_problem(d["prot"], (8, 8, 4))
    y = torch.zeros((4, 256), device="cuda")
    with pytest.raises(mpm.MPMError) as e:
        mpm.mpm_fit(p, mpm.make_opts(gn_iters=2), to_dev(x), y)
    assert e.value.status == mpm._lib.ERR_NUMERIC


def test_deterministic(mpm):
    import torch
    d = dataset((40, 24, 10), seed=5)
    p = mpm.make_problem(d["prot"], (40, 24, 10))
    outs = []
    for _ in range(2):
        y = torch.zeros((4, 40 * 24 * 10), device="cuda")
        st, rep = mpm.mpm_fit(p, mpm.make_opts(gn_iters=3), to_dev(d["x"]), y, to_dev(d["b1p"]),
                              to_dev(d["b1m"]))
        outs.append((to_np(y), np.array(rep.F[:4])))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])


def test_resume(mpm):
    """6 updates equal 3 updates then 3 more from their result (state is y)."""
    import torch
    d = dataset((20, 12, 6), seed=6)
    p = mpm.make_problem(d["prot"], (20, 12, 6))
    N = 20 * 12 * 6
    a = torch.zeros((4, N), device="cuda")
    mpm.mpm_fit(p, mpm.make_opts(gn_iters=6), to_dev(d["x"]), a, to_dev(d["b1p"]), to_dev(d["b1m"]))
    b = torch.zeros((4, N), device="cuda")
    mpm.mpm_fit(p, mpm.make_opts(gn_iters=3), to_dev(d["x"]), b, to_dev(d["b1p"]), to_dev(d["b1m"]))
    mpm.mpm_fit(p, mpm.make_opts(gn_iters=3, init=False), to_dev(d["x"]), b, to_dev(d["b1p"]),
                to_dev(d["b1m"]))
    assert torch.equal(a, b)


@pytest.mark.parametrize("echoes,b1m", [((15, 4), True), ((16, 4), False), ((20, 3), True)])
def test_voxel_pass_at_the_staging_limit(mpm, echoes, b1m):
    """The staged voxel pass takes a contrast's B1- and echoes as one group
    of at most 16 rows; 16 rows (15 echoes with B1-, 16 without) stage, 21 do
    not and take the unstaged pass.  Both against the oracle."""
    shape = (24, 16, 6)
    d = dataset(shape, seed=31, contrasts=("PDw", "T1w"), n_echoes=echoes, b1m=b1m)
    pg = mpm.make_problem(d["prot"], shape)
    po = orc.make_problem(d["prot"], shape)
    rng = np.random.default_rng(32)
    y = (d["y_true"] + 0.05 * rng.standard_normal(d["y_true"].shape)).astype(np.float32)
    g, h, nll = mpm.mpm_grad_hess(pg, to_dev(d["x"]), to_dev(y), to_dev(d["b1p"]), to_dev(d["b1m"]))
    nll_o, g_o, h_o = orc.grad_hess(po, d["x"], y, d["b1p"], d["b1m"])
    from cases import assert_close_scaled
    assert_close_scaled(to_np(g), g_o, 1e-4, "g")
    assert_close_scaled(to_np(h), h_o, 1e-4, "h")
    assert abs(nll.item() - nll_o) <= 2e-6 * abs(nll_o)
