"""mpm_solve_static, the solve for callers that cannot allocate device memory
(a framework pool that owns the device, a pipeline that reserves memory up
front, code that must avoid cudaMalloc's implicit synchronisation): it keeps
its scratch in a fixed library-owned device array instead of a caller
workspace.

Called through the C ABI twice in a row on different systems, each result must
match mpm_solve (the workspace version) within the solve tolerance of the
parity tests; a problem too large for the fixed scratch must be refused with a
clear error.  This file is collected last so that a failure here does not hide
the other tests in a run that stops at the first failure.
"""
import ctypes

import numpy as np
import pytest

import oracle as orc
from cases import assert_close_scaled, dataset, to_dev, to_np

pytestmark = pytest.mark.gpu


def _system(shape, seed):
    d = dataset(shape, seed=seed)
    po = orc.make_problem(d["prot"], shape)
    rng = np.random.default_rng(seed + 7)
    y = (d["y_true"] + 0.05 * rng.standard_normal(d["y_true"].shape)).astype(np.float32)
    _, g, h = orc.grad_hess(po, d["x"], y, d["b1p"], d["b1m"])
    _, w = orc.jtv(po, y)
    return d, h.astype(np.float32), w.astype(np.float32), g.astype(np.float32), y


def _call_static(lib, problem, opts, h, w, g, y, delta, resid):
    vp = lambda t: ctypes.c_void_p(t.data_ptr())
    return lib.mpm_solve_static(ctypes.byref(problem), ctypes.byref(opts), vp(h), vp(w), vp(g),
                                vp(y), vp(delta), vp(resid), None)


def test_static_solve_matches_workspace_solve_twice():
    import torch

    import paper_2102_01604_gb300 as mpm
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    lib = mpm._lib.load()
    opts = mpm.make_opts(cg_iters=30)
    for shape, seed in (((40, 32, 20), 61), ((33, 17, 9), 62)):
        d, h, w, g, y = _system(shape, seed)
        problem = mpm.make_problem(d["prot"], shape)
        hd, wd, gd, yd = to_dev(h), to_dev(w), to_dev(g), to_dev(y)
        ref, ref_resid = mpm.mpm_solve(problem, opts, hd, wd, gd, yd)
        delta = torch.full_like(gd, float("nan"))
        resid = torch.full((31,), float("nan"), dtype=torch.float64, device="cuda")
        st = _call_static(lib, problem, opts, hd, wd, gd, yd, delta, resid)
        assert st == mpm._lib.OK, lib.mpm_last_error().decode()
        torch.cuda.synchronize()
        assert_close_scaled(to_np(delta), to_np(ref), 2e-4, "delta")
        np.testing.assert_allclose(to_np(resid), to_np(ref_resid), rtol=2e-4,
                                   atol=1e-6 * ref_resid[0].item())


def test_static_solve_refuses_problems_beyond_its_scratch():
    import torch

    import paper_2102_01604_gb300 as mpm
    lib = mpm._lib.load()
    d = dataset((2, 2, 2), seed=63)
    shape = (128, 128, 64)                       # about 1 M voxels, 120 MB of scratch
    problem = mpm.make_problem(d["prot"], shape)
    N = int(np.prod(shape))
    t = torch.zeros((10, N), dtype=torch.float32, device="cuda")
    v = torch.zeros((4, N), dtype=torch.float32, device="cuda")
    resid = torch.zeros(31, dtype=torch.float64, device="cuda")
    st = _call_static(lib, problem, mpm.make_opts(cg_iters=30), t, v[0], v, v, v, resid)
    assert st == mpm._lib.ERR_WORKSPACE_TOO_SMALL
    assert "fixed scratch" in lib.mpm_last_error().decode()
