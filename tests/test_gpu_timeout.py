"""The bounded copy waits of the TMA-staged PCG iteration and of the staged
voxel pass, driven to their timeout on the GPU without any fault.

The test hook mpm_test_copy_timeout makes the iteration's producer warp issue
no copies and bounds every wait at 1 ms, so each compute warp's first wait
runs out.  The launch must then skip its work, drain its own copies (none
here), record the timeout in the workspace status and return; the solve stops
without a step.  Afterwards, with the hook off, the same context solves the
same system and matches the oracle: nothing was left hung or corrupted.
"""
import time

import numpy as np
import pytest

import oracle as orc
from cases import assert_close_scaled, dataset, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mpm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2102_01604_gb300 as m
    m._lib.load()
    return m


def test_copy_wait_timeout_is_reported_and_the_context_survives(mpm):
    import torch
    from paper_2102_01604_gb300 import _lib
    shape = (64, 32, 12)                   # the TMA iteration applies: nx % 4 == 0, tiles fit
    d = dataset(shape, seed=91)
    pg = mpm.make_problem(d["prot"], shape)
    po = orc.make_problem(d["prot"], shape)
    rng = np.random.default_rng(92)
    y = (d["y_true"] + 0.05 * rng.standard_normal(d["y_true"].shape)).astype(np.float32)
    _, g, h = orc.grad_hess(po, d["x"], y, d["b1p"], d["b1m"])
    _, w = orc.jtv(po, y)
    h, w, g = h.astype(np.float32), w.astype(np.float32), g.astype(np.float32)
    opts = mpm.make_opts(cg_iters=10)
    ws = mpm.workspace(pg, opts, _lib.CALL_SOLVE)
    args = (to_dev(h), to_dev(w), to_dev(g), to_dev(y))
    d_o, _, _ = orc.solve(po, h, w, g, y, 10)

    delta, _ = mpm.mpm_solve(pg, opts, *args, ws=ws)
    assert mpm.mpm_workspace_status(ws) == _lib.OK
    assert_close_scaled(to_np(delta), d_o, 2e-4, "delta before")

    mpm.mpm_test_copy_timeout(True, 1000.0)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        delta_t, resid_t = mpm.mpm_solve(pg, opts, *args, ws=ws)
        torch.cuda.synchronize()
        elapsed = time.perf_counter() - t0
        st = mpm.mpm_workspace_status(ws)
        msg = _lib.load().mpm_last_error().decode()
    finally:
        mpm.mpm_test_copy_timeout(False, 0.0)
    assert st == _lib.ERR_NUMERIC, st
    assert "copy wait timed out" in msg, msg
    # one launch waits about 1 ms per warp before it gives up; the solve then
    # stops, so the call ends far inside the default 2 s bound of one wait
    assert elapsed < 1.0, elapsed
    assert not torch.any(delta_t != 0).item()          # no step was taken
    r = to_np(resid_t)
    assert np.isfinite(r[0]) and np.all(np.isnan(r[1:]))

    delta2, resid2 = mpm.mpm_solve(pg, opts, *args, ws=ws)
    assert mpm.mpm_workspace_status(ws) == _lib.OK
    assert_close_scaled(to_np(delta2), d_o, 2e-4, "delta after")


@pytest.mark.parametrize("bf16", [False, True])
def test_voxel_pass_copy_timeout(mpm, bf16):
    """The staged voxel pass (N a multiple of 8, aligned arrays) under the
    same hook: its producer issues no row copies, every compute warp's first
    wait runs out, the timeout is recorded, and afterwards the same context
    computes g, h and the NLL of the oracle."""
    import torch
    from paper_2102_01604_gb300 import _lib
    shape = (40, 24, 12)
    d = dataset(shape, seed=93)
    pg = mpm.make_problem(d["prot"], shape, echo_dtype=1 if bf16 else 0)
    po = orc.make_problem(d["prot"], shape)
    x = to_dev(d["x"])
    if bf16:
        x = x.to(torch.bfloat16)
        d["x"] = x.float().cpu().numpy()
    y = d["y_true"].astype(np.float32)
    ws = mpm.workspace(pg, None, _lib.CALL_GRAD_HESS)
    args = (x, to_dev(y), to_dev(d["b1p"]), to_dev(d["b1m"]))
    mpm.mpm_test_copy_timeout(True, 1000.0)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mpm.mpm_grad_hess(pg, *args, ws=ws)
        torch.cuda.synchronize()
        elapsed = time.perf_counter() - t0
        st = mpm.mpm_workspace_status(ws)
        msg = _lib.load().mpm_last_error().decode()
    finally:
        mpm.mpm_test_copy_timeout(False, 0.0)
    assert st == _lib.ERR_NUMERIC, st
    assert "copy wait timed out" in msg, msg
    assert elapsed < 1.0, elapsed

    g, h, nll = mpm.mpm_grad_hess(pg, *args, ws=ws)
    assert mpm.mpm_workspace_status(ws) == _lib.OK
    nll_o, g_o, h_o = orc.grad_hess(po, d["x"], y, d["b1p"], d["b1m"])
    assert_close_scaled(to_np(g), g_o, 1e-4, "g")
    assert_close_scaled(to_np(h), h_o, 1e-4, "h")
    assert abs(nll.item() - nll_o) <= 2e-6 * abs(nll_o)
