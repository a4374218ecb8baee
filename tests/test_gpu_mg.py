"""The multigrid-preconditioned CG (opts.mg_levels > 0, an option beside the
paper's block preconditioner) against the FP64 oracle's orc_mg_pcg: the same
V-cycle (aggregation levels, Galerkin coarse operators, damped block-Jacobi
sweeps) and the same CG recurrence, compared after a fixed number of
iterations, element by element.

Tolerances as for the block-Jacobi solve (float32 arithmetic through the
cycle and the recurrence): delta within 2e-4 x (|ref| + rms of the map),
residual norms within the same relative bound above 1e-6 |r_0|; the whole fit
at the fit tolerances.
"""
import numpy as np
import pytest

import oracle as orc
from cases import assert_close_scaled, dataset, map_error, to_dev, to_np

pytestmark = pytest.mark.gpu

MG = dict(mg_levels=8, mg_nu=1, mg_omega=0.7, mg_coarse_sweeps=20)


@pytest.fixture(scope="module")
def mpm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2102_01604_gb300 as m
    m._lib.load()
    return m


def _omg(**kw):
    return orc.make_mg(levels=kw.get("mg_levels", 8), nu=kw.get("mg_nu", 1),
                       omega=kw.get("mg_omega", 0.7), coarse_sweeps=kw.get("mg_coarse_sweeps", 20))


def _case(shape, seed, vx=(1.0, 1.0, 1.0), contrasts=("PDw", "T1w", "MTw"), n_echoes=(8, 8, 6)):
    d = dataset(shape, seed=seed, contrasts=contrasts, n_echoes=n_echoes)
    po = orc.make_problem(d["prot"], shape, vx=vx, lam=10.0, eps=1e-3)
    rng = np.random.default_rng(seed + 1)
    y = (d["y_true"] + 0.05 * rng.standard_normal(d["y_true"].shape)).astype(np.float32)
    _, g, h = orc.grad_hess(po, d["x"], y, d["b1p"], d["b1m"])
    _, w = orc.jtv(po, y)
    return d, po, h.astype(np.float32), w.astype(np.float32), g.astype(np.float32), y


@pytest.mark.parametrize("shape,vx,cg", [((32, 32, 16), (1.0, 1.0, 1.0), 1),
                                         ((32, 32, 16), (1.0, 1.0, 1.0), 10),
                                         ((37, 11, 5), (0.8, 1.1, 1.7), 4),
                                         ((48, 40, 24), (1.0, 1.0, 1.0), 6)])
def test_mg_solve_matches_the_oracle(mpm, shape, vx, cg):
    d, po, h, w, g, y = _case(shape, 7, vx)
    pg = mpm.make_problem(d["prot"], shape, vx=vx, lam=10.0, eps=1e-3)
    opts = mpm.make_opts(cg_iters=cg, **MG)
    delta, resid = mpm.mpm_solve(pg, opts, to_dev(h), to_dev(w), to_dev(g), to_dev(y))
    d_o, it, r_o = orc.mg_solve(po, h, w, g, y, cg, _omg(**MG))
    assert it == cg
    assert_close_scaled(to_np(delta), d_o, 2e-4, "delta")
    r = to_np(resid)
    np.testing.assert_allclose(r[:it + 1], r_o, rtol=2e-4 * max(1, cg) ** 0.5 + 1e-5,
                               atol=1e-6 * r_o[0])


def test_mg_three_maps_and_few_levels(mpm):
    """K = 3 (no MT contrast), two levels only, two sweeps per side."""
    kw = dict(mg_levels=2, mg_nu=2, mg_omega=0.6, mg_coarse_sweeps=5)
    d, po, h, w, g, y = _case((30, 22, 12), 9, contrasts=("PDw", "T1w"), n_echoes=(6, 5))
    pg = mpm.make_problem(d["prot"], (30, 22, 12), lam=10.0, eps=1e-3)
    assert pg.n_maps == 3
    delta, _ = mpm.mpm_solve(pg, mpm.make_opts(cg_iters=5, **kw), to_dev(h), to_dev(w),
                             to_dev(g), to_dev(y))
    d_o, it, _ = orc.mg_solve(po, h, w, g, y, 5, _omg(**kw))
    assert_close_scaled(to_np(delta), d_o, 2e-4, "delta")


def test_mg_tolerance_stop(mpm):
    d, po, h, w, g, y = _case((40, 32, 20), 11)
    pg = mpm.make_problem(d["prot"], (40, 32, 20), lam=10.0, eps=1e-3)
    delta, resid = mpm.mpm_solve(pg, mpm.make_opts(cg_iters=100, tol_cg=1e-3, **MG), to_dev(h),
                                 to_dev(w), to_dev(g), to_dev(y))
    d_o, it, r_o = orc.mg_solve(po, h, w, g, y, 100, _omg(**MG), tol=1e-3)
    r = to_np(resid)
    ran = int(np.sum(np.isfinite(r))) - 1
    assert ran == it, (ran, it)
    assert_close_scaled(to_np(delta), d_o, 1e-3, "delta")


def test_mg_fit_matches_the_oracle(mpm):
    import torch
    shape = (32, 24, 16)
    d = dataset(shape, seed=13)
    pg = mpm.make_problem(d["prot"], shape)
    po = orc.make_problem(d["prot"], shape)
    K, N = pg.n_maps, int(np.prod(shape))
    y = torch.zeros((K, N), dtype=torch.float32, device="cuda")
    st, rep = mpm.mpm_fit(pg, mpm.make_opts(gn_iters=4, cg_iters=8, **MG), to_dev(d["x"]), y,
                          to_dev(d["b1p"]), to_dev(d["b1m"]))
    ref = orc.fit(po, d["x"], None, d["b1p"], d["b1m"], gn_iters=4, cg_iters=8, mg=_omg(**MG))
    assert rep.iters == ref["iters"] == 4
    np.testing.assert_allclose(np.array(rep.F[:5]), ref["F"], rtol=1e-5)
    assert map_error(to_np(y), ref["y"]).max() <= 1e-3
