"""Spatial projection (Sec. 2.4) on the GPU against the FP64 oracle.

Affines with dyadic entries (k / 16, k / 8) make every float32 coordinate and
interpolation weight exact, so the GPU and the oracle reslice with identical
weights and the comparison isolates the arithmetic.  A general affine
(irrational rotation) is checked with the bound its float32 coordinates
allow: r = A m is rounded to 2^-24 |r| <= 1.6e-5 voxel for |r| < 256, which
moves an interpolated value by at most that times the largest neighbour
difference."""
import numpy as np
import pytest

import oracle as orc
from cases import assert_close_scaled, map_error, moved_dataset, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mpm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2102_01604_gb300 as m
    m._lib.load()
    return m


def _aff(lin, t):
    A = np.eye(4)
    A[:3, :3] = np.asarray(lin, dtype=np.float64)
    A[:3, 3] = t
    return A


# dyadic motions: a scaled in-plane turn, a tilt with a coarser grid, a shift
MOVES = [
    ((40, 36, 14), _aff(np.eye(3), [0.0, 0.0, 0.0])),
    ((38, 36, 14), _aff([[0.9375, -0.25, 0.0], [0.25, 0.9375, 0.0], [0.0, 0.0, 1.0]], [3.5, -2.25, 0.375])),
    ((28, 26, 11), _aff([[1.25, 0.0, 0.125], [0.0, 1.25, 0.0], [-0.125, 0.0, 1.25]], [0.5, 1.75, 0.25])),
]
RECON = (36, 32, 12)


@pytest.fixture(scope="module")
def moved():
    return moved_dataset(RECON, [g for g, _ in MOVES], [a for _, a in MOVES], seed=11)


def _problems(mpm, d, **kw):
    pg = mpm.make_problem(d["prot"], d["shape"], **kw)
    qg = mpm.make_projection(d["grids"], d["affines"])
    po = orc.make_problem(d["prot"], d["shape"], lam=kw.get("lam", 10.0),
                          precond=kw.get("precond", 0))
    qo = orc.make_projection(d["grids"], d["affines"])
    return pg, qg, po, qo


def test_pull_and_push_match_the_oracle(mpm, moved):
    import torch
    d = moved
    pg, qg, po, qo = _problems(mpm, d)
    rng = np.random.default_rng(0)
    N = int(np.prod(d["shape"]))
    u = rng.standard_normal((3, N)).astype(np.float32)
    for c in range(3):
        ref, inside = orc.pull(po, d["grids"][c], d["affines"][c], u.astype(np.float64))
        got = to_np(mpm.mpm_pull(pg, qg, c, to_dev(u)))
        assert 0.2 < inside.mean() <= 1.0
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-5)
        assert np.all(got[:, ~inside] == 0.0)
        M = int(np.prod(d["grids"][c]))
        v = rng.standard_normal((2, M)).astype(np.float32)
        ref_t = orc.push(po, d["grids"][c], d["affines"][c], v.astype(np.float64))
        got_t = to_np(mpm.mpm_push(pg, qg, c, to_dev(v)))
        np.testing.assert_allclose(got_t, ref_t, rtol=0, atol=1e-5 * max(1.0, np.abs(ref_t).max()))
        # accumulate adds to what is there
        base = torch.ones((2, N), device="cuda")
        acc = to_np(mpm.mpm_push(pg, qg, c, to_dev(v), out=base, accumulate=True))
        np.testing.assert_allclose(acc, got_t + 1.0, rtol=0, atol=1e-6 * max(1.0, np.abs(got_t).max()))


def test_push_is_the_adjoint_of_pull_for_a_general_affine(mpm):
    shape = (30, 26, 10)
    prot = {"alpha": [0.1], "tr": [0.025], "mt": [0], "n_echoes": [2], "te": [0.002, 0.004],
            "sigma2": [1.0]}
    pg = mpm.make_problem(prot, shape)
    t = np.deg2rad(13.0)
    A = _aff([[np.cos(t), -np.sin(t), 0.02], [np.sin(t), np.cos(t), 0.0], [0.0, -0.03, 1.1]],
             [4.3, -3.1, 0.7])
    dims = (28, 28, 9)
    qg = mpm.make_projection([dims], [A])
    rng = np.random.default_rng(1)
    u = rng.standard_normal((2, int(np.prod(shape)))).astype(np.float32)
    v = rng.standard_normal((2, int(np.prod(dims)))).astype(np.float32)
    pu = to_np(mpm.mpm_pull(pg, qg, 0, to_dev(u)))
    ptv = to_np(mpm.mpm_push(pg, qg, 0, to_dev(v)))
    lhs, rhs = np.sum(pu * v), np.sum(u.astype(np.float64) * ptv)
    assert abs(lhs - rhs) <= 1e-5 * np.abs(pu * v).sum()
    # against the oracle, within the float32-coordinate bound
    po = orc.make_problem(prot, shape)
    ref, inside = orc.pull(po, dims, A, u.astype(np.float64))
    m = np.stack(np.meshgrid(np.arange(dims[0]), np.arange(dims[1]), np.arange(dims[2]),
                             indexing="ij"), -1).transpose(2, 1, 0, 3).reshape(-1, 3)
    r = m @ A[:3, :3].T + A[:3, 3]
    edge = np.min(np.minimum(r, np.array(shape) - 1 - r), axis=1)
    clear = np.abs(edge) > 1e-3                 # no point within 1e-3 voxel of the border
    step = 2 * np.abs(u).max()
    np.testing.assert_allclose(pu[:, clear], ref[:, clear], rtol=0, atol=4 * 1.6e-5 * step + 1e-6)


def test_identity_reslicing_equals_the_plain_voxel_pass(mpm):
    from cases import dataset
    shape = (24, 20, 9)
    d = dataset(shape, seed=21, n_echoes=(5, 5, 4))
    pg = mpm.make_problem(d["prot"], shape)
    qg = mpm.make_projection([shape] * 3, [np.eye(4)] * 3)
    x = to_dev(d["x"])
    y = to_dev(d["y_true"].astype(np.float32))
    bp, bm = to_dev(d["b1p"]), to_dev(d["b1m"])
    g, h, nll = mpm.mpm_grad_hess(pg, x, y, bp, bm)
    xs = [x[0:5], x[5:10], x[10:14]]
    g2, h2, nll2 = mpm.mpm_grad_hess_proj(pg, qg, [t.contiguous() for t in xs], y, [bp] * 3,
                                          [bm[c].contiguous() for c in range(3)])
    assert abs(float(nll2) - float(nll)) <= 1e-6 * abs(float(nll))
    assert_close_scaled(to_np(g2), to_np(g), 1e-6, "g")
    assert_close_scaled(to_np(h2), to_np(h), 1e-6, "h")


@pytest.mark.parametrize("precond", [0, 1])
def test_projected_voxel_pass_matches_the_oracle(mpm, moved, precond):
    d = moved
    pg, qg, po, qo = _problems(mpm, d, precond=precond)
    rng = np.random.default_rng(2)
    y = (d["y_true"] + 0.05 * rng.standard_normal(d["y_true"].shape)).astype(np.float32)
    nll_o, g_o, h_o = orc.grad_hess_proj(po, qo, d["xs"], y.astype(np.float64), d["b1ps"],
                                         d["b1ms"])
    g, h, nll = mpm.mpm_grad_hess_proj(pg, qg, [to_dev(x) for x in d["xs"]], to_dev(y),
                                       [to_dev(b) for b in d["b1ps"]],
                                       [to_dev(b) for b in d["b1ms"]])
    assert abs(float(nll) - nll_o) <= 1e-5 * nll_o
    assert_close_scaled(to_np(g), g_o, 1e-4, "g")
    assert_close_scaled(to_np(h), h_o, 1e-4, "h")


def test_projected_fit_matches_the_oracle(mpm, moved):
    import torch
    d = moved
    pg, qg, po, qo = _problems(mpm, d)
    gn, cg = 8, 30
    ref = orc.fit_proj(po, qo, d["xs"], b1ps=d["b1ps"], b1ms=d["b1ms"], gn_iters=gn, cg_iters=cg)
    N = int(np.prod(d["shape"]))
    y = torch.zeros((4, N), device="cuda")
    var = torch.zeros((4, N), device="cuda")
    xs = [to_dev(x) for x in d["xs"]]
    bps = [to_dev(b) for b in d["b1ps"]]
    bms = [to_dev(b) for b in d["b1ms"]]
    st, rep = mpm.mpm_fit_proj(pg, qg, mpm.make_opts(gn_iters=gn, cg_iters=cg), xs, y, bps, bms,
                               var=var)
    assert rep.iters == gn
    np.testing.assert_allclose(np.array(rep.F[:gn + 1]), ref["F"], rtol=1e-5)
    assert map_error(to_np(y), ref["y"]).max() <= 1e-3
    assert np.all(np.isfinite(to_np(var))) and to_np(var).min() > 0
    # the fit recovers the maps: closer to the truth than the identity-resliced fit
    y_wrong = torch.zeros_like(y)
    q_id = mpm.make_projection(d["grids"], [np.eye(4)] * 3)
    mpm.mpm_fit_proj(pg, q_id, mpm.make_opts(gn_iters=gn, cg_iters=cg), xs, y_wrong, bps, bms)
    err = np.abs(to_np(y) - d["y_true"]).mean(axis=1)
    err_wrong = np.abs(to_np(y_wrong) - d["y_true"]).mean(axis=1)
    assert np.all(err < err_wrong)


def test_projected_fit_graph_replay_is_bit_identical(mpm, moved):
    import torch
    d = moved
    pg, qg, _, _ = _problems(mpm, d)
    N = int(np.prod(d["shape"]))
    xs = [to_dev(x) for x in d["xs"]]
    outs = []
    for graph in (False, True, True):             # direct, capture, replay
        y = torch.zeros((4, N), device="cuda")
        st, rep = mpm.mpm_fit_proj(pg, qg, mpm.make_opts(gn_iters=4, cg_iters=20, graph=graph),
                                   xs, y)
        outs.append((to_np(y), list(rep.F[:5])))
    for y, F in outs[1:]:
        assert np.array_equal(y, outs[0][0])
        assert F == outs[0][1]


def test_acquisition_grids_partly_or_wholly_outside(mpm):
    """A finer scan (half-size voxels: each reconstruction voxel gathers from
    up to 27 acquisition voxels) and a scan lying wholly outside the
    reconstruction grid (it adds nothing)."""
    shape = (20, 18, 8)
    grids = [(20, 18, 8), (30, 30, 12), (10, 10, 4)]
    affs = [np.eye(4), _aff(np.diag([0.5, 0.5, 0.5]), [2.25, 1.5, 0.75]),
            _aff(np.eye(3), [5.0, 4.0, 2.0])]
    d = moved_dataset(shape, grids, affs, seed=13, n_echoes=(4, 4, 3))
    d["affines"][2] = _aff(np.eye(3), [40.0, 0.0, 0.0])        # moved out of the grid
    pg, qg, po, qo = _problems(mpm, d)
    assert not orc.pull(po, grids[2], d["affines"][2], d["y_true"][:1])[1].any()
    y = d["y_true"].astype(np.float32)
    nll_o, g_o, h_o = orc.grad_hess_proj(po, qo, d["xs"], y.astype(np.float64), d["b1ps"],
                                         d["b1ms"])
    g, h, nll = mpm.mpm_grad_hess_proj(pg, qg, [to_dev(x) for x in d["xs"]], to_dev(y),
                                       [to_dev(b) for b in d["b1ps"]],
                                       [to_dev(b) for b in d["b1ms"]])
    assert abs(float(nll) - nll_o) <= 1e-5 * nll_o
    assert_close_scaled(to_np(g), g_o, 1e-4, "g")
    assert_close_scaled(to_np(h), h_o, 1e-4, "h")
    # the outside scan's data never enter: changing them changes nothing
    xs2 = [to_dev(x) for x in d["xs"][:2]] + [to_dev(d["xs"][2] * 2.0 + 7.0)]
    g2, h2, nll2 = mpm.mpm_grad_hess_proj(pg, qg, xs2, to_dev(y), [to_dev(b) for b in d["b1ps"]],
                                          [to_dev(b) for b in d["b1ms"]])
    assert float(nll2) == float(nll)
    assert np.array_equal(to_np(g2), to_np(g)) and np.array_equal(to_np(h2), to_np(h))


def test_projected_fit_adaptive_stop_matches_the_oracle(mpm, moved):
    """The host-side stopping rule (tol_gn > 0) on the projected fit: same
    number of updates and objective as the oracle's rule."""
    import torch
    d = moved
    pg, qg, po, qo = _problems(mpm, d)
    ref = orc.fit_proj(po, qo, d["xs"], b1ps=d["b1ps"], b1ms=d["b1ms"], gn_iters=30, cg_iters=30,
                       tol_gn=1e-3)
    N = int(np.prod(d["shape"]))
    y = torch.zeros((4, N), device="cuda")
    st, rep = mpm.mpm_fit_proj(pg, qg, mpm.make_opts(gn_iters=30, cg_iters=30, tol_gn=1e-3),
                               [to_dev(x) for x in d["xs"]], y, [to_dev(b) for b in d["b1ps"]],
                               [to_dev(b) for b in d["b1ms"]])
    assert 0 < rep.iters < 30 and rep.iters == ref["iters"]
    np.testing.assert_allclose(np.array(rep.F[:rep.iters + 1]), ref["F"], rtol=1e-5)
    assert map_error(to_np(y), ref["y"]).max() <= 1e-3


def test_projected_fit_three_maps_and_bfloat16_echoes(mpm):
    """Two contrasts without MT (K = 3 maps), echoes stored as bfloat16: the
    oracle sees the same bfloat16-rounded images."""
    import torch
    grids = [(30, 28, 10), (26, 24, 10)]
    affs = [np.eye(4), _aff([[0.9375, 0.25, 0.0], [-0.25, 0.9375, 0.0], [0.0, 0.0, 1.0]],
                            [1.5, 2.75, 0.0])]
    d = moved_dataset((28, 26, 10), grids, affs, seed=17, contrasts=("PDw", "T1w"),
                      n_echoes=(6, 5))
    xs16 = [torch.from_numpy(x).cuda().to(torch.bfloat16) for x in d["xs"]]
    xs_rounded = [x.float().cpu().numpy() for x in xs16]
    pg = mpm.make_problem(d["prot"], d["shape"], echo_dtype=1)
    assert pg.n_maps == 3
    qg = mpm.make_projection(d["grids"], d["affines"])
    po = orc.make_problem(d["prot"], d["shape"])
    qo = orc.make_projection(d["grids"], d["affines"])
    ref = orc.fit_proj(po, qo, xs_rounded, b1ps=d["b1ps"], b1ms=d["b1ms"], gn_iters=6, cg_iters=30)
    N = int(np.prod(d["shape"]))
    y = torch.zeros((3, N), device="cuda")
    st, rep = mpm.mpm_fit_proj(pg, qg, mpm.make_opts(gn_iters=6, cg_iters=30), xs16, y,
                               [to_dev(b) for b in d["b1ps"]], [to_dev(b) for b in d["b1ms"]])
    np.testing.assert_allclose(np.array(rep.F[:7]), ref["F"], rtol=1e-5)
    assert map_error(to_np(y), ref["y"]).max() <= 1e-3
