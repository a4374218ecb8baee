"""Parity of every C-ABI call against the FP64 oracle, element by element, on
seeded inputs spanning several stencil tiles and ragged tails.

Tolerances, from float32 rounding (2^-24 relative per operation) grown over
the sums and solves each output goes through:
  forward, gradient, Hessian   1e-4 x (|ref| + rms of the row)
  likelihood, JTV energy       2e-6 relative
  JTV weights                  1e-5 relative
  PCG update delta             2e-4 x (|ref| + rms of the map)
  uncertainty (float64 math)   1e-5 relative
  whole fit                    1e-3 x max(1, |y|) per voxel and map (log space),
                               1e-5 relative on the objective at every update
"""
import numpy as np
import pytest

import oracle as orc
from cases import assert_close_scaled, dataset, map_error, to_dev, to_np

pytestmark = pytest.mark.gpu

SHAPES = [(32, 32, 16), (37, 11, 5), (1, 9, 7), (65, 3, 2)]


@pytest.fixture(scope="module")
def mpm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2102_01604_gb300 as m
    m._lib.load()
    return m


def _problems(mpm, d, **kw):
    return (mpm.make_problem(d["prot"], d["shape"], **kw),
            orc.make_problem(d["prot"], d["shape"], **{k: v for k, v in kw.items()
                                                       if k != "echo_dtype"}))


@pytest.mark.parametrize("shape", SHAPES)
def test_forward(mpm, shape):
    d = dataset(shape, seed=1)
    pg, po = _problems(mpm, d)
    y32 = d["y_true"].astype(np.float32)
    s = mpm.mpm_forward(pg, to_dev(y32), to_dev(d["b1p"]), to_dev(d["b1m"]))
    ref = orc.forward(po, y32, d["b1p"], d["b1m"])
    assert_close_scaled(to_np(s), ref, 1e-5, "forward")


@pytest.mark.parametrize("precond", [0, 1, 2])
@pytest.mark.parametrize("shape", SHAPES)
def test_grad_hess(mpm, shape, precond):
    d = dataset(shape, seed=2)
    pg, po = _problems(mpm, d, precond=precond)
    rng = np.random.default_rng(3)
    y = (d["y_true"] + 0.05 * rng.standard_normal(d["y_true"].shape)).astype(np.float32)
    g, h, nll = mpm.mpm_grad_hess(pg, to_dev(d["x"]), to_dev(y), to_dev(d["b1p"]),
                                  to_dev(d["b1m"]))
    nll_o, g_o, h_o = orc.grad_hess(po, d["x"], y, d["b1p"], d["b1m"])
    assert_close_scaled(to_np(g), g_o, 1e-4, "g")
    assert_close_scaled(to_np(h), h_o, 1e-4, "h")
    assert abs(nll.item() - nll_o) <= 2e-6 * abs(nll_o)


@pytest.mark.parametrize("bf16,contrasts,echoes", [
    (False, ("PDw", "T1w", "MTw"), (8, 8, 6)),
    (True, ("PDw", "T1w", "MTw"), (8, 8, 6)),
    (False, ("T1w", "MTw", "PDw"), (6, 8, 8)),
    (False, ("MTw", "PDw", "VFA15", "T1w"), (5, 7, 7, 4)),
])
def test_grad_hess_pairs_equal_single_voxels(mpm, bf16, contrasts, echoes):
    """The voxel pass stages its rows in shared memory when N is a multiple of
    8 and every array is 16-byte aligned; otherwise it takes two voxels per
    thread when N is even and every array is aligned to two elements, else one.
    With the images 0, 2 and 1 elements off, the three forms run on the same
    inputs.  Each voxel's arithmetic is the same, so g and h agree bit for bit
    (the NLL sums in another order).  The staged form reuses contrast 0's flip
    factors for the contrasts at its angle and the previous contrast's echo
    exponentials for the same echo times; the contrast orders cover reuse and
    none (T1w first: no other contrast at 21 degrees)."""
    import torch
    shape = (36, 22, 10)
    d = dataset(shape, seed=21, contrasts=contrasts, n_echoes=echoes)
    pg, po = _problems(mpm, d)
    if bf16:
        pg.echo_dtype = 1
    xt = torch.bfloat16 if bf16 else torch.float32
    x = to_dev(d["x"]).to(xt)
    y = to_dev(d["y_true"].astype(np.float32))
    out = []
    for off in (0, 2, 1):
        buf = torch.empty(x.numel() + off, dtype=xt, device="cuda")
        x_off = buf[off:].view(x.shape)
        x_off.copy_(x)
        out.append(mpm.mpm_grad_hess(pg, x_off, y, to_dev(d["b1p"]), to_dev(d["b1m"])))
    (g2, h2, n2) = out[0]
    for g1, h1, n1 in out[1:]:
        assert np.array_equal(to_np(g1), to_np(g2))
        assert np.array_equal(to_np(h1), to_np(h2))
        assert abs(n1.item() - n2.item()) <= 1e-6 * abs(n1.item())
    if not bf16:
        nll_o, g_o, h_o = orc.grad_hess(po, d["x"], d["y_true"].astype(np.float32), d["b1p"],
                                        d["b1m"])
        assert_close_scaled(to_np(g2), g_o, 1e-4, "g")
        assert_close_scaled(to_np(h2), h_o, 1e-4, "h")


def test_grad_hess_without_b1_and_mt(mpm):
    d = dataset((20, 9, 4), seed=4, contrasts=("PDw", "T1w"), n_echoes=(6, 5), b1p=False,
                b1m=False)
    pg, po = _problems(mpm, d)
    assert pg.n_maps == 3
    y = d["y_true"].astype(np.float32)
    g, h, nll = mpm.mpm_grad_hess(pg, to_dev(d["x"]), to_dev(y))
    nll_o, g_o, h_o = orc.grad_hess(po, d["x"], y)
    assert_close_scaled(to_np(g), g_o, 1e-4, "g")
    assert_close_scaled(to_np(h), h_o, 1e-4, "h")
    assert abs(nll.item() - nll_o) <= 2e-6 * abs(nll_o)


# plus volumes with several z ranges per tile column and a 3-plane one
JTV_SHAPES = SHAPES + [(48, 20, 9), (44, 10, 3), (64, 24, 40)]


@pytest.mark.parametrize("shape", JTV_SHAPES)
@pytest.mark.parametrize("vx", [(1.0, 1.0, 1.0), (0.8, 1.1, 1.7)])
def test_jtv_weights(mpm, shape, vx):
    d = dataset(shape, seed=5)
    pg, po = _problems(mpm, d, vx=vx, lam=(10.0, 7.0, 4.0, 2.0), eps=1e-3)
    rng = np.random.default_rng(6)
    y = (d["y_true"] + 0.02 * rng.standard_normal(d["y_true"].shape)).astype(np.float32)
    w, jtv = mpm.mpm_jtv_weights(pg, to_dev(y))
    e_o, w_o = orc.jtv(po, y)
    np.testing.assert_allclose(to_np(w), w_o, rtol=1e-5)
    assert abs(jtv.item() - e_o) <= 2e-6 * e_o


def _system(d, po, seed):
    """Newton-system inputs computed by the oracle, rounded to float32."""
    rng = np.random.default_rng(seed)
    y = (d["y_true"] + 0.05 * rng.standard_normal(d["y_true"].shape)).astype(np.float32)
    _, g, h = orc.grad_hess(po, d["x"], y, d["b1p"], d["b1m"])
    _, w = orc.jtv(po, y)
    return h.astype(np.float32), w.astype(np.float32), g.astype(np.float32), y


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("cg_iters", [1, 2, 30])
def test_solve(mpm, shape, cg_iters):
    d = dataset(shape, seed=7)
    pg, po = _problems(mpm, d)
    h, w, g, y = _system(d, po, 8)
    opts = mpm.make_opts(cg_iters=cg_iters)
    delta, resid = mpm.mpm_solve(pg, opts, to_dev(h), to_dev(w), to_dev(g), to_dev(y))
    d_o, it, r_o = orc.solve(po, h, w, g, y, cg_iters)
    assert it == cg_iters
    assert_close_scaled(to_np(delta), d_o, 2e-4, "delta")
    r = to_np(resid)
    # float32 residuals bottom out near 1e-7 of |r_0|: compare above that floor
    np.testing.assert_allclose(r[:it + 1], r_o, rtol=2e-4 * max(1, cg_iters) ** 0.5 + 1e-5,
                               atol=1e-6 * r_o[0])


def test_solve_tolerance_stop(mpm):
    d = dataset((24, 16, 8), seed=9)
    pg, po = _problems(mpm, d)
    h, w, g, y = _system(d, po, 10)
    opts = mpm.make_opts(cg_iters=200, tol_cg=1e-3)
    delta, resid = mpm.mpm_solve(pg, opts, to_dev(h), to_dev(w), to_dev(g), to_dev(y))
    d_o, it, r_o = orc.solve(po, h, w, g, y, 200, tol=1e-3)
    r = to_np(resid)
    ran = int(np.sum(np.isfinite(r))) - 1
    assert ran == it, (ran, it)
    assert_close_scaled(to_np(delta), d_o, 1e-3, "delta")


# (65, 3, 2): N even with nx odd, so the two-voxel threads' pairs straddle rows
@pytest.mark.parametrize("shape", SHAPES[:2] + [(65, 3, 2)])
def test_uncertainty(mpm, shape):
    d = dataset(shape, seed=11)
    pg, po = _problems(mpm, d)
    h, w, g, y = _system(d, po, 12)
    var, logdet, mom = mpm.mpm_uncertainty(pg, to_dev(h), to_dev(w), to_dev(y),
                                           want_moments=True)
    v_o, ld_o, m_o, st = orc.uncertainty(po, h, w, y)
    assert st == 0
    np.testing.assert_allclose(to_np(var), v_o, rtol=1e-5)
    np.testing.assert_allclose(to_np(logdet), ld_o, rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(to_np(mom), m_o, rtol=1e-5)
    # two voxels per thread (N even, arrays 8-byte aligned) or one (an output
    # one element off): the same arithmetic per voxel, the same bits
    import torch
    K, N = pg.n_maps, h.shape[1]
    buf = torch.empty(K * N + 1, dtype=torch.float32, device="cuda")
    var1 = buf[1:].view(K, N)
    mpm.mpm_uncertainty(pg, to_dev(h), to_dev(w), to_dev(y), var=var1, want_moments=True)
    assert np.array_equal(to_np(var1), to_np(var))


def test_uncertainty_ill_conditioned_blocks(mpm):
    """The variances come from float32 Cholesky factors of the equilibrated
    blocks; a block whose smallest equilibrated pivot is below 1e-2 is inverted
    in float64 instead.  Every third voxel gets a block whose first two maps
    are correlated at 0.999 (pivot 2e-3, condition number about 2000, where
    float32 would miss 1e-5), the prior made too weak to mend it; every voxel
    matches the oracle.  A block that is not positive definite gives non-finite
    variances (mpm_uncertainty takes no workspace to report it)."""
    d = dataset((16, 12, 6), seed=13)
    pg, po = _problems(mpm, d)
    h, w, g, y = _system(d, po, 14)
    K, N = pg.n_maps, h.shape[1]
    tri = {}
    t = 0
    for a in range(K):
        for b in range(a, K):
            tri[(a, b)] = t
            t += 1
    w = np.full_like(w, 1e-6)
    sel = np.arange(0, N, 3)
    for (a, b), t in tri.items():
        if a != b:
            h[t, sel] = 0.0
    h[tri[(0, 1)], sel] = (0.999 * np.sqrt(h[tri[(0, 0)], sel].astype(np.float64)
                                           * h[tri[(1, 1)], sel])).astype(np.float32)
    var, logdet, mom = mpm.mpm_uncertainty(pg, to_dev(h), to_dev(w), to_dev(y), want_moments=True)
    v_o, ld_o, m_o, st = orc.uncertainty(po, h, w, y)
    assert st == 0
    np.testing.assert_allclose(to_np(var), v_o, rtol=1e-5)
    np.testing.assert_allclose(to_np(logdet), ld_o, rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(to_np(mom), m_o, rtol=1e-5)
    # an indefinite block
    h[tri[(0, 1)], 4] = 1.5 * np.sqrt(h[tri[(0, 0)], 4] * h[tri[(1, 1)], 4])
    for (a, b), t in tri.items():
        if a != b and (a, b) != (0, 1):
            h[t, 4] = 0.0
    var, _, _ = mpm.mpm_uncertainty(pg, to_dev(h), to_dev(w), want_logdet=False)
    v = to_np(var)
    assert not np.all(np.isfinite(v[:, 4]))
    ok = np.ones(N, bool)
    ok[4] = False
    assert np.all(np.isfinite(v[:, ok]))


def _fit_both(mpm, d, gn_iters=10, cg_iters=30, npi=1, tol_gn=0.0, tol_cg=0.0, **kw):
    import torch
    pg, po = _problems(mpm, d, **kw)
    K, N = pg.n_maps, int(np.prod(d["shape"]))
    y = torch.zeros((K, N), dtype=torch.float32, device="cuda")
    opts = mpm.make_opts(gn_iters=gn_iters, cg_iters=cg_iters, newton_per_irls=npi,
                         tol_gn=tol_gn, tol_cg=tol_cg)
    var = torch.empty((K, N), dtype=torch.float32, device="cuda")
    st, rep = mpm.mpm_fit(pg, opts, to_dev(d["x"]), y, to_dev(d["b1p"]), to_dev(d["b1m"]),
                          var=var)
    ref = orc.fit(po, d["x"], None, d["b1p"], d["b1m"], gn_iters=gn_iters, cg_iters=cg_iters,
                  newton_per_irls=npi, tol_gn=tol_gn, tol_cg=tol_cg)
    return st, rep, to_np(y), to_np(var), ref, po


def _check_fit(rep, y, ref):
    assert rep.iters == ref["iters"]
    F = np.array(rep.F[:rep.iters + 1])
    np.testing.assert_allclose(F, ref["F"], rtol=1e-5)
    err = map_error(y, ref["y"])
    assert err.max() <= 1e-3, f"max map error {err.max():.3e} (map {np.unravel_index(err.argmax(), err.shape)})"
    return err


def test_fit_plain_32x32x16(mpm):
    """The small configuration: 32x32x16, PDw/T1w/MTw 8/8/6 echoes, Rician
    SNR 20, JTV lambda = 10, 10 updates x 30 PCG iterations."""
    d = dataset((32, 32, 16), seed=0, b1m=False)
    st, rep, y, var, ref, po = _fit_both(mpm, d)
    err = _check_fit(rep, y, ref)
    print(f"fit 32x32x16: max map error {err.max():.2e}, F {rep.F[rep.iters]:.6e}")
    # Uncertainty at the final maps.  The GPU's variance is Eq. 43 at its own
    # final maps, which sit within the 1e-3 map bound of the oracle's; H and w
    # move with the maps (the echo signal is exponential in log R2*, so H's
    # terms move by a few times the map error), hence 5e-3 relative, not the
    # 1e-5 of the per-call test, which feeds both sides the same H and w.
    _, w_o = orc.jtv(po, ref["y"])
    _, _, h_o = orc.grad_hess(po, d["x"], ref["y"], d["b1p"], d["b1m"])
    v_o, _, _, _ = orc.uncertainty(po, h_o, w_o)
    assert np.all(np.abs(var - v_o) <= 5e-3 * v_o), np.max(np.abs(var - v_o) / v_o)


@pytest.mark.parametrize("case", ["no_mt", "ragged", "irls5", "aniso", "rowsum", "tol"])
def test_fit_variants(mpm, case):
    if case == "no_mt":
        d = dataset((17, 13, 6), seed=21, contrasts=("PDw", "T1w"), n_echoes=(8, 8))
        st, rep, y, var, ref, _ = _fit_both(mpm, d, gn_iters=6)
    elif case == "ragged":
        d = dataset((33, 9, 5), seed=22)
        st, rep, y, var, ref, _ = _fit_both(mpm, d, gn_iters=6)
    elif case == "irls5":
        d = dataset((20, 20, 6), seed=23)
        st, rep, y, var, ref, _ = _fit_both(mpm, d, gn_iters=10, npi=5)
    elif case == "aniso":
        d = dataset((20, 16, 6), seed=24)
        st, rep, y, var, ref, _ = _fit_both(mpm, d, gn_iters=6, vx=(0.8, 0.8, 1.6))
    elif case == "rowsum":
        d = dataset((20, 16, 6), seed=25)
        st, rep, y, var, ref, _ = _fit_both(mpm, d, gn_iters=6, precond=1)
    else:
        d = dataset((20, 16, 6), seed=26)
        st, rep, y, var, ref, _ = _fit_both(mpm, d, gn_iters=60, tol_gn=1e-4, tol_cg=1e-3,
                                            cg_iters=100)
        assert rep.iters < 60
    _check_fit(rep, y, ref)


def test_initial_maps(mpm):
    import torch
    d = dataset((24, 12, 5), seed=31)
    pg, po = _problems(mpm, d)
    y = torch.zeros((pg.n_maps, 24 * 12 * 5), dtype=torch.float32, device="cuda")
    mpm.mpm_fit(pg, mpm.make_opts(gn_iters=0), to_dev(d["x"]), y, to_dev(d["b1p"]),
                to_dev(d["b1m"]))
    y0 = orc.init(po, d["x"])
    np.testing.assert_allclose(to_np(y), y0, rtol=1e-6, atol=1e-6)


def test_bf16_echoes(mpm):
    """Echoes stored as bfloat16: the oracle is given the same rounded values."""
    import torch
    d = dataset((32, 16, 8), seed=41)
    xb = torch.from_numpy(d["x"]).to(torch.bfloat16)
    d["x"] = xb.to(torch.float32).numpy()
    pg, po = _problems(mpm, d, echo_dtype=1)
    y = d["y_true"].astype(np.float32)
    g, h, nll = mpm.mpm_grad_hess(pg, xb.cuda(), to_dev(y), to_dev(d["b1p"]), to_dev(d["b1m"]))
    nll_o, g_o, h_o = orc.grad_hess(po, d["x"], y, d["b1p"], d["b1m"])
    assert_close_scaled(to_np(g), g_o, 1e-4, "g")
    assert_close_scaled(to_np(h), h_o, 1e-4, "h")
    assert abs(nll.item() - nll_o) <= 2e-6 * abs(nll_o)
    K, N = pg.n_maps, 32 * 16 * 8
    yy = torch.zeros((K, N), dtype=torch.float32, device="cuda")
    st, rep = mpm.mpm_fit(pg, mpm.make_opts(gn_iters=5), xb.cuda(), yy, to_dev(d["b1p"]),
                          to_dev(d["b1m"]))
    ref = orc.fit(po, d["x"], None, d["b1p"], d["b1m"], gn_iters=5, cg_iters=30)
    _check_fit(rep, to_np(yy), ref)


@pytest.mark.parametrize("tile", [0, 1, 2])
def test_solve_every_stencil_tile_shape(mpm, tile):
    """The TMA PCG iteration in each tile shape (16x16, 32x8, 32x16) on a volume with
    ragged tiles in x and y, against the oracle."""
    shape = (76, 21, 9)
    d = dataset(shape, seed=81)
    pg, po = _problems(mpm, d)
    got, _ = mpm.mpm_autotune(pg, mpm.make_opts(), tile=tile)
    assert got == tile
    h, w, g, y = _system(d, po, 82)
    delta, resid = mpm.mpm_solve(pg, mpm.make_opts(cg_iters=30), to_dev(h), to_dev(w), to_dev(g),
                                 to_dev(y))
    d_o, it, r_o = orc.solve(po, h, w, g, y, 30)
    assert_close_scaled(to_np(delta), d_o, 2e-4, "delta")


def test_autotune_times_the_shapes(mpm):
    d = dataset((96, 48, 20), seed=83)
    pg = mpm.make_problem(d["prot"], (96, 48, 20))
    tile, ms = mpm.mpm_autotune(pg, mpm.make_opts())
    assert tile in (0, 1, 2)
    assert all(t > 0 for t in ms)
    assert ms[tile] == min(ms)


def _irregular_dataset(shape, seed):
    """Eight contrasts (the maximum), two with an MT pulse, 1 to 12 echoes each
    (46 images), three TRs, and irregular echo times in four contrasts: the
    echo loop's general branch, next to equally spaced and single-echo ones."""
    import math
    from cases import f32, round_protocol
    from paper_2102_01604_gb300 import phantom
    rng = np.random.default_rng(seed)
    n_echoes = [8, 1, 6, 3, 12, 2, 5, 9]
    te = []
    for c, ne in enumerate(n_echoes):
        if c in (0, 3):
            te += [0.0023 * (k + 1) for k in range(ne)]
        else:
            te += list(np.sort(rng.uniform(0.002, 0.03, ne)))
    prot = round_protocol({
        "names": [f"c{c}" for c in range(8)],
        "alpha": [math.radians(a) for a in (6, 21, 6, 15, 10, 30, 4, 18)],
        "tr": [0.025, 0.025, 0.025, 0.030, 0.018, 0.025, 0.040, 0.025],
        "mt": [0, 0, 1, 0, 1, 0, 0, 0], "n_echoes": n_echoes, "te": te, "sigma2": [1.0] * 8})
    ph = phantom.phantom(shape, seed=seed, n_contrasts=8)
    bp, bm = f32(ph["b1p"]), f32(ph["b1m"])
    s = orc.forward(orc.make_problem(prot, shape), ph["y"], bp, bm)
    prot["sigma2"] = [float(np.float32(v)) for v in phantom.noise_sigma2(s, prot)]
    prot = round_protocol(prot)
    x = f32(phantom.rician(s, prot, seed=seed + 1))
    return {"prot": prot, "shape": tuple(shape), "y_true": ph["y"], "b1p": bp, "b1m": bm, "x": x}


def test_irregular_echoes_and_most_contrasts(mpm):
    d = _irregular_dataset((19, 13, 5), seed=41)
    assert len(d["prot"]["te"]) == 46
    for precond in (0, 1):
        pg, po = _problems(mpm, d, precond=precond)
        y = (d["y_true"] + 0.05 * np.random.default_rng(5).standard_normal(d["y_true"].shape)
             ).astype(np.float32)
        if precond == 0:
            s = mpm.mpm_forward(pg, to_dev(y), to_dev(d["b1p"]), to_dev(d["b1m"]))
            assert_close_scaled(to_np(s), orc.forward(po, y, d["b1p"], d["b1m"]), 1e-5, "forward")
        g, h, nll = mpm.mpm_grad_hess(pg, to_dev(d["x"]), to_dev(y), to_dev(d["b1p"]),
                                      to_dev(d["b1m"]))
        nll_o, g_o, h_o = orc.grad_hess(po, d["x"], y, d["b1p"], d["b1m"])
        assert_close_scaled(to_np(g), g_o, 1e-4, "g")
        assert_close_scaled(to_np(h), h_o, 1e-4, "h")
        assert abs(nll.item() - nll_o) <= 2e-6 * abs(nll_o)
    st, rep, y, var, ref, _ = _fit_both(mpm, d, gn_iters=4, cg_iters=20)
    _check_fit(rep, y, ref)
