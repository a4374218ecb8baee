"""Pins of the oracle's multigrid preconditioner (an option beside the
paper's block preconditioner of Sec. 2.6, Eq. 42).

The V-cycle is checked against what must hold for any correct implementation
of its definition, never against a retyping of it:
  - the coarse operators are Galerkin products: for a vector e of level l,
    e' A_l e equals (P e)' A (P e) with A built densely from the materialised
    finite-difference matrix G and P e the coarse values copied to every fine
    voxel they cover;
  - the cycle, as a matrix (applied to unit vectors), is symmetric and
    positive definite, so it is a valid CG preconditioner;
  - with one level, one undamped sweep, it is the block preconditioner, and
    CG then reproduces orc_pcg's iterates;
  - CG with it converges to the dense solve, and reaches the paper's 1e-3
    tolerance in far fewer iterations than the block preconditioner.
"""
import numpy as np
import pytest

from paper_2102_01604_gb300 import phantom
from test_oracle_pcg_trajectory import _blocks
from test_oracle_prior import dense_G


def _system(orc, shape, vx=(1.0, 1.0, 1.0), lam=(10.0, 7.0, 3.0, 2.0), seed=0, contrasts=None):
    prot = phantom.protocol() if contrasts is None else phantom.protocol(*contrasts)
    with_mt = any(prot["mt"])
    ph = phantom.phantom(shape, seed=seed, n_contrasts=len(prot["alpha"]), with_mt=with_mt)
    p0 = orc.make_problem(prot, shape, vx=vx)
    s = orc.forward(p0, ph["y"], ph["b1p"], ph["b1m"])
    prot["sigma2"] = phantom.noise_sigma2(s, prot)
    x = phantom.rician(s, prot, seed=seed + 1)
    p = orc.make_problem(prot, shape, vx=vx, lam=lam, eps=1e-2)
    rng = np.random.default_rng(seed + 2)
    y = ph["y"] + 0.2 * rng.standard_normal(ph["y"].shape)
    _, g, h = orc.grad_hess(p, x, y, ph["b1p"], ph["b1m"])
    _, w = orc.jtv(p, y)
    return p, g, h, w, y


def _dense_A(p, h, w, shape, vx, lam):
    K, N = p.n_maps, int(np.prod(shape))
    G = dense_G(shape, vx)
    GWG = G.T @ np.kron(np.diag(w), np.eye(6)) @ G
    return _blocks(h, K, N) + np.kron(np.diag(lam[:K]), GWG)


def _sparse_A(p, h, w, shape, vx, lam):
    """A = H + lambda (x) G'WG with G assembled as a sparse matrix (rows
    (n, d): (e_m - e_n) / h_d for the d-th neighbour m of n inside the volume)."""
    import scipy.sparse as sp
    nx, ny, nz = shape
    N = nx * ny * nz
    rows, cols, vals = [], [], []
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    n = (x + nx * (y + ny * z)).ravel()
    offs = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    for d, (dx, dy, dz) in enumerate(offs):
        xx, yy, zz = x.ravel() + dx, y.ravel() + dy, z.ravel() + dz
        ok = (xx >= 0) & (xx < nx) & (yy >= 0) & (yy < ny) & (zz >= 0) & (zz < nz)
        m = xx + nx * (yy + ny * zz)
        r = 6 * n[ok] + d
        hd = vx[d // 2]
        rows += [r, r]
        cols += [m[ok], n[ok]]
        vals += [np.full(ok.sum(), 1.0 / hd), np.full(ok.sum(), -1.0 / hd)]
    G = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(6 * N, N))
    GWG = G.T @ sp.diags(np.repeat(w, 6)) @ G
    K = p.n_maps
    t = 0
    idx = np.arange(N)
    rr, cc, vv = [], [], []
    for a in range(K):
        for b in range(a, K):
            rr += [a * N + idx] + ([b * N + idx] if a != b else [])
            cc += [b * N + idx] + ([a * N + idx] if a != b else [])
            vv += [h[t]] + ([h[t]] if a != b else [])
            t += 1
    Hs = sp.csr_matrix((np.concatenate(vv), (np.concatenate(rr), np.concatenate(cc))),
                       shape=(K * N, K * N))
    return (Hs + sp.kron(sp.diags(lam[:K]), GWG)).tocsr()


def _upsample(e, dims_c, shape):
    """P e: each fine voxel (x, y, z) takes the value of coarse voxel
    (x // f, y // f, z // f) of the level, f = 2^l."""
    K = e.shape[0]
    nx, ny, nz = shape
    f = [int(round(np.ceil(n / m))) for n, m in zip(shape, dims_c)]
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cidx = (x // f[0]) + dims_c[0] * ((y // f[1]) + dims_c[1] * (z // f[2]))
    return e[:, cidx.ravel()]


MG = dict(levels=8, nu=1, omega=0.7, coarse_sweeps=20)


def test_level_dimensions(orc):
    p = orc.make_problem(phantom.protocol(), (176, 240, 256))
    dims = orc.mg_levels(p, orc.make_mg(**MG))
    assert dims == [(176, 240, 256), (88, 120, 128), (44, 60, 64), (22, 30, 32), (11, 15, 16),
                    (6, 8, 8)]
    p = orc.make_problem(phantom.protocol(), (9, 5, 1))
    assert orc.mg_levels(p, orc.make_mg(**MG)) == [(9, 5, 1)]            # 45 voxels: one level
    p = orc.make_problem(phantom.protocol(), (17, 9, 6))
    assert orc.mg_levels(p, orc.make_mg(levels=2)) == [(17, 9, 6), (9, 5, 3)]


@pytest.mark.parametrize("shape,vx", [((20, 18, 12), (1.0, 1.0, 1.0)), ((19, 17, 13), (0.8, 1.3, 2.0))])
def test_coarse_operators_are_galerkin_products(orc, shape, vx):
    """Three levels (4000-odd voxels, coarsened twice)."""
    lam = (10.0, 7.0, 3.0, 2.0)
    p, g, h, w, y = _system(orc, shape, vx, lam)
    mg = orc.make_mg(levels=8, nu=1, omega=0.7, coarse_sweeps=2)
    dims = orc.mg_levels(p, mg)
    assert len(dims) == 3
    A = _sparse_A(p, h, w, shape, vx, lam)
    rng = np.random.default_rng(3)
    for lev, dc in enumerate(dims):
        for _ in range(3):
            e = rng.standard_normal((p.n_maps, int(np.prod(dc))))
            Pe = _upsample(e, dc, shape).ravel()
            got = orc.mg_energy(p, h, w, mg, lev, e)
            assert got == pytest.approx(Pe @ (A @ Pe), rel=1e-11), lev


@pytest.mark.parametrize("shape,k3", [((10, 8, 8), False), ((11, 9, 7), True)])
def test_vcycle_is_symmetric_positive_definite(orc, shape, k3):
    """Two levels (640 and 693 voxels; the coarse level holds at most 512)."""
    contrasts = (("PDw", "T1w"), (6, 5)) if k3 else None
    p, g, h, w, y = _system(orc, shape, contrasts=contrasts)
    K, N = p.n_maps, int(np.prod(shape))
    mg = orc.make_mg(levels=3, nu=1, omega=0.7, coarse_sweeps=4)
    assert len(orc.mg_levels(p, mg)) == 2
    B = np.zeros((K * N, K * N))
    for i in range(K * N):
        e = np.zeros(K * N)
        e[i] = 1.0
        B[:, i] = orc.mg_vcycle(p, h, w, mg, e.reshape(K, N)).ravel()
    asym = np.abs(B - B.T).max() / np.abs(B).max()
    assert asym < 1e-12, asym
    ev = np.linalg.eigvalsh(0.5 * (B + B.T))
    assert ev.min() > 0.0, ev.min()


def test_one_level_is_the_block_preconditioner(orc):
    """One level, one undamped sweep from zero: z = D^-1 r with D the voxel
    blocks H + diag(lambda d) of Eq. 42, so CG takes orc_pcg's iterates."""
    shape = (9, 7, 4)
    p, g, h, w, y = _system(orc, shape)
    K, N = p.n_maps, int(np.prod(shape))
    b = np.random.default_rng(5).standard_normal((K, N)) * np.abs(g).mean()
    mg = orc.make_mg(levels=1, nu=1, omega=1.0, coarse_sweeps=1)
    for it in (1, 2, 5, 12):
        xm, im, rm = orc.mg_pcg(p, h, w, b, it, mg)
        xo, io, ro = orc.pcg(p, h, w, b, it)
        assert im == io == it
        assert np.abs(xm - xo).max() <= 1e-11 * np.abs(xo).max()
        np.testing.assert_allclose(rm, ro, rtol=1e-10)


def test_mg_pcg_reaches_the_dense_solve(orc):
    shape = (10, 8, 6)
    lam = (10.0, 7.0, 3.0, 2.0)
    p, g, h, w, y = _system(orc, shape, lam=lam)
    K, N = p.n_maps, int(np.prod(shape))
    A = _dense_A(p, h, w, shape, (1.0, 1.0, 1.0), lam)
    b = np.random.default_rng(6).standard_normal(K * N)
    ref = np.linalg.solve(A, b)
    mg = orc.make_mg(levels=3, nu=1, omega=0.7, coarse_sweeps=10)
    x, it, res = orc.mg_pcg(p, h, w, b.reshape(K, N), 200, mg, tol=1e-12)
    assert it < 200
    assert np.abs(x.ravel() - ref).max() <= 1e-9 * np.abs(ref).max()


def test_mg_needs_far_fewer_iterations(orc):
    """On a Newton system of the fit's first update (constant maps, so the
    JTV weights are all 1/eps and the prior dominates), CG with the V-cycle
    reaches |r| <= 1e-3 |r_0| in a fraction of the iterations the block
    preconditioner needs."""
    from cases import dataset
    shape = (32, 32, 16)
    d = dataset(shape, seed=0)
    p = orc.make_problem(d["prot"], shape, lam=10.0, eps=1e-3)
    y0 = orc.init(p, d["x"])
    _, g, h = orc.grad_hess(p, d["x"], y0, d["b1p"], d["b1m"])
    _, w = orc.jtv(p, y0)
    _, it_b, _ = orc.solve(p, h, w, g, y0, 400, tol=1e-3)
    _, it_m, _ = orc.mg_solve(p, h, w, g, y0, 400, orc.make_mg(**MG), tol=1e-3)
    assert 0 < it_m * 4 <= it_b, (it_m, it_b)
