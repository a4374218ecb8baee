"""Pins of the oracle's JTV prior and weighted membrane operator (Sec. 2.5,
Eqs. 38-40).

The oracle applies G'WG as a 6-neighbour stencil; here the finite-difference
matrix G (forward and backward differences about every voxel, out-of-volume
neighbours dropped) is materialised densely and the products are formed with
plain matrix algebra.
"""
import math

import numpy as np
import pytest

from paper_2102_01604_gb300 import phantom

SHAPES = [(3, 2, 2), (5, 3, 2), (1, 4, 3), (4, 1, 1), (2, 2, 5)]


def dense_G(shape, vx):
    """G in R^{6N x N}: row (n, d) = (e_m - e_n)/h_d for the d-th neighbour m of
    n (order -x, +x, -y, +y, -z, +z), or zero when m is outside the volume."""
    nx, ny, nz = shape
    N = nx * ny * nz
    G = np.zeros((6 * N, N))
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                n = x + nx * (y + ny * z)
                offs = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
                for d, (dx, dy, dz) in enumerate(offs):
                    xx, yy, zz = x + dx, y + dy, z + dz
                    if 0 <= xx < nx and 0 <= yy < ny and 0 <= zz < nz:
                        m = xx + nx * (yy + ny * zz)
                        h = vx[d // 2]
                        G[6 * n + d, m] += 1.0 / h
                        G[6 * n + d, n] -= 1.0 / h
    return G


def _setup(orc, shape, vx=(1.0, 1.0, 1.0), lam=(10.0, 7.0, 3.0, 2.0), seed=0):
    prot = phantom.protocol()
    p = orc.make_problem(prot, shape, vx=vx, lam=lam, eps=1e-2)
    rng = np.random.default_rng(seed)
    N = int(np.prod(shape))
    y = rng.standard_normal((4, N)) * 0.3
    return p, y, N


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("vx", [(1.0, 1.0, 1.0), (0.8, 1.3, 2.0)])
def test_jtv_weights_match_dense_G(orc, shape, vx):
    lam = (10.0, 7.0, 3.0, 2.0)
    p, y, N = _setup(orc, shape, vx, lam)
    G = dense_G(shape, vx)
    Gy = [(G @ y[k]).reshape(N, 6) for k in range(4)]
    u = sum(lam[k] * np.sum(Gy[k] ** 2, axis=1) for k in range(4))
    e, w = orc.jtv(p, y)
    assert np.allclose(w, 1.0 / np.sqrt(u + p.eps ** 2), rtol=1e-13)
    assert e == pytest.approx(np.sum(np.sqrt(u + p.eps ** 2)), rel=1e-13)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("vx", [(1.0, 1.0, 1.0), (0.8, 1.3, 2.0)])
def test_membrane_matches_dense_GtWG(orc, shape, vx):
    lam = (10.0, 7.0, 3.0, 2.0)
    p, y, N = _setup(orc, shape, vx, lam)
    G = dense_G(shape, vx)
    w = np.random.default_rng(1).uniform(0.1, 5.0, N)
    W = np.kron(np.diag(w), np.eye(6))
    A = G.T @ W @ G
    v = np.random.default_rng(2).standard_normal((4, N))
    out = orc.membrane(p, w, v)
    for k in range(4):
        assert np.allclose(out[k], lam[k] * (A @ v[k]), rtol=1e-12, atol=1e-12)
    assert np.allclose(orc.membrane_diag(p, w), np.diag(A), rtol=1e-13)
    # Neumann boundary: constants are in the null space (L 1 = 0)
    assert np.allclose(orc.membrane(p, w, np.ones((4, N))), 0.0, atol=1e-12)


def test_quadratic_form_is_half_weighted_jtv(orc):
    """(1/2) y'Ly equals (1/2) sum_n w_n sum_k lambda_k |G_n y_k|^2 (Eq. 39)."""
    shape = (4, 3, 2)
    lam = (10.0, 7.0, 3.0, 2.0)
    p, y, N = _setup(orc, shape, lam=lam)
    _, w = orc.jtv(p, y)
    Ly = orc.membrane(p, w, y)
    G = dense_G(shape, (1, 1, 1))
    u = sum(lam[k] * np.sum(((G @ y[k]).reshape(N, 6)) ** 2, axis=1) for k in range(4))
    assert 0.5 * np.sum(y * Ly) == pytest.approx(0.5 * np.sum(w * u), rel=1e-12)


def test_weights_minimise_the_irls_bound(orc):
    """At fixed y, w_n = (u_n + eps^2)^-1/2 minimises 1/(2w) + w (u + eps^2)/2 and
    the bound is tight there (Eq. 39)."""
    shape = (3, 3, 2)
    p, y, N = _setup(orc, shape)
    e, w = orc.jtv(p, y)
    v = (1.0 / w) ** 2                     # u + eps^2
    bound = lambda ww: np.sum(1.0 / (2 * ww) + ww * v / 2)
    assert bound(w) == pytest.approx(e, rel=1e-13)
    for f in (0.5, 0.9, 1.1, 2.0):
        assert bound(w * f) > bound(w)
