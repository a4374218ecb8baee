"""Pins of the oracle's signal derivatives, likelihood gradient and approximate
Hessian (Eqs. 6, 24, 25, 27-34).

Everything here is checked against finite differences of the signal or of the
likelihood, or against a Jacobian assembled from finite differences of the
forward images, never against a retyped formula.
"""
import math

import numpy as np
import pytest

from paper_2102_01604_gb300 import phantom


def _samples():
    rng = np.random.default_rng(11)
    out = []
    # phantom-like voxels
    for _ in range(6):
        y = np.array([math.log(rng.uniform(2000, 4000)), math.log(rng.uniform(0.5, 1.5)),
                      math.log(rng.uniform(10, 40)),
                      math.log((d := rng.uniform(0.002, 0.02)) / (1 - d))])
        out.append((y, math.radians(rng.choice([6.0, 21.0])), 0.025,
                    0.0023 * rng.integers(1, 9), int(rng.integers(0, 2)),
                    rng.uniform(0.8, 1.2), rng.uniform(0.9, 1.1)))
    # wide-range voxels (the convergence-experiment sampler)
    for prot, y in phantom.single_voxel_protocols(6, seed=5):
        out.append((y, prot["alpha"][2], prot["tr"][2], prot["te"][10], 1, 1.0, 1.0))
        out.append((y, prot["alpha"][0], prot["tr"][0], prot["te"][0], 0, 1.0, 1.0))
    return out


SAMPLES = _samples()


@pytest.mark.parametrize("k", range(len(SAMPLES)))
def test_gradient_matches_central_differences(orc, k):
    y, al, tr, te, mt, bp, bm = SAMPLES[k]
    s, ds, _ = orc.signal_jet(y, al, tr, te, mt, bp, bm)
    h = 1e-6
    for j in range(4):
        e = np.zeros(4); e[j] = h
        fd = (orc.signal(y + e, al, tr, te, mt, bp, bm)
              - orc.signal(y - e, al, tr, te, mt, bp, bm)) / (2 * h)
        assert abs(ds[j] - fd) <= 1e-7 * (abs(s) + abs(ds[j])) + 1e-300, (j, ds[j], fd)
    if not mt:
        assert ds[3] == 0.0


@pytest.mark.parametrize("k", range(len(SAMPLES)))
def test_hessian_matches_second_differences(orc, k):
    y, al, tr, te, mt, bp, bm = SAMPLES[k]
    s, ds, d2s = orc.signal_jet(y, al, tr, te, mt, bp, bm)
    # step shrunk where the log-derivatives are large, so that the truncation
    # error (~ h^2 q^4 s) stays below the tolerance
    qmax = float(np.abs(ds).max() / abs(s)) if s != 0 else 1.0
    h = 1e-4 / max(1.0, qmax)
    f = lambda v: orc.signal(v, al, tr, te, mt, bp, bm)
    scale = abs(s) + np.abs(ds).max() + np.abs(d2s).max()
    for i in range(4):
        for j in range(4):
            ei = np.zeros(4); ei[i] = h
            ej = np.zeros(4); ej[j] = h
            if i == j:
                fd = (f(y + ei) - 2 * f(y) + f(y - ei)) / h ** 2
            else:
                fd = (f(y + ei + ej) - f(y + ei - ej) - f(y - ei + ej) + f(y - ei - ej)) / (4 * h * h)
            assert abs(d2s[i, j] - fd) <= 2e-6 * scale, (i, j, d2s[i, j], fd)


def _problem(orc, shape=(3, 2, 2), precond=0, seed=1, noise=True):
    prot = phantom.protocol()
    ph = phantom.phantom(shape, seed=seed)
    p0 = orc.make_problem(prot, shape)
    s = orc.forward(p0, ph["y"], ph["b1p"], ph["b1m"])
    prot["sigma2"] = phantom.noise_sigma2(s, prot)
    p = orc.make_problem(prot, shape, precond=precond)
    rho = np.zeros_like(s)
    if noise:
        rho = np.random.default_rng(seed + 100).standard_normal(s.shape) * 15.0
    return p, prot, ph, s, s + rho, rho


def test_nll_equals_planted_residuals(orc):
    p, prot, ph, s, x, rho = _problem(orc)
    nll, _, _ = orc.grad_hess(p, x, ph["y"], ph["b1p"], ph["b1m"])
    i, ref = 0, 0.0
    for c, ne in enumerate(prot["n_echoes"]):
        ref += np.sum(rho[i:i + ne] ** 2) / (2 * prot["sigma2"][c])
        i += ne
    assert nll == pytest.approx(ref, rel=1e-10)


def test_gradient_is_derivative_of_nll(orc):
    p, prot, ph, s, x, rho = _problem(orc)
    y = ph["y"] + 0.05          # away from the truth
    _, g, _ = orc.grad_hess(p, x, y, ph["b1p"], ph["b1m"])
    h = 1e-6
    for n in (0, 5, 11):
        for k in range(4):
            yp, ym = y.copy(), y.copy()
            yp[k, n] += h
            ym[k, n] -= h
            fp, _, _ = orc.grad_hess(p, x, yp, ph["b1p"], ph["b1m"])
            fm, _, _ = orc.grad_hess(p, x, ym, ph["b1p"], ph["b1m"])
            fd = (fp - fm) / (2 * h)
            assert g[k, n] == pytest.approx(fd, rel=1e-5, abs=1e-6 * np.abs(g).max())


def _unpack(h, K, n):
    M = np.zeros((K, K))
    t = 0
    for a in range(K):
        for b in range(a, K):
            M[a, b] = M[b, a] = h[t, n]
            t += 1
    return M


def _fd_jacobian(orc, p, y, b1p, b1m, n, hstep=1e-6):
    """d(images at voxel n)/d(y[:, n]) by central differences of orc_forward."""
    K = p.n_maps
    cols = []
    for k in range(K):
        yp, ym = y.copy(), y.copy()
        yp[k, n] += hstep
        ym[k, n] -= hstep
        cols.append((orc.forward(p, yp, b1p, b1m)[:, n] - orc.forward(p, ym, b1p, b1m)[:, n])
                    / (2 * hstep))
    return np.stack(cols, axis=1)                        # [I, K]


def _fd_second(orc, p, y, b1p, b1m, n, hstep=1e-4):
    """d2(images at voxel n)/dy_k dy_j by second differences of orc_forward."""
    K = p.n_maps
    out = np.zeros((p.n_contrasts and sum(p.n_echoes[c] for c in range(p.n_contrasts)), K, K))
    f = lambda v: orc.forward(p, v, b1p, b1m)[:, n]
    for a in range(K):
        for b in range(K):
            def sh(da, db):
                v = y.copy()
                v[a, n] += da
                v[b, n] += db
                return f(v)
            if a == b:
                out[:, a, a] = (sh(hstep, 0) - 2 * f(y) + sh(-hstep, 0)) / hstep ** 2
            else:
                out[:, a, b] = (sh(hstep, hstep) - sh(hstep, -hstep) - sh(-hstep, hstep)
                                + sh(-hstep, -hstep)) / (4 * hstep ** 2)
    return out


def _inv_sigma2_per_image(prot):
    return np.concatenate([[1.0 / prot["sigma2"][c]] * ne for c, ne in enumerate(prot["n_echoes"])])


@pytest.mark.parametrize("precond", [0, 1, 2])
def test_approximate_hessian_structure(orc, precond):
    """h = J' S J + loading, with J and the second derivatives taken by finite
    differences of the forward images and the residuals from the data."""
    p, prot, ph, s, x, rho = _problem(orc, precond=precond)
    y = ph["y"] + 0.03
    _, _, h = orc.grad_hess(p, x, y, ph["b1p"], ph["b1m"])
    isg = _inv_sigma2_per_image(prot)
    r = orc.forward(p, y, ph["b1p"], ph["b1m"]) - x
    for n in (0, 6, 11):
        J = _fd_jacobian(orc, p, y, ph["b1p"], ph["b1m"], n)
        gn = J.T @ (isg[:, None] * J)
        d2 = _fd_second(orc, p, y, ph["b1p"], ph["b1m"], n)
        if precond == 0:
            load = np.einsum("i,i,ik->k", isg, np.abs(r[:, n]), np.abs(np.einsum("ikk->ik", d2)))
        elif precond == 1:
            load = np.einsum("i,i,ik->k", isg, np.abs(r[:, n]), np.abs(d2).sum(axis=2))
        else:
            load = np.zeros(4)
        ref = gn + np.diag(load)
        got = _unpack(h, 4, n)
        assert np.allclose(got, ref, rtol=1e-5, atol=1e-6 * np.abs(ref).max()), (got, ref)


def _true_hessian(orc, p, x, y, b1p, b1m, n, hstep=1e-6):
    """Hessian of the likelihood at voxel n by central differences of g."""
    K = p.n_maps
    H = np.zeros((K, K))
    for k in range(K):
        yp, ym = y.copy(), y.copy()
        yp[k, n] += hstep
        ym[k, n] -= hstep
        gp = orc.grad_hess(p, x, yp, b1p, b1m)[1][:, n]
        gm = orc.grad_hess(p, x, ym, b1p, b1m)[1][:, n]
        H[:, k] = (gp - gm) / (2 * hstep)
    return 0.5 * (H + H.T)


def _wide_voxels(orc, n_vox=40, seed=7):
    """Single voxels from the convergence sampler with Gaussian noise, sigma^2 = 1."""
    rng = np.random.default_rng(seed)
    for prot, y in phantom.single_voxel_protocols(n_vox, seed=seed):
        p = orc.make_problem(prot, (1, 1, 1), lam=0.0)
        s = orc.forward(p, y[:, None])
        x = s + rng.standard_normal(s.shape)
        yield prot, p, y, x


def test_approximate_hessian_positive_definite(orc):
    """Eq. 24 with either loading is positive definite (Sec. 2.3)."""
    checked = 0
    rng = np.random.default_rng(3)
    for prot, p, y, x in _wide_voxels(orc, 200):
        for precond in (0, 1):
            p.precond = precond
            yy = (y + rng.uniform(-1, 1, 4))[:, None]
            _, _, h = orc.grad_hess(p, x, yy)
            M = _unpack(h, 4, 0)
            if not np.all(np.isfinite(M)) or np.abs(M).max() == 0:
                continue
            ev = np.linalg.eigvalsh(M / np.abs(M).max())
            assert ev.min() > -1e-12
            checked += 1
    assert checked > 300


def test_rowsum_loading_majorises_true_hessian(orc):
    """The |H_f| 1 loading ("Proposed+") majorises the Hessian of the likelihood
    (Sec. 2.3, by diagonal dominance); the |H_f| diagonal loading need not."""
    frac_diag = []
    for prot, p, y, x in _wide_voxels(orc, 30, seed=9):
        yy = (y + 0.3)[:, None]
        Ht = _true_hessian(orc, p, x, yy, None, None, 0)
        p.precond = 1
        Pp = _unpack(orc.grad_hess(p, x, yy)[2], 4, 0)
        scale = np.abs(Pp).max() + np.abs(Ht).max()
        if not np.isfinite(scale) or scale == 0:
            continue
        assert np.linalg.eigvalsh(Pp - Ht).min() >= -1e-6 * scale
        p.precond = 0
        Pd = _unpack(orc.grad_hess(p, x, yy)[2], 4, 0)
        frac_diag.append(np.linalg.eigvalsh(Pd - Ht).min() >= -1e-6 * scale)
    assert len(frac_diag) > 20
