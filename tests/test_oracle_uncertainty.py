"""Pins of the oracle's Laplace uncertainty (Sec. 3.6, Eqs. 43-47)."""
import numpy as np
import pytest

from test_oracle_solve import _system


def test_variance_is_diagonal_of_block_inverse(orc):
    p, g, h, w, y = _system(orc, (3, 2, 2))
    K, N = p.n_maps, 12
    d = orc.membrane_diag(p, w)
    var, logdet, mom, st = orc.uncertainty(p, h, w, y)
    assert st == 0
    for n in range(N):
        M = np.zeros((K, K))
        t = 0
        for a in range(K):
            for b in range(a, K):
                M[a, b] = M[b, a] = h[t, n]
                t += 1
        M += np.diag([p.lam[k] * d[n] for k in range(K)])
        inv = np.linalg.inv(M)
        assert np.allclose(var[:, n], np.diag(inv), rtol=1e-10)
        sign, ld = np.linalg.slogdet(inv)
        assert sign > 0 and logdet[n] == pytest.approx(ld, rel=1e-10, abs=1e-10)


def test_lognormal_moments_match_monte_carlo(orc):
    """E and V of r1 = exp(log R1) and t1 = 1/r1 when log R1 ~ Normal(y, var)."""
    p, g, h, w, y = _system(orc, (2, 2, 1))
    var, _, mom, _ = orc.uncertainty(p, h, w, y)
    rng = np.random.default_rng(0)
    for n in range(4):
        # widen the variance so the Monte-Carlo test has something to measure
        v = var[1, n]
        smp = y[1, n] + np.sqrt(v) * rng.standard_normal(2_000_000)
        r1, t1 = np.exp(smp), np.exp(-smp)
        se = lambda a: np.std(a) / np.sqrt(a.size)
        assert abs(mom[0, n] - r1.mean()) < 5 * se(r1) + 1e-12
        assert abs(mom[2, n] - t1.mean()) < 5 * se(t1) + 1e-12
        assert mom[1, n] == pytest.approx(r1.var(), rel=0.02, abs=1e-14)
        assert mom[3, n] == pytest.approx(t1.var(), rel=0.02, abs=1e-14)


def test_lognormal_moments_wide_variance(orc):
    """Same check with a posterior variance (0.1 to 0.4) large enough that the
    log-normal correction is far from 1: H diagonal, no prior."""
    p, g, h, w, y = _system(orc, (2, 1, 1), lam=0.0)
    h = np.zeros_like(h)
    for k, t in enumerate((0, 4, 7, 9)):
        h[t] = [10.0, 2.5]
    var, _, mom, st = orc.uncertainty(p, h, w, y)
    assert st == 0
    assert np.allclose(var, [[0.1, 0.4]] * 4)
    rng = np.random.default_rng(1)
    for n in range(2):
        smp = y[1, n] + np.sqrt(var[1, n]) * rng.standard_normal(4_000_000)
        r1, t1 = np.exp(smp), np.exp(-smp)
        assert mom[0, n] == pytest.approx(r1.mean(), rel=0.003)
        assert mom[1, n] == pytest.approx(r1.var(), rel=0.03)
        assert mom[2, n] == pytest.approx(t1.mean(), rel=0.003)
        assert mom[3, n] == pytest.approx(t1.var(), rel=0.03)
