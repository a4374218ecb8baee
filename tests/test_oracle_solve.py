"""Pins of the oracle's Newton-system solve (Sec. 2.6, Eq. 42): PCG against a
dense factorisation of H + L built from a materialised G."""
import numpy as np
import pytest

from paper_2102_01604_gb300 import phantom
from test_oracle_prior import dense_G


def _system(orc, shape, lam=10.0, seed=0, eps=1e-2):
    prot = phantom.protocol()
    ph = phantom.phantom(shape, seed=seed)
    p0 = orc.make_problem(prot, shape)
    s = orc.forward(p0, ph["y"], ph["b1p"], ph["b1m"])
    prot["sigma2"] = phantom.noise_sigma2(s, prot)
    x = phantom.rician(s, prot, seed=seed + 1)
    p = orc.make_problem(prot, shape, lam=lam, eps=eps)
    y = ph["y"] + 0.1 * np.random.default_rng(seed).standard_normal(ph["y"].shape)
    _, g, h = orc.grad_hess(p, x, y, ph["b1p"], ph["b1m"])
    _, w = orc.jtv(p, y)
    return p, g, h, w, y


def _dense(p, h, w, shape):
    K, N = p.n_maps, int(np.prod(shape))
    G = dense_G(shape, (p.vx[0], p.vx[1], p.vx[2]))
    GWG = G.T @ np.kron(np.diag(w), np.eye(6)) @ G
    A = np.kron(np.diag([p.lam[k] for k in range(K)]), GWG)
    t = 0
    for a in range(K):
        for b in range(a, K):
            A[a * N + np.arange(N), b * N + np.arange(N)] += h[t]
            if a != b:
                A[b * N + np.arange(N), a * N + np.arange(N)] += h[t]
            t += 1
    return A, GWG


@pytest.mark.parametrize("shape", [(3, 2, 2), (4, 3, 1), (2, 2, 3)])
def test_pcg_matches_dense_solve(orc, shape):
    p, g, h, w, y = _system(orc, shape)
    K, N = p.n_maps, int(np.prod(shape))
    A, GWG = _dense(p, h, w, shape)
    lamv = np.repeat([p.lam[k] for k in range(K)], N)
    b = g.ravel() + lamv * np.kron(np.eye(K), GWG) @ y.ravel()
    ref = np.linalg.solve(A, b)
    delta, it, resid = orc.solve(p, h, w, g, y, iters=4 * K * N)
    assert np.allclose(delta.ravel(), ref, rtol=1e-8, atol=1e-10 * np.abs(ref).max())
    assert resid[-1] <= 1e-8 * resid[0]


def test_pcg_tolerance_stops_early(orc):
    p, g, h, w, y = _system(orc, (4, 4, 3))
    delta, it, resid = orc.solve(p, h, w, g, y, iters=500, tol=1e-3)
    assert it < 500
    assert resid[-1] <= 1e-3 * resid[0]
    assert resid[-2] > 1e-3 * resid[0]


def test_block_preconditioner_is_exact_without_prior(orc):
    """With lambda = 0 the system is block diagonal and equals its
    preconditioner, so one PCG iteration is the exact Newton step."""
    p, g, h, w, y = _system(orc, (3, 3, 2), lam=0.0)
    K, N = p.n_maps, 18
    delta, it, _ = orc.solve(p, h, w, g, y, iters=1)
    for n in range(N):
        M = np.zeros((K, K))
        t = 0
        for a in range(K):
            for b in range(a, K):
                M[a, b] = M[b, a] = h[t, n]
                t += 1
        assert np.allclose(delta[:, n], np.linalg.solve(M, g[:, n]), rtol=1e-9)


def test_pcg_energy_error_decreases(orc):
    """CG minimises the A-norm of the error over growing Krylov spaces, so it
    is non-increasing from one iteration to the next."""
    shape = (3, 3, 2)
    p, g, h, w, y = _system(orc, shape)
    K, N = p.n_maps, 18
    A, _ = _dense(p, h, w, shape)
    b = np.random.default_rng(4).standard_normal(K * N)
    xs = np.linalg.solve(A, b)
    errs = []
    for it in range(1, 25):
        x, _, _ = orc.pcg(p, h, w, b.reshape(K, N), it)
        e = x.ravel() - xs
        errs.append(e @ A @ e)
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-9) + 1e-20 for i in range(len(errs) - 1))
