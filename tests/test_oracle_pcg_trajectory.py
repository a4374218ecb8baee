"""Pin of the oracle's PCG iterates at a fixed iteration count (Sec. 2.6,
Eq. 42 and the block preconditioner stated there).

The GPU solve is compared with the oracle after 1, 2 or 30 iterations, so the
iterates themselves -- not only the limit -- are the contract.  A converged
solve, a monotone A-norm error or exactness without the prior hold for any
symmetric positive definite preconditioner; this test fixes which one.

Preconditioned CG started at zero has a closed characterisation: its k-th
iterate is the A-norm minimiser of the error over the preconditioned Krylov
space span{M^-1 b, (M^-1 A) M^-1 b, ..., (M^-1 A)^(k-1) M^-1 b}.  Here A and M
are built densely from the materialised finite-difference matrix G:

    A = H + lambda (x) G'WG              (the Newton system)
    M = H + lambda (x) (G'WG o I)        (the paper's block preconditioner)

and the minimiser is found by a Galerkin projection onto an orthonormal basis
of that space (a dense least-squares statement, not the CG recurrence).
"""
import numpy as np
import pytest

from paper_2102_01604_gb300 import phantom
from test_oracle_prior import dense_G

LAM = (1000.0, 700.0, 300.0, 200.0)   # prior comparable with H, so M depends on it
VX = (0.8, 1.3, 2.0)


def _system(orc, shape, seed=0):
    prot = phantom.protocol()
    ph = phantom.phantom(shape, seed=seed)
    p0 = orc.make_problem(prot, shape, vx=VX)
    s = orc.forward(p0, ph["y"], ph["b1p"], ph["b1m"])
    prot["sigma2"] = phantom.noise_sigma2(s, prot)
    x = phantom.rician(s, prot, seed=seed + 1)
    p = orc.make_problem(prot, shape, vx=VX, lam=LAM, eps=1e-2)
    rng = np.random.default_rng(seed + 2)
    y = ph["y"] + 0.2 * rng.standard_normal(ph["y"].shape)
    _, g, h = orc.grad_hess(p, x, y, ph["b1p"], ph["b1m"])
    _, w = orc.jtv(p, y)
    return p, g, h, w


def _blocks(h, K, N):
    """H as a dense (K N) x (K N) matrix from its packed upper triangle."""
    H = np.zeros((K * N, K * N))
    idx = np.arange(N)
    t = 0
    for a in range(K):
        for b in range(a, K):
            H[a * N + idx, b * N + idx] = h[t]
            H[b * N + idx, a * N + idx] = h[t]
            t += 1
    return H


def _dense_system(p, h, w, shape, lam=LAM, vx=VX, diag_of=None):
    """A and M densely.  `diag_of` replaces diag(G'WG) in M (used to check
    that the pin tells plausible mistakes apart)."""
    K, N = p.n_maps, int(np.prod(shape))
    G = dense_G(shape, vx)
    GWG = G.T @ np.kron(np.diag(w), np.eye(6)) @ G
    L = np.diag(lam[:K])
    H = _blocks(h, K, N)
    A = H + np.kron(L, GWG)
    d = np.diag(GWG) if diag_of is None else diag_of
    M = H + np.kron(L, np.diag(d))
    return A, M


def _krylov_iterate(A, M, b, k):
    """argmin over x in span{(M^-1 A)^j M^-1 b, j < k} of |x - A^-1 b|_A."""
    v = np.linalg.solve(M, b)
    cols = []
    for _ in range(k):
        cols.append(v)
        v = np.linalg.solve(M, A @ v)
    Q, _ = np.linalg.qr(np.stack(cols, axis=1))
    c = np.linalg.solve(Q.T @ A @ Q, Q.T @ b)
    return Q @ c


@pytest.mark.parametrize("shape", [(3, 2, 2), (2, 3, 3), (4, 2, 1)])
def test_pcg_iterates_are_the_krylov_minimisers(orc, shape):
    p, g, h, w = _system(orc, shape)
    K, N = p.n_maps, int(np.prod(shape))
    A, M = _dense_system(p, h, w, shape)
    b = np.random.default_rng(7).standard_normal(K * N) * np.abs(g).mean()
    for k in range(1, 5):
        ref = _krylov_iterate(A, M, b, k)
        x, it, _ = orc.pcg(p, h, w, b.reshape(K, N), k)
        assert it == k
        err = np.abs(x.ravel() - ref).max() / np.abs(ref).max()
        assert err < 1e-9, (k, err)


def test_pin_tells_plausible_preconditioner_slips_apart(orc):
    """The Krylov iterates of three plausible wrong preconditioners (lambda_k
    left out, the 1/h^2 of the voxel size left out of diag(G'WG), the centre
    weight w_n left out of it) differ from the oracle's after two iterations
    by far more than the pin's tolerance, so a slip of either kind in the
    oracle would fail it."""
    shape = (3, 2, 2)
    p, g, h, w = _system(orc, shape)
    K, N = p.n_maps, int(np.prod(shape))
    G = dense_G(shape, VX)
    GWG = G.T @ np.kron(np.diag(w), np.eye(6)) @ G
    b = np.random.default_rng(7).standard_normal(K * N) * np.abs(g).mean()
    x, _, _ = orc.pcg(p, h, w, b.reshape(K, N), 2)
    G1 = dense_G(shape, (1.0, 1.0, 1.0))
    d_noh = np.diag(G1.T @ np.kron(np.diag(w), np.eye(6)) @ G1)
    A, _ = _dense_system(p, h, w, shape)
    # diag(G'WG)_n = sum_m (w_n + w_m) / h^2; sum_m 1 / h^2 = diag(G'G)_n / 2
    inv_h2 = np.diag(G.T @ G) / 2
    wrong = {
        "no lambda": _blocks(h, K, N) + np.kron(np.eye(K), np.diag(np.diag(GWG))),
        "no 1/h^2": _blocks(h, K, N) + np.kron(np.diag(LAM[:K]), np.diag(d_noh)),
        "no centre weight": _blocks(h, K, N)
        + np.kron(np.diag(LAM[:K]), np.diag(np.diag(GWG) - w * inv_h2)),
    }
    for name, Mw in wrong.items():
        alt = _krylov_iterate(A, Mw, b, 2)
        dif = np.abs(x.ravel() - alt).max() / np.abs(alt).max()
        assert dif > 1e-3, (name, dif)
