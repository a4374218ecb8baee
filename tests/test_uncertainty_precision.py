"""The reading behind the float32 uncertainty pass (Eq. 43 on the GPU).

The pass inverts each preconditioner block M = H_n + diag(lambda_k d_n) from
the float32 Cholesky factor of the equilibrated block A = S M S (S the inverse
square roots of M's diagonal), and falls back to float64 when A's smallest
pivot is below 1e-2.  These checks run the same arithmetic in numpy float32
on the oracle's blocks at the end of an oracle fit of the seeded phantom, and
compare with the float64 inverse: the phantom's equilibrated blocks stay well
conditioned (no fallback), the float32 variances meet the 1e-5 bound of the
GPU parity tests, and a block with two maps correlated at 0.999 does need the
fallback.  CPU only.
"""
import numpy as np

import oracle as orc
from cases import dataset


def _blocks(h, dn, lam):
    K = {6: 3, 10: 4}[h.shape[0]]
    N = h.shape[1]
    M = np.zeros((N, K, K), dtype=np.float64)
    t = 0
    for a in range(K):
        for b in range(a, K):
            M[:, a, b] = M[:, b, a] = h[t]
            t += 1
    for a in range(K):
        M[:, a, a] += lam[a] * dn
    return M


def _f32_equilibrated(M):
    """(variances, smallest pivot) per block, in float32 as the GPU pass."""
    M = M.astype(np.float32)
    s = (1.0 / np.sqrt(np.einsum("nii->ni", M))).astype(np.float32)
    A = (M * s[:, :, None] * s[:, None, :]).astype(np.float32)
    L = np.linalg.cholesky(A)
    piv = np.einsum("nii->ni", L).astype(np.float64) ** 2
    Li = np.linalg.inv(L).astype(np.float32)
    var = np.einsum("nji,nji->ni", Li, Li) * s * s
    return var.astype(np.float64), piv.min(axis=1)


def test_phantom_blocks_take_the_float32_path_within_1e5():
    d = dataset((24, 20, 10), seed=5)
    po = orc.make_problem(d["prot"], d["shape"])
    ref = orc.fit(po, d["x"], None, d["b1p"], d["b1m"], gn_iters=4, cg_iters=20)
    y = ref["y"].astype(np.float32)
    _, _, h = orc.grad_hess(po, d["x"], y, d["b1p"], d["b1m"])
    _, w = orc.jtv(po, y)
    h = h.astype(np.float32).astype(np.float64)
    dn = orc.membrane_diag(po, w.astype(np.float32))
    M = _blocks(h, dn, [10.0] * 4)
    v64 = np.einsum("nii->ni", np.linalg.inv(M))
    v32, pmin = _f32_equilibrated(M)
    assert pmin.min() > 1e-2                    # no block needs the float64 path
    assert np.max(np.abs(v32 - v64) / v64) < 1e-5
    # the oracle's own variances are the float64 inverse of the same blocks
    var_o, _, _, _ = orc.uncertainty(po, h, w.astype(np.float32))
    np.testing.assert_allclose(var_o.T, v64, rtol=1e-9)


def test_correlated_block_needs_the_float64_path():
    rng = np.random.default_rng(3)
    a, b = 10.0 ** rng.uniform(2, 5, 2)
    M = np.diag([a, b, 3e3, 4e2])
    M[0, 1] = M[1, 0] = 0.999 * np.sqrt(a * b)
    v64 = np.einsum("nii->ni", np.linalg.inv(M[None]))
    v32, pmin = _f32_equilibrated(M[None])
    assert pmin[0] < 1e-2                       # declined by the float32 path
    assert np.max(np.abs(v32 - v64) / v64) > 1e-5  # where float32 alone would miss the bound
