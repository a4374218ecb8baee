"""Pins of the oracle's spatial projection (Sec. 2.4): reslicing Psi (pull),
its adjoint (push), the projected likelihood with its block-diagonal
majoriser, and the projected fit.

Each property is fixed by something other than the oracle's own formulas:
index permutations for integer shifts and 90-degree rotations, exactness of
trilinear interpolation on affine functions, the adjoint identity, the plain
(unprojected) likelihood and fit for identity reslicing, finite differences,
and the Loewner order against a materialised Psi' H Psi."""
import numpy as np
import pytest

import oracle as orc
from cases import round_protocol
from paper_2102_01604_gb300 import phantom

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _rot(ax, deg):
    t = np.deg2rad(deg)
    c, s = np.cos(t), np.sin(t)
    R = np.eye(3)
    i, j = [(1, 2), (0, 2), (0, 1)][ax]
    R[i, i], R[i, j], R[j, i], R[j, j] = c, -s, s, c
    return R


def _affine(R, t):
    A = np.eye(4)
    A[:3, :3] = R
    A[:3, 3] = t
    return A


def _problem(shape, contrasts=("PDw", "T1w", "MTw"), echoes=(3, 3, 2), lam=10.0, precond=0):
    prot = round_protocol(phantom.protocol(contrasts, echoes))
    return orc.make_problem(prot, shape, lam=lam, precond=precond), prot


def _maps(rng, K, N):
    base = np.array([np.log(3000.0), np.log(1.0), np.log(25.0), np.log(0.01 / 0.99)])[:K]
    return base[:, None] + 0.1 * rng.standard_normal((K, N))


def test_integer_shift_is_an_index_shift():
    p, _ = _problem((7, 6, 5))
    rng = np.random.default_rng(0)
    y = rng.standard_normal((2, 7 * 6 * 5))
    dims, t = (6, 6, 5), np.array([2.0, -1.0, 1.0])
    out, inside = orc.pull(p, dims, _affine(np.eye(3), t), y)
    Y = y.reshape(2, 5, 6, 7)
    O = out.reshape(2, 5, 6, 6)
    I = inside.reshape(5, 6, 6)
    for k in range(5):
        for j in range(6):
            for i in range(6):
                x, yy, z = i + 2, j - 1, k + 1
                ok = 0 <= x < 7 and 0 <= yy < 6 and 0 <= z < 5
                assert I[k, j, i] == ok
                expect = Y[:, z, yy, x] if ok else np.zeros(2)
                assert np.array_equal(O[:, k, j, i], expect)


def test_quarter_turn_is_a_permutation():
    nx, ny, nz = 5, 4, 3
    p, _ = _problem((nx, ny, nz))
    mx, my, mz = ny, nx, nz                     # r_x = j, r_y = mx - 1 - i, r_z = k
    A = np.array([[0.0, 1.0, 0.0, 0.0], [-1.0, 0.0, 0.0, mx - 1.0], [0.0, 0.0, 1.0, 0.0]])
    y = np.arange(nx * ny * nz, dtype=np.float64)[None]
    out, inside = orc.pull(p, (mx, my, mz), A, y)
    assert inside.all()
    Y = y.reshape(nz, ny, nx)
    O = out.reshape(mz, my, mx)
    for k in range(mz):
        for j in range(my):
            for i in range(mx):
                assert O[k, j, i] == Y[k, mx - 1 - i, j]
    # the push of a permutation is the inverse permutation
    back = orc.push(p, (mx, my, mz), A, out)
    assert np.array_equal(back, y)


def test_interpolation_reproduces_affine_functions():
    shape = (9, 8, 7)
    p, _ = _problem(shape)
    g = np.stack(np.meshgrid(np.arange(9), np.arange(8), np.arange(7), indexing="ij"), -1)
    pos = g.transpose(2, 1, 0, 3).reshape(-1, 3).astype(np.float64)   # voxel n -> (x, y, z)
    a = np.array([[0.3, -0.7, 1.1], [2.0, 0.5, -0.25]])
    b = np.array([0.4, -3.0])
    y = a @ pos.T + b[:, None]
    A = _affine(_rot(2, 11.0) @ _rot(0, -7.0) * 0.93, [1.3, 0.6, 0.9])
    dims = (8, 8, 6)
    out, inside = orc.pull(p, dims, A, y)
    assert 0.3 < inside.mean() < 1.0
    gm = np.stack(np.meshgrid(np.arange(8), np.arange(8), np.arange(6), indexing="ij"), -1)
    m = gm.transpose(2, 1, 0, 3).reshape(-1, 3).astype(np.float64)
    r = m @ A[:3, :3].T + A[:3, 3]
    expect = a @ r.T + b[:, None]
    np.testing.assert_allclose(out[:, inside], expect[:, inside], rtol=0, atol=1e-12)
    assert np.all(out[:, ~inside] == 0.0)
    inside_expect = np.all((r >= 0) & (r <= np.array(shape) - 1), axis=1)
    assert np.array_equal(inside, inside_expect)


def test_push_is_the_adjoint_of_pull():
    p, _ = _problem((8, 7, 6))
    rng = np.random.default_rng(1)
    A = _affine(_rot(1, 23.0) @ np.diag([1.1, 0.9, 1.2]), [2.1, -0.4, 0.7])
    dims = (9, 6, 7)
    u = rng.standard_normal((3, 8 * 7 * 6))
    v = rng.standard_normal((3, 9 * 6 * 7))
    pu, _ = orc.pull(p, dims, A, u)
    ptv = orc.push(p, dims, A, v)
    lhs, rhs = np.sum(pu * v), np.sum(u * ptv)
    assert abs(lhs - rhs) <= 1e-12 * (np.abs(pu * v).sum())


def _split(x, prot):
    out, i = [], 0
    for e in prot["n_echoes"]:
        out.append(x[i:i + e])
        i += e
    return out


def test_identity_reslicing_gives_the_plain_likelihood():
    shape = (6, 5, 4)
    N = 120
    p, prot = _problem(shape)
    rng = np.random.default_rng(2)
    y = _maps(rng, 4, N)
    b1p = 1 + 0.1 * rng.standard_normal(N)
    b1m = 1 + 0.05 * rng.standard_normal((3, N))
    s = orc.forward(p, y + 0.05 * rng.standard_normal(y.shape), b1p, b1m)
    x = s + 5.0 * rng.standard_normal(s.shape)
    nll, g, h = orc.grad_hess(p, x, y, b1p, b1m)
    q = orc.make_projection([shape] * 3, [np.eye(4)] * 3)
    nll2, g2, h2 = orc.grad_hess_proj(p, q, _split(x, prot), y, [b1p] * 3, list(b1m))
    assert abs(nll2 - nll) <= 1e-12 * nll
    np.testing.assert_allclose(g2, g, rtol=1e-12, atol=1e-12 * np.abs(g).max())
    np.testing.assert_allclose(h2, h, rtol=1e-12, atol=1e-12 * np.abs(h).max())


def _moved_case(seed, shape=(7, 6, 5), echoes=(3, 3, 2), lam=10.0, precond=0):
    """Three contrasts; the T1w and MTw scans moved (rotation + translation,
    MTw on a coarser grid)."""
    p, prot = _problem(shape, echoes=echoes, lam=lam, precond=precond)
    rng = np.random.default_rng(seed)
    N = int(np.prod(shape))
    dims = [shape, (6, 6, 5), (5, 5, 4)]
    affs = [np.eye(4), _affine(_rot(2, 8.0), [0.6, 0.3, 0.2]),
            _affine(_rot(0, 5.0) @ np.diag([1.2, 1.2, 1.25]), [0.4, 0.3, 0.2])]
    q = orc.make_projection(dims, affs)
    y_true = _maps(rng, 4, N)
    xs = []
    for c in range(3):
        yc, inside = orc.pull(p, dims[c], affs[c], y_true)
        sub = orc.make_problem({k: (v[c:c + 1] if k != "te" else
                                    v[sum(prot["n_echoes"][:c]):sum(prot["n_echoes"][:c + 1])])
                                for k, v in prot.items()}, dims[c], n_maps=4)
        sc = orc.forward(sub, yc)
        xs.append(sc + np.sqrt(prot["sigma2"][c]) * rng.standard_normal(sc.shape))
    return p, prot, q, dims, affs, xs, y_true, rng


def test_projected_gradient_matches_finite_differences():
    p, prot, q, dims, affs, xs, y_true, rng = _moved_case(3)
    y = y_true + 0.05 * rng.standard_normal(y_true.shape)
    nll, g, _ = orc.grad_hess_proj(p, q, xs, y)
    N = y.shape[1]
    for k, n in [(0, 3), (1, 40), (2, 77), (3, 101), (1, 150), (0, N - 1)]:
        hstep = 1e-6
        yp, ym = y.copy(), y.copy()
        yp[k, n] += hstep
        ym[k, n] -= hstep
        fd = (orc.grad_hess_proj(p, q, xs, yp)[0] - orc.grad_hess_proj(p, q, xs, ym)[0]) / (2 * hstep)
        assert abs(fd - g[k, n]) <= 1e-5 * max(1.0, abs(g[k, n])), (k, n, fd, g[k, n])


@pytest.mark.parametrize("precond", [0, 2])
def test_pushed_hessian_majorises_psi_t_h_psi(precond):
    shape = (4, 4, 3)
    p, prot = _problem(shape, contrasts=("MTw",), echoes=(3,), precond=precond)
    rng = np.random.default_rng(4)
    N, K, T = 48, 4, 10
    dims = (4, 3, 3)
    A = _affine(_rot(2, 17.0) @ np.diag([0.9, 1.1, 1.0]), [0.8, 0.5, 0.4])
    q = orc.make_projection([dims], [A])
    y = _maps(rng, K, N)
    yc, inside = orc.pull(p, dims, A, y)
    M = int(np.prod(dims))
    sub = orc.make_problem(prot, dims, precond=precond)
    x = orc.forward(sub, yc) * (1 + 0.1 * rng.standard_normal((3, M)))
    _, g_c, h_c = orc.grad_hess(sub, x, yc)
    g_c[:, ~inside] = 0.0
    h_c[:, ~inside] = 0.0
    nll, g, h = orc.grad_hess_proj(p, q, [x], y)
    # Psi materialised column by column
    Psi = np.zeros((M, N))
    for n in range(N):
        e = np.zeros((1, N))
        e[0, n] = 1.0
        Psi[:, n] = orc.pull(p, dims, A, e)[0][0]
    np.testing.assert_allclose(g, (Psi.T @ g_c.T).T, rtol=1e-12, atol=1e-12 * np.abs(g).max())
    tri = [(a, b) for a in range(K) for b in range(a, K)]

    def blocks(hh, n_vox):
        B = np.zeros((n_vox, K, K))
        for t, (a, b) in enumerate(tri):
            B[:, a, b] = hh[t]
            B[:, b, a] = hh[t]
        return B
    Hc = blocks(h_c, M)
    # Q = (Psi (x) I)' blockdiag(Hc) (Psi (x) I), voxel-major ordering
    PsiK = np.kron(Psi, np.eye(K))
    BD = np.zeros((M * K, M * K))
    for m in range(M):
        BD[m * K:(m + 1) * K, m * K:(m + 1) * K] = Hc[m]
    Q = PsiK.T @ BD @ PsiK
    B = np.zeros((N * K, N * K))
    Hr = blocks(h, N)
    for n in range(N):
        B[n * K:(n + 1) * K, n * K:(n + 1) * K] = Hr[n]
    ev = np.linalg.eigvalsh(B - Q)
    assert ev.min() >= -1e-9 * np.abs(ev).max()
    assert ev.max() > 0                       # a real bound, not an equality


def test_identity_reslicing_gives_the_plain_fit():
    shape = (6, 5, 4)
    p, prot = _problem(shape)
    rng = np.random.default_rng(5)
    N = 120
    y = _maps(rng, 4, N)
    s = orc.forward(p, y)
    x = s * (1 + 0.05 * rng.standard_normal(s.shape))
    ref = orc.fit(p, x, gn_iters=4, cg_iters=20)
    q = orc.make_projection([shape] * 3, [np.eye(4)] * 3)
    out = orc.fit_proj(p, q, _split(x, prot), gn_iters=4, cg_iters=20)
    np.testing.assert_allclose(out["F"], ref["F"], rtol=1e-11)
    np.testing.assert_allclose(out["y"], ref["y"], rtol=0, atol=1e-9)


def test_projected_fit_lowers_the_objective():
    p, prot, q, dims, affs, xs, y_true, rng = _moved_case(6, lam=1.0)
    out = orc.fit_proj(p, q, xs, gn_iters=6, cg_iters=40)
    F = out["F"]
    assert out["iters"] == 6
    assert F[-1] < 0.5 * F[0]
    # with the motion modelled the fit lands near the truth; reslicing the
    # moved scans away (identity) fits them far worse
    wrong = orc.fit_proj(p, orc.make_projection(dims, [np.eye(4)] * 3), xs, gn_iters=6, cg_iters=40)
    assert wrong["F"][-1] > 1.5 * F[-1]
