"""FP64 CPU oracle of the model-based multi-parameter-mapping fit.

TEST INFRASTRUCTURE.  This package is the plain, slow, double-precision
reference (``mpm_oracle.c``) that the CUDA library is checked against, plus a
ctypes wrapper taking numpy arrays.  Only ``tests/``, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py`` may import it; the product package
never does, and the two share no code.

Array conventions follow ``mpm_oracle.h``: float64, C-contiguous, voxel index
``x + nx*(y + ny*z)``; maps ``[K][N]``, images ``[I][N]`` contrast-major,
packed upper-triangular Hessian ``[K(K+1)/2][N]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpm_oracle.c")
_SO = os.path.join(_HERE, "libmpm_oracle.so")
_SO_OMP = os.path.join(_HERE, "libmpm_oracle_omp.so")

MAX_CONTRASTS = 8
MAX_IMAGES = 128

_handles = {}
_variant = "serial"


def _compile(out: str, extra) -> None:
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", *extra,
           "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(cmd, check=True)
    except BaseException:
        os.unlink(tmp)
        raise
    os.replace(tmp, out)


def _fresh(path: str) -> bool:
    return os.path.exists(path) and os.path.getmtime(path) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "mpm_oracle.h")))


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, no FP contraction so that x86
    and Arm hosts round identically): the serial library and, from the same
    source with -fopenmp, the threaded one.  Returns the serial library's
    path."""
    if force or not _fresh(_SO):
        _compile(_SO, [])
    if force or not _fresh(_SO_OMP):
        _compile(_SO_OMP, ["-fopenmp"])
    return _SO


def use_threads(n: int) -> int:
    """Run the following oracle calls serially (n == 1) or on n OpenMP threads
    (n > 1; n <= 0: all host cores).  The results are bit-identical either
    way.  Returns the thread count in use."""
    global _variant
    _variant = "serial" if n == 1 else "omp"
    return _lib().orc_threads(n if n > 1 else 0)


class OrcProblem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("vx", ctypes.c_double * 3),
        ("n_contrasts", ctypes.c_int),
        ("n_echoes", ctypes.c_int * MAX_CONTRASTS),
        ("alpha", ctypes.c_double * MAX_CONTRASTS),
        ("tr", ctypes.c_double * MAX_CONTRASTS),
        ("mt", ctypes.c_int * MAX_CONTRASTS),
        ("sigma2", ctypes.c_double * MAX_CONTRASTS),
        ("te", ctypes.c_double * MAX_IMAGES),
        ("n_maps", ctypes.c_int),
        ("lam", ctypes.c_double * 4),
        ("eps", ctypes.c_double),
        ("precond", ctypes.c_int),
    ]


class OrcProjection(ctypes.Structure):
    _fields_ = [
        ("dims", (ctypes.c_int * 3) * MAX_CONTRASTS),
        ("affine", (ctypes.c_double * 12) * MAX_CONTRASTS),
    ]


class OrcOpts(ctypes.Structure):
    _fields_ = [
        ("gn_iters", ctypes.c_int), ("cg_iters", ctypes.c_int),
        ("newton_per_irls", ctypes.c_int), ("init", ctypes.c_int),
        ("tol_gn", ctypes.c_double), ("tol_cg", ctypes.c_double),
        ("mg_levels", ctypes.c_int), ("mg_nu", ctypes.c_int),
        ("mg_omega", ctypes.c_double), ("mg_coarse_sweeps", ctypes.c_int),
    ]


class OrcMG(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("nu", ctypes.c_int), ("omega", ctypes.c_double),
                ("coarse_sweeps", ctypes.c_int)]


def make_mg(levels=8, nu=1, omega=0.7, coarse_sweeps=20) -> OrcMG:
    """Multigrid V-cycle settings (levels: at most this many)."""
    return OrcMG(int(levels), int(nu), float(omega), int(coarse_sweeps))


_D = ctypes.POINTER(ctypes.c_double)
_P = ctypes.POINTER(OrcProblem)
_Q = ctypes.POINTER(OrcProjection)
_DD = ctypes.POINTER(_D)
_U8 = ctypes.POINTER(ctypes.c_uint8)


def _lib():
    lib = _handles.get(_variant)
    if lib is None:
        build()
        lib = ctypes.CDLL(_SO if _variant == "serial" else _SO_OMP)
        lib.orc_threads.restype = ctypes.c_int
        lib.orc_threads.argtypes = [ctypes.c_int]
        lib.orc_signal.restype = ctypes.c_double
        lib.orc_signal.argtypes = [_D, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_int, ctypes.c_double, ctypes.c_double]
        lib.orc_signal_jet.restype = None
        lib.orc_signal_jet.argtypes = [_D, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                       _D, _D, _D]
        lib.orc_forward.argtypes = [_P, _D, _D, _D, _D]
        lib.orc_forward.restype = None
        lib.orc_grad_hess.argtypes = [_P, _D, _D, _D, _D, _D, _D]
        lib.orc_grad_hess.restype = ctypes.c_double
        lib.orc_jtv.argtypes = [_P, _D, _D]
        lib.orc_jtv.restype = ctypes.c_double
        lib.orc_membrane.argtypes = [_P, _D, _D, _D]
        lib.orc_membrane.restype = None
        lib.orc_membrane_diag.argtypes = [_P, _D, _D]
        lib.orc_membrane_diag.restype = None
        lib.orc_pcg.argtypes = [_P, _D, _D, _D, _D, ctypes.c_int, ctypes.c_double, _D]
        lib.orc_pcg.restype = ctypes.c_int
        lib.orc_solve.argtypes = [_P, _D, _D, _D, _D, _D, ctypes.c_int, ctypes.c_double, _D]
        lib.orc_solve.restype = ctypes.c_int
        lib.orc_uncertainty.argtypes = [_P, _D, _D, _D, _D, _D, _D]
        lib.orc_uncertainty.restype = ctypes.c_int
        lib.orc_init.argtypes = [_P, _D, _D]
        lib.orc_init.restype = None
        lib.orc_fit.argtypes = [_P, ctypes.POINTER(OrcOpts), _D, _D, _D, _D, _D, _D, _D, _D]
        lib.orc_fit.restype = ctypes.c_int
        lib.orc_pull.argtypes = [_P, ctypes.POINTER(ctypes.c_int), _D, ctypes.c_int, _D, _D, _U8]
        lib.orc_pull.restype = None
        lib.orc_push.argtypes = [_P, ctypes.POINTER(ctypes.c_int), _D, ctypes.c_int, _D, _D]
        lib.orc_push.restype = None
        lib.orc_grad_hess_proj.argtypes = [_P, _Q, _DD, _DD, _DD, _D, _D, _D]
        lib.orc_grad_hess_proj.restype = ctypes.c_double
        lib.orc_init_proj.argtypes = [_P, _Q, _DD, _D]
        lib.orc_init_proj.restype = None
        lib.orc_fit_proj.argtypes = [_P, _Q, ctypes.POINTER(OrcOpts), _DD, _DD, _DD, _D, _D, _D,
                                     _D, _D]
        lib.orc_fit_proj.restype = ctypes.c_int
        _G = ctypes.POINTER(OrcMG)
        lib.orc_mg_levels.argtypes = [_P, _G, ctypes.POINTER(ctypes.c_int * 3)]
        lib.orc_mg_levels.restype = ctypes.c_int
        lib.orc_mg_vcycle.argtypes = [_P, _D, _D, _G, _D, _D]
        lib.orc_mg_vcycle.restype = None
        lib.orc_mg_energy.argtypes = [_P, _D, _D, _G, ctypes.c_int, _D]
        lib.orc_mg_energy.restype = ctypes.c_double
        lib.orc_mg_pcg.argtypes = [_P, _D, _D, _D, _D, ctypes.c_int, ctypes.c_double, _G, _D]
        lib.orc_mg_pcg.restype = ctypes.c_int
        lib.orc_mg_solve.argtypes = [_P, _D, _D, _D, _D, _D, ctypes.c_int, ctypes.c_double, _G, _D]
        lib.orc_mg_solve.restype = ctypes.c_int
        _handles[_variant] = lib
    return lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def n_maps_for(protocol) -> int:
    return 4 if any(protocol["mt"]) else 3


def make_problem(protocol: dict, shape, vx=(1.0, 1.0, 1.0), lam=10.0, eps=1e-3,
                 precond: int = 0, n_maps: int | None = None) -> OrcProblem:
    """Build the oracle problem from a protocol dict (keys ``alpha`` (rad),
    ``tr`` (s), ``mt``, ``n_echoes``, ``te`` (s, flat, contrast-major),
    ``sigma2``) and a grid shape ``(nx, ny, nz)``."""
    p = OrcProblem()
    p.nx, p.ny, p.nz = (int(v) for v in shape)
    for d in range(3):
        p.vx[d] = float(vx[d])
    C = len(protocol["alpha"])
    assert C <= MAX_CONTRASTS
    p.n_contrasts = C
    for c in range(C):
        p.n_echoes[c] = int(protocol["n_echoes"][c])
        p.alpha[c] = float(protocol["alpha"][c])
        p.tr[c] = float(protocol["tr"][c])
        p.mt[c] = int(protocol["mt"][c])
        p.sigma2[c] = float(protocol["sigma2"][c])
    te = list(protocol["te"])
    assert len(te) == sum(protocol["n_echoes"]) <= MAX_IMAGES
    for i, t in enumerate(te):
        p.te[i] = float(t)
    p.n_maps = int(n_maps if n_maps is not None else n_maps_for(protocol))
    lam = np.broadcast_to(np.asarray(lam, dtype=np.float64), (4,))
    for k in range(4):
        p.lam[k] = float(lam[k])
    p.eps = float(eps)
    p.precond = int(precond)
    return p


def _nvox(p):
    return p.nx * p.ny * p.nz


def _nimg(p):
    return sum(p.n_echoes[c] for c in range(p.n_contrasts))


def signal(y4, alpha, tr, te, mt, b1p=1.0, b1m=1.0) -> float:
    y = np.zeros(4)
    y[:len(y4)] = y4
    return _lib().orc_signal(_ptr(y), alpha, tr, te, int(mt), b1p, b1m)


def signal_jet(y4, alpha, tr, te, mt, b1p=1.0, b1m=1.0):
    y = np.zeros(4)
    y[:len(y4)] = y4
    s = ctypes.c_double()
    ds = np.zeros(4)
    d2s = np.zeros(16)
    _lib().orc_signal_jet(_ptr(y), alpha, tr, te, int(mt), b1p, b1m,
                          ctypes.byref(s), _ptr(ds), _ptr(d2s))
    return s.value, ds, d2s.reshape(4, 4)


def forward(p, y, b1p=None, b1m=None):
    y, b1p, b1m = _f64(y), _f64(b1p), _f64(b1m)
    s = np.zeros((_nimg(p), _nvox(p)))
    _lib().orc_forward(ctypes.byref(p), _ptr(y), _ptr(b1p), _ptr(b1m), _ptr(s))
    return s


def grad_hess(p, x, y, b1p=None, b1m=None):
    """Returns (nll, g [K][N], h [T][N])."""
    x, y, b1p, b1m = _f64(x), _f64(y), _f64(b1p), _f64(b1m)
    K = p.n_maps
    g = np.zeros((K, _nvox(p)))
    h = np.zeros((K * (K + 1) // 2, _nvox(p)))
    nll = _lib().orc_grad_hess(ctypes.byref(p), _ptr(x), _ptr(y), _ptr(b1p), _ptr(b1m),
                               _ptr(g), _ptr(h))
    return nll, g, h


def jtv(p, y, want_w=True):
    """Returns (JTV_eps, w [N] or None)."""
    y = _f64(y)
    w = np.zeros(_nvox(p)) if want_w else None
    e = _lib().orc_jtv(ctypes.byref(p), _ptr(y), _ptr(w))
    return e, w


def membrane(p, w, v):
    w, v = _f64(w), _f64(v)
    out = np.zeros((p.n_maps, _nvox(p)))
    _lib().orc_membrane(ctypes.byref(p), _ptr(w), _ptr(v), _ptr(out))
    return out


def membrane_diag(p, w):
    w = _f64(w)
    d = np.zeros(_nvox(p))
    _lib().orc_membrane_diag(ctypes.byref(p), _ptr(w), _ptr(d))
    return d


def pcg(p, h, w, b, iters, tol=0.0):
    """Returns (x, iterations run, resid[0..iters])."""
    h, w, b = _f64(h), _f64(w), _f64(b)
    x = np.zeros((p.n_maps, _nvox(p)))
    resid = np.zeros(iters + 1)
    it = _lib().orc_pcg(ctypes.byref(p), _ptr(h), _ptr(w), _ptr(b), _ptr(x), iters, tol,
                        _ptr(resid))
    return x, it, resid[:max(it, 0) + 1]


def solve(p, h, w, g, y, iters, tol=0.0):
    """delta = (H + L)^-1 (g + L y).  Returns (delta, iterations, resid)."""
    h, w, g, y = _f64(h), _f64(w), _f64(g), _f64(y)
    d = np.zeros((p.n_maps, _nvox(p)))
    resid = np.zeros(iters + 1)
    it = _lib().orc_solve(ctypes.byref(p), _ptr(h), _ptr(w), _ptr(g), _ptr(y), _ptr(d),
                          iters, tol, _ptr(resid))
    return d, it, resid[:max(it, 0) + 1]


def mg_levels(p, mg):
    """Dimensions (nx, ny, nz) of every multigrid level."""
    dims = ((ctypes.c_int * 3) * 16)()
    L = _lib().orc_mg_levels(ctypes.byref(p), ctypes.byref(mg), dims)
    return [tuple(dims[l]) for l in range(L)]


def mg_vcycle(p, h, w, mg, r):
    h, w, r = _f64(h), _f64(w), _f64(r)
    z = np.zeros((p.n_maps, _nvox(p)))
    _lib().orc_mg_vcycle(ctypes.byref(p), _ptr(h), _ptr(w), ctypes.byref(mg), _ptr(r), _ptr(z))
    return z


def mg_energy(p, h, w, mg, level, e):
    """e' A_l e on multigrid level `level` (e is [K][N_l])."""
    h, w, e = _f64(h), _f64(w), _f64(e)
    return _lib().orc_mg_energy(ctypes.byref(p), _ptr(h), _ptr(w), ctypes.byref(mg), int(level),
                                _ptr(e))


def mg_pcg(p, h, w, b, iters, mg, tol=0.0):
    """orc_pcg with the multigrid preconditioner: (x, iterations, resid)."""
    h, w, b = _f64(h), _f64(w), _f64(b)
    x = np.zeros((p.n_maps, _nvox(p)))
    resid = np.zeros(iters + 1)
    it = _lib().orc_mg_pcg(ctypes.byref(p), _ptr(h), _ptr(w), _ptr(b), _ptr(x), iters, tol,
                           ctypes.byref(mg), _ptr(resid))
    return x, it, resid[:max(it, 0) + 1]


def mg_solve(p, h, w, g, y, iters, mg, tol=0.0):
    """delta = (H + L)^-1 (g + L y) by mg_pcg: (delta, iterations, resid)."""
    h, w, g, y = _f64(h), _f64(w), _f64(g), _f64(y)
    d = np.zeros((p.n_maps, _nvox(p)))
    resid = np.zeros(iters + 1)
    it = _lib().orc_mg_solve(ctypes.byref(p), _ptr(h), _ptr(w), _ptr(g), _ptr(y), _ptr(d), iters,
                             tol, ctypes.byref(mg), _ptr(resid))
    return d, it, resid[:max(it, 0) + 1]


def uncertainty(p, h, w, y=None):
    """Returns (var [K][N], logdet [N], moments [4][N] or None, status)."""
    h, w, y = _f64(h), _f64(w), _f64(y)
    N = _nvox(p)
    var = np.zeros((p.n_maps, N))
    logdet = np.zeros(N)
    mom = np.zeros((4, N)) if y is not None else None
    st = _lib().orc_uncertainty(ctypes.byref(p), _ptr(h), _ptr(w), _ptr(y), _ptr(var),
                                _ptr(logdet), _ptr(mom))
    return var, logdet, mom, st


def init(p, x):
    x = _f64(x)
    y = np.zeros((p.n_maps, _nvox(p)))
    _lib().orc_init(ctypes.byref(p), _ptr(x), _ptr(y))
    return y


def fit(p, x, y0=None, b1p=None, b1m=None, gn_iters=10, cg_iters=30, newton_per_irls=1,
        tol_gn=0.0, tol_cg=0.0, mg=None):
    """Whole fit.  ``y0=None`` starts from the constant initial maps; ``mg``
    (make_mg) solves with the multigrid-preconditioned CG.  Returns a dict
    with ``y``, ``iters``, ``F``, ``nll``, ``jtv``, ``cg_rel``."""
    x, b1p, b1m = _f64(x), _f64(b1p), _f64(b1m)
    o = OrcOpts(gn_iters, cg_iters, newton_per_irls, 1 if y0 is None else 0, tol_gn, tol_cg)
    if mg is not None:
        o.mg_levels, o.mg_nu, o.mg_omega, o.mg_coarse_sweeps = (mg.levels, mg.nu, mg.omega,
                                                                 mg.coarse_sweeps)
    y = np.zeros((p.n_maps, _nvox(p))) if y0 is None else np.array(y0, dtype=np.float64)
    F = np.zeros(gn_iters + 1)
    nll = np.zeros(gn_iters + 1)
    jt = np.zeros(gn_iters + 1)
    cg = np.zeros(max(gn_iters, 1))
    it = _lib().orc_fit(ctypes.byref(p), ctypes.byref(o), _ptr(x), _ptr(b1p), _ptr(b1m),
                        _ptr(y), _ptr(F), _ptr(nll), _ptr(jt), _ptr(cg))
    n = max(it, 0)
    return {"y": y, "iters": it, "F": F[:n + 1], "nll": nll[:n + 1], "jtv": jt[:n + 1],
            "cg_rel": cg[:n]}


# ------------------------------------------------------------ spatial projection

def make_projection(dims, affines) -> OrcProjection:
    """Per contrast: acquisition grid ``dims[c] = (mx, my, mz)`` and the 3 x 4
    (or 4 x 4) affine from its voxel coordinates to reconstruction voxel
    coordinates."""
    q = OrcProjection()
    for c, (d, a) in enumerate(zip(dims, affines)):
        a = np.asarray(a, dtype=np.float64)[:3, :4].reshape(12)
        for k in range(3):
            q.dims[c][k] = int(d[k])
        for k in range(12):
            q.affine[c][k] = float(a[k])
    return q


def _dims_aff(dims, A):
    d = (ctypes.c_int * 3)(*(int(v) for v in dims))
    a = np.ascontiguousarray(np.asarray(A, dtype=np.float64)[:3, :4].reshape(12))
    return d, a


def pull(p, dims, A, u):
    """Psi u for u [ch][N] -> (out [ch][M], inside [M] bool)."""
    u = _f64(np.atleast_2d(u))
    d, a = _dims_aff(dims, A)
    M = int(np.prod(dims))
    out = np.zeros((u.shape[0], M))
    inside = np.zeros(M, dtype=np.uint8)
    _lib().orc_pull(ctypes.byref(p), d, _ptr(a), u.shape[0], _ptr(u), _ptr(out),
                    inside.ctypes.data_as(_U8))
    return out, inside.astype(bool)


def push(p, dims, A, u):
    """Psi' u for u [ch][M] -> [ch][N]."""
    u = _f64(np.atleast_2d(u))
    d, a = _dims_aff(dims, A)
    out = np.zeros((u.shape[0], _nvox(p)))
    _lib().orc_push(ctypes.byref(p), d, _ptr(a), u.shape[0], _ptr(u), _ptr(out))
    return out


def _ptr_list(arrs, C):
    keep = [None if a is None else _f64(a) for a in (arrs if arrs is not None else [None] * C)]
    arr = (_D * C)(*[_ptr(a) if a is not None else None for a in keep])
    return arr, keep


def grad_hess_proj(p, q, xs, y, b1ps=None, b1ms=None):
    """Projected likelihood: xs[c] is [E_c][M_c].  Returns (nll, g, h)."""
    C = p.n_contrasts
    X, kx = _ptr_list(xs, C)
    BP, kp = _ptr_list(b1ps, C)
    BM, km = _ptr_list(b1ms, C)
    y = _f64(y)
    K = p.n_maps
    g = np.zeros((K, _nvox(p)))
    h = np.zeros((K * (K + 1) // 2, _nvox(p)))
    nll = _lib().orc_grad_hess_proj(ctypes.byref(p), ctypes.byref(q), X, BP, BM, _ptr(y),
                                    _ptr(g), _ptr(h))
    return nll, g, h


def init_proj(p, q, xs):
    X, kx = _ptr_list(xs, p.n_contrasts)
    y = np.zeros((p.n_maps, _nvox(p)))
    _lib().orc_init_proj(ctypes.byref(p), ctypes.byref(q), X, _ptr(y))
    return y


def fit_proj(p, q, xs, y0=None, b1ps=None, b1ms=None, gn_iters=10, cg_iters=30,
             newton_per_irls=1, tol_gn=0.0, tol_cg=0.0):
    """fit() with the projected likelihood."""
    C = p.n_contrasts
    X, kx = _ptr_list(xs, C)
    BP, kp = _ptr_list(b1ps, C)
    BM, km = _ptr_list(b1ms, C)
    o = OrcOpts(gn_iters, cg_iters, newton_per_irls, 1 if y0 is None else 0, tol_gn, tol_cg)
    y = np.zeros((p.n_maps, _nvox(p))) if y0 is None else np.array(y0, dtype=np.float64)
    F = np.zeros(gn_iters + 1)
    nll = np.zeros(gn_iters + 1)
    jt = np.zeros(gn_iters + 1)
    cg = np.zeros(max(gn_iters, 1))
    it = _lib().orc_fit_proj(ctypes.byref(p), ctypes.byref(q), ctypes.byref(o), X, BP, BM,
                             _ptr(y), _ptr(F), _ptr(nll), _ptr(jt), _ptr(cg))
    n = max(it, 0)
    return {"y": y, "iters": it, "F": F[:n + 1], "nll": nll[:n + 1], "jtv": jt[:n + 1],
            "cg_rel": cg[:n]}
