"""GB300-native (sm_103a) model-based multi-parameter mapping.

Python binding of the C ABI in ``include/mpm.h``: every function here only
checks and marshals torch CUDA tensors (device memory, the current stream)
into the library call of the same name; all arithmetic runs in the CUDA
kernels of ``libmpm.so``.  Importing this package does not load the library;
the first call does, and fails if it has not been built.

Layouts: maps ``[K, N]``, images ``[I, N]`` (contrast-major), Hessian
``[K(K+1)/2, N]`` packed upper triangle, ``N = nx * ny * nz`` with x fastest.
"""
from __future__ import annotations

import ctypes

from . import _lib
from ._lib import MPMError, Opts, Problem, Projection, Report

__all__ = [
    "make_problem", "make_opts", "workspace", "mpm_workspace_size", "mpm_forward",
    "mpm_grad_hess", "mpm_jtv_weights", "mpm_solve", "mpm_uncertainty", "mpm_fit", "mpm_fit_batch",
    "mpm_workspace_status", "mpm_autotune", "mpm_test_copy_timeout", "mpm_kernel_launches", "mpm_profile_enable", "mpm_profile_read",
    "MPMError", "Problem", "Opts", "Report", "Server",
    "Projection", "make_projection", "mpm_workspace_size_proj", "workspace_proj", "mpm_pull",
    "mpm_push", "mpm_grad_hess_proj", "mpm_fit_proj",
]


def make_problem(protocol: dict, shape, vx=(1.0, 1.0, 1.0), lam=10.0, eps=1e-3,
                 precond: int = 0, echo_dtype: int = 0) -> Problem:
    """Problem statement from a protocol dict (``alpha`` (rad), ``tr`` (s),
    ``mt``, ``n_echoes``, ``te`` (s, flat, contrast-major), ``sigma2``)."""
    p = Problem()
    p.nx, p.ny, p.nz = (int(v) for v in shape)
    for d in range(3):
        p.vx[d] = float(vx[d])
    C = len(protocol["alpha"])
    if C > _lib.MAX_CONTRASTS:
        raise ValueError("too many contrasts")
    p.n_contrasts = C
    for c in range(C):
        p.n_echoes[c] = int(protocol["n_echoes"][c])
        p.alpha[c] = float(protocol["alpha"][c])
        p.tr[c] = float(protocol["tr"][c])
        p.mt[c] = int(protocol["mt"][c])
        p.sigma2[c] = float(protocol["sigma2"][c])
    te = list(protocol["te"])
    if len(te) > _lib.MAX_IMAGES:
        raise ValueError("too many images")
    for i, t in enumerate(te):
        p.te[i] = float(t)
    p.n_maps = 4 if any(protocol["mt"]) else 3
    lam = list(lam) if hasattr(lam, "__len__") else [lam] * 4
    for k in range(4):
        p.lam[k] = float(lam[k] if k < len(lam) else lam[-1])
    p.eps = float(eps)
    p.precond = int(precond)
    p.echo_dtype = int(echo_dtype)
    return p


def make_opts(gn_iters=10, cg_iters=30, newton_per_irls=1, init=True, tol_gn=0.0,
              tol_cg=0.0, graph=False, mg_levels=0, mg_nu=1, mg_omega=0.7,
              mg_coarse_sweeps=20) -> Opts:
    """Schedule of a fit or solve (mpm_opts).  graph: False / True (one
    captured graph, subjects in lanes) or "phased" (one launch per phase across
    the subjects of a batch).  mg_levels > 0 selects the
    multigrid-preconditioned CG (an option; 0 is the paper's block
    preconditioner)."""
    g = 2 if graph == "phased" else (1 if graph else 0)
    return Opts(int(gn_iters), int(cg_iters), int(newton_per_irls), 1 if init else 0,
                float(tol_gn), float(tol_cg), g, int(mg_levels), int(mg_nu),
                float(mg_omega), int(mg_coarse_sweeps))


def _ptr(t, name, dtype=None, optional=False):
    if t is None:
        if optional:
            return None
        raise ValueError(f"{name} is required")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _f32():
    import torch
    return torch.float32


def mpm_workspace_size(problem: Problem, opts: Opts | None = None, call: int = _lib.CALL_FIT) -> int:
    lib = _lib.load()
    n = ctypes.c_size_t()
    _lib.check(lib.mpm_workspace_size(ctypes.byref(problem),
                                      ctypes.byref(opts) if opts is not None else None,
                                      call, ctypes.byref(n)), "mpm_workspace_size")
    return n.value


def workspace(problem: Problem, opts: Opts | None = None, call: int = _lib.CALL_FIT, device="cuda"):
    """Allocate a device workspace (torch uint8 tensor) for ``call``."""
    import torch
    return torch.empty(max(mpm_workspace_size(problem, opts, call), 1), dtype=torch.uint8,
                       device=device)


def mpm_forward(problem, y, b1p=None, b1m=None, out=None, stream=None):
    import torch
    lib = _lib.load()
    N = problem.nx * problem.ny * problem.nz
    I = sum(problem.n_echoes[c] for c in range(problem.n_contrasts))
    if out is None:
        out = torch.empty((I, N), dtype=torch.float32, device=y.device)
    _lib.check(lib.mpm_forward(ctypes.byref(problem), _ptr(y, "y", _f32()),
                               _ptr(b1p, "b1p", _f32(), True), _ptr(b1m, "b1m", _f32(), True),
                               _ptr(out, "s", _f32()), _stream(stream)), "mpm_forward")
    return out


def mpm_grad_hess(problem, x, y, b1p=None, b1m=None, g=None, h=None, nll=None, ws=None,
                  stream=None):
    """Returns (g [K,N], h [T,N], nll (device double tensor of one element))."""
    import torch
    lib = _lib.load()
    K, N = problem.n_maps, problem.nx * problem.ny * problem.nz
    dev = y.device
    g = torch.empty((K, N), dtype=torch.float32, device=dev) if g is None else g
    h = torch.empty((K * (K + 1) // 2, N), dtype=torch.float32, device=dev) if h is None else h
    nll = torch.empty(1, dtype=torch.float64, device=dev) if nll is None else nll
    ws = workspace(problem, None, _lib.CALL_GRAD_HESS, dev) if ws is None else ws
    xdt = torch.bfloat16 if problem.echo_dtype == 1 else torch.float32
    _lib.check(lib.mpm_grad_hess(ctypes.byref(problem), _ptr(x, "x", xdt), _ptr(y, "y", _f32()),
                                 _ptr(b1p, "b1p", _f32(), True), _ptr(b1m, "b1m", _f32(), True),
                                 _ptr(g, "g", _f32()), _ptr(h, "h", _f32()),
                                 _ptr(nll, "nll", torch.float64), _ptr(ws, "ws"), ws.numel(),
                                 _stream(stream)), "mpm_grad_hess")
    return g, h, nll


def mpm_jtv_weights(problem, y, w=None, jtv=None, ws=None, want_w=True, stream=None):
    """Returns (w [N] or None, jtv (device double tensor of one element))."""
    import torch
    lib = _lib.load()
    N = problem.nx * problem.ny * problem.nz
    dev = y.device
    if want_w and w is None:
        w = torch.empty(N, dtype=torch.float32, device=dev)
    jtv = torch.empty(1, dtype=torch.float64, device=dev) if jtv is None else jtv
    ws = workspace(problem, None, _lib.CALL_JTV, dev) if ws is None else ws
    _lib.check(lib.mpm_jtv_weights(ctypes.byref(problem), _ptr(y, "y", _f32()),
                                   _ptr(w, "w", _f32(), True), _ptr(jtv, "jtv", torch.float64),
                                   _ptr(ws, "ws"), ws.numel(), _stream(stream)),
               "mpm_jtv_weights")
    return w, jtv


def mpm_solve(problem, opts, h, w, g, y, delta=None, resid=None, ws=None, stream=None):
    """Returns (delta [K,N], resid (device doubles, cg_iters + 1))."""
    import torch
    lib = _lib.load()
    dev = y.device
    delta = torch.empty_like(g) if delta is None else delta
    resid = torch.full((opts.cg_iters + 1,), float("nan"), dtype=torch.float64,
                       device=dev) if resid is None else resid
    ws = workspace(problem, opts, _lib.CALL_SOLVE, dev) if ws is None else ws
    _lib.check(lib.mpm_solve(ctypes.byref(problem), ctypes.byref(opts), _ptr(h, "h", _f32()),
                             _ptr(w, "w", _f32()), _ptr(g, "g", _f32()), _ptr(y, "y", _f32()),
                             _ptr(delta, "delta", _f32()), _ptr(resid, "resid", torch.float64, True),
                             _ptr(ws, "ws"), ws.numel(), _stream(stream)), "mpm_solve")
    return delta, resid


def mpm_uncertainty(problem, h, w, y=None, var=None, logdet=None, moments=None,
                    want_logdet=True, want_moments=False, stream=None):
    """Returns (var [K,N], logdet [N] or None, moments [4,N] or None)."""
    import torch
    lib = _lib.load()
    dev = h.device
    K, N = problem.n_maps, problem.nx * problem.ny * problem.nz
    var = torch.empty((K, N), dtype=torch.float32, device=dev) if var is None else var
    if want_logdet and logdet is None:
        logdet = torch.empty(N, dtype=torch.float32, device=dev)
    if want_moments and moments is None:
        moments = torch.empty((4, N), dtype=torch.float32, device=dev)
    _lib.check(lib.mpm_uncertainty(ctypes.byref(problem), _ptr(h, "h", _f32()), _ptr(w, "w", _f32()),
                                   _ptr(y, "y", _f32(), True), _ptr(var, "var", _f32()),
                                   _ptr(logdet, "logdet", _f32(), True),
                                   _ptr(moments, "moments", _f32(), True), _stream(stream)),
               "mpm_uncertainty")
    return var, logdet, moments


def mpm_fit(problem, opts, x, y, b1p=None, b1m=None, var=None, ws=None, stream=None,
            allow_not_converged=True):
    """Fit in place: ``y`` holds the starting maps (ignored when ``opts.init``)
    and receives the result.  Returns (status, Report)."""
    import torch
    lib = _lib.load()
    ws = workspace(problem, opts, _lib.CALL_FIT, y.device) if ws is None else ws
    rep = Report()
    xdt = torch.bfloat16 if problem.echo_dtype == 1 else torch.float32
    allow = (_lib.OK, _lib.WARN_NOT_CONVERGED) if allow_not_converged else (_lib.OK,)
    st = _lib.check(lib.mpm_fit(ctypes.byref(problem), ctypes.byref(opts), _ptr(x, "x", xdt),
                                _ptr(b1p, "b1p", _f32(), True), _ptr(b1m, "b1m", _f32(), True),
                                _ptr(y, "y", _f32()), _ptr(var, "var", _f32(), True),
                                _ptr(ws, "ws"), ws.numel(), ctypes.byref(rep), _stream(stream)),
                    "mpm_fit", allow)
    return st, rep


def mpm_autotune(problem, opts, ws=None, stream=None, tile=-1):
    """Pick the stencil tile shape for this volume by timing each candidate
    (or pin ``tile`` >= 0 without timing).  Returns (tile index or -1,
    per-shape milliseconds)."""
    lib = _lib.load()
    if tile < 0 and ws is None:
        ws = workspace(problem, opts, _lib.CALL_SOLVE)
    tile = ctypes.c_int(tile)
    ms = (ctypes.c_float * _lib.TILE_SHAPES)()
    _lib.check(lib.mpm_autotune(ctypes.byref(problem), ctypes.byref(opts),
                                _ptr(ws, "ws", optional=True), ws.numel() if ws is not None else 0,
                                _stream(stream), ctypes.byref(tile), ms),
               "mpm_autotune")
    return tile.value, list(ms)


def mpm_fit_batch(problems, opts, xs, ys, b1ps=None, b1ms=None, vars=None, wss=None,
                  stream=None, allow_not_converged=True):
    """Fit several subjects together (see mpm_fit_batch in mpm.h).  Lists hold
    one entry per subject; ``wss`` defaults to freshly allocated workspaces.
    Returns (status, [Report])."""
    import torch
    lib = _lib.load()
    n = len(problems)
    if wss is None:
        wss = [workspace(p, opts, _lib.CALL_FIT, y.device) for p, y in zip(problems, ys)]
    V = ctypes.c_void_p
    P = ctypes.POINTER(Problem)
    parr = (P * n)(*[ctypes.pointer(p) for p in problems])
    xdt = lambda p: torch.bfloat16 if p.echo_dtype == 1 else torch.float32
    arr = lambda ts, name, dt=None, opt=False: (V * n)(*[
        _ptr(t, f"{name}[{i}]", dt(problems[i]) if callable(dt) else dt, opt)
        for i, t in enumerate(ts)])
    xa = arr(xs, "x", xdt)
    ya = arr(ys, "y", _f32())
    bpa = arr(b1ps, "b1p", _f32(), True) if b1ps is not None else None
    bma = arr(b1ms, "b1m", _f32(), True) if b1ms is not None else None
    va = arr(vars, "var", _f32(), True) if vars is not None else None
    wa = arr(wss, "ws")
    wb = (ctypes.c_size_t * n)(*[w.numel() for w in wss])
    reps = (Report * n)()
    allow = (_lib.OK, _lib.WARN_NOT_CONVERGED) if allow_not_converged else (_lib.OK,)
    st = _lib.check(lib.mpm_fit_batch(n, parr, ctypes.byref(opts), xa, bpa, bma, ya, va, wa, wb,
                                      reps, _stream(stream)), "mpm_fit_batch", allow)
    return st, list(reps)


# ------------------------------------------------------------ spatial projection

def make_projection(dims, affines) -> Projection:
    """Per contrast: acquisition grid ``dims[c] = (mx, my, mz)`` and the
    3 x 4 (or 4 x 4) affine from its voxel coordinates to reconstruction
    voxel coordinates (see mpm_projection in mpm.h)."""
    q = Projection()
    for c, (d, a) in enumerate(zip(dims, affines)):
        rows = [list(map(float, r[:4])) for r in list(a)[:3]]
        for k in range(3):
            q.dims[c][k] = int(d[k])
        for r in range(3):
            for k in range(4):
                q.affine[c][4 * r + k] = rows[r][k]
    return q


def mpm_workspace_size_proj(problem, proj, opts=None, call=_lib.CALL_FIT) -> int:
    lib = _lib.load()
    n = ctypes.c_size_t()
    _lib.check(lib.mpm_workspace_size_proj(ctypes.byref(problem), ctypes.byref(proj),
                                           ctypes.byref(opts) if opts is not None else None,
                                           int(call), ctypes.byref(n)), "mpm_workspace_size_proj")
    return n.value


def workspace_proj(problem, proj, opts=None, call=_lib.CALL_FIT, device="cuda"):
    import torch
    return torch.empty(max(mpm_workspace_size_proj(problem, proj, opts, call), 1),
                       dtype=torch.uint8, device=device)


def _ptr_array(ts, name, dtype, optional, C):
    ts = list(ts) if ts is not None else [None] * C
    return (ctypes.c_void_p * C)(*[_ptr(t, f"{name}[{c}]", dtype, optional)
                                   for c, t in enumerate(ts)])


def mpm_pull(problem, proj, contrast, u, stream=None):
    """Psi_c u for u ``[ch, N]`` -> ``[ch, M_c]``."""
    import torch
    lib = _lib.load()
    u2 = u.reshape(-1, u.shape[-1]) if u.dim() > 1 else u.reshape(1, -1)
    d = proj.dims[contrast]
    out = torch.empty((u2.shape[0], d[0] * d[1] * d[2]), dtype=torch.float32, device=u.device)
    _lib.check(lib.mpm_pull(ctypes.byref(problem), ctypes.byref(proj), int(contrast), u2.shape[0],
                            _ptr(u2, "u", _f32()), _ptr(out, "out", _f32()), _stream(stream)),
               "mpm_pull")
    return out


def mpm_push(problem, proj, contrast, u, out=None, accumulate=False, stream=None):
    """Psi_c' u for u ``[ch, M_c]`` -> ``[ch, N]`` (added to ``out`` if
    ``accumulate``)."""
    import torch
    lib = _lib.load()
    u2 = u.reshape(-1, u.shape[-1]) if u.dim() > 1 else u.reshape(1, -1)
    N = problem.nx * problem.ny * problem.nz
    if out is None:
        out = torch.zeros((u2.shape[0], N), dtype=torch.float32, device=u.device)
    _lib.check(lib.mpm_push(ctypes.byref(problem), ctypes.byref(proj), int(contrast), u2.shape[0],
                            _ptr(u2, "u", _f32()), _ptr(out, "out", _f32()), int(accumulate),
                            _stream(stream)), "mpm_push")
    return out


def mpm_grad_hess_proj(problem, proj, xs, y, b1ps=None, b1ms=None, ws=None, stream=None):
    """Projected voxel pass.  ``xs[c]``: contrast c's echoes ``[E_c, M_c]``.
    Returns (g ``[K, N]``, h ``[T, N]``, nll as a 0-d float64 CUDA tensor)."""
    import torch
    lib = _lib.load()
    C = problem.n_contrasts
    K = problem.n_maps
    N = problem.nx * problem.ny * problem.nz
    xdt = torch.bfloat16 if problem.echo_dtype == 1 else torch.float32
    ws = workspace_proj(problem, proj, None, _lib.CALL_GRAD_HESS, y.device) if ws is None else ws
    g = torch.empty((K, N), dtype=torch.float32, device=y.device)
    h = torch.empty((K * (K + 1) // 2, N), dtype=torch.float32, device=y.device)
    nll = torch.zeros((), dtype=torch.float64, device=y.device)
    _lib.check(lib.mpm_grad_hess_proj(ctypes.byref(problem), ctypes.byref(proj),
                                      _ptr_array(xs, "x", xdt, False, C),
                                      _ptr_array(b1ps, "b1p", _f32(), True, C),
                                      _ptr_array(b1ms, "b1m", _f32(), True, C),
                                      _ptr(y, "y", _f32()), _ptr(g, "g", _f32()),
                                      _ptr(h, "h", _f32()), _ptr(nll, "nll"), _ptr(ws, "ws"),
                                      ws.numel(), _stream(stream)), "mpm_grad_hess_proj")
    return g, h, nll


def mpm_fit_proj(problem, proj, opts, xs, y, b1ps=None, b1ms=None, var=None, ws=None,
                 stream=None, allow_not_converged=True):
    """mpm_fit with the projected likelihood; ``xs[c]`` is ``[E_c, M_c]``.
    Returns (status, Report)."""
    import torch
    lib = _lib.load()
    C = problem.n_contrasts
    xdt = torch.bfloat16 if problem.echo_dtype == 1 else torch.float32
    ws = workspace_proj(problem, proj, opts, _lib.CALL_FIT, y.device) if ws is None else ws
    rep = Report()
    allow = (_lib.OK, _lib.WARN_NOT_CONVERGED) if allow_not_converged else (_lib.OK,)
    st = _lib.check(lib.mpm_fit_proj(ctypes.byref(problem), ctypes.byref(proj), ctypes.byref(opts),
                                     _ptr_array(xs, "x", xdt, False, C),
                                     _ptr_array(b1ps, "b1p", _f32(), True, C),
                                     _ptr_array(b1ms, "b1m", _f32(), True, C),
                                     _ptr(y, "y", _f32()), _ptr(var, "var", _f32(), True),
                                     _ptr(ws, "ws"), ws.numel(), ctypes.byref(rep),
                                     _stream(stream)), "mpm_fit_proj", allow)
    return st, rep


class Server:
    """Continuous-batching fit server over a caller-provided device arena
    (see mpm_server_* in mpm.h).  Keeps references to every submitted
    request's tensors until it is done."""

    def __init__(self, arena, max_slots=8, stream=None):
        self._lib = _lib.load()
        self.arena = arena
        h = ctypes.c_void_p()
        _lib.check(self._lib.mpm_server_create(_ptr(arena, "arena"), arena.numel(), int(max_slots),
                                               _stream(stream), ctypes.byref(h)),
                   "mpm_server_create")
        self._h = h
        self._keep = {}

    def submit(self, problem, opts, x, y, b1p=None, b1m=None, var=None) -> int:
        import torch
        t = ctypes.c_int()
        xdt = torch.bfloat16 if problem.echo_dtype == 1 else torch.float32
        _lib.check(self._lib.mpm_server_submit(
            self._h, ctypes.byref(problem), ctypes.byref(opts), _ptr(x, "x", xdt),
            _ptr(b1p, "b1p", _f32(), True), _ptr(b1m, "b1m", _f32(), True), _ptr(y, "y", _f32()),
            _ptr(var, "var", _f32(), True), ctypes.byref(t)), "mpm_server_submit")
        self._keep[t.value] = (problem, opts, x, y, b1p, b1m, var)
        return t.value

    def step(self):
        """One non-blocking pass: advances every request whose last enqueued
        work has completed, admits queued ones; returns (active, queued,
        finished).  Call it in a loop."""
        a, q, f = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _lib.check(self._lib.mpm_server_step(self._h, ctypes.byref(a), ctypes.byref(q),
                                             ctypes.byref(f)), "mpm_server_step")
        return a.value, q.value, f.value

    def poll(self, ticket):
        """Returns (state, status, Report or None)."""
        state, status = ctypes.c_int(), ctypes.c_int()
        rep = Report()
        _lib.check(self._lib.mpm_server_poll(self._h, int(ticket), ctypes.byref(state),
                                             ctypes.byref(status), ctypes.byref(rep)),
                   "mpm_server_poll")
        done = state.value in (_lib.REQ_DONE, _lib.REQ_FAILED)
        if done:
            self._keep.pop(ticket, None)
        return state.value, status.value, rep if done else None

    def release(self, ticket):
        """Forget a finished ticket (its state and report)."""
        _lib.check(self._lib.mpm_server_release(self._h, int(ticket)), "mpm_server_release")

    def close(self):
        if self._h:
            self._lib.mpm_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mpm_workspace_status(ws, stream=None) -> int:
    lib = _lib.load()
    return lib.mpm_workspace_status(_ptr(ws, "ws"), ws.numel(), _stream(stream))


def mpm_test_copy_timeout(withhold: bool, wait_us: float = 0.0) -> None:
    """Test hook: the TMA PCG iteration's producer withholds its copies and
    every copy wait gives up after ``wait_us`` microseconds (0: default)."""
    _lib.check(_lib.load().mpm_test_copy_timeout(1 if withhold else 0, float(wait_us)),
               "mpm_test_copy_timeout")


def mpm_kernel_launches() -> int:
    return int(_lib.load().mpm_kernel_launches())


def mpm_profile_enable(on: bool = True) -> None:
    _lib.check(_lib.load().mpm_profile_enable(1 if on else 0), "mpm_profile_enable")


def mpm_profile_read() -> dict:
    """Per kernel kind: {"ms": summed milliseconds, "launches": count}; clears
    the records."""
    n = len(_lib.KERNEL_KINDS)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_ulonglong * n)()
    _lib.check(_lib.load().mpm_profile_read(ms, cnt, n), "mpm_profile_read")
    return {k: {"ms": ms[i], "launches": int(cnt[i])} for i, k in enumerate(_lib.KERNEL_KINDS)}
