"""ctypes view of the C ABI in ``include/mpm.h`` (``libmpm.so``).

Structures mirror the header field by field; prototypes are declared once
on first load.  Loading fails loudly when the library has not been built:
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmpm.so")

MAX_CONTRASTS = 8
MAX_IMAGES = 64
MAX_REPORT = 256
MAX_BATCH = 64

OK = 0
WARN_NOT_CONVERGED = 1
ERR_INVALID_ARG = -1
ERR_WORKSPACE_TOO_SMALL = -2
ERR_CUDA = -3
ERR_NUMERIC = -4
ERR_TIMEOUT = -5

CALL_FIT, CALL_SOLVE, CALL_GRAD_HESS, CALL_JTV = 0, 1, 2, 3
REQ_QUEUED, REQ_ACTIVE, REQ_DONE, REQ_FAILED = 0, 1, 2, 3


class Problem(ctypes.Structure):
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
        ("echo_dtype", ctypes.c_int),
    ]


class Opts(ctypes.Structure):
    _fields_ = [
        ("gn_iters", ctypes.c_int), ("cg_iters", ctypes.c_int),
        ("newton_per_irls", ctypes.c_int), ("init", ctypes.c_int),
        ("tol_gn", ctypes.c_double), ("tol_cg", ctypes.c_double),
        ("graph", ctypes.c_int),
        ("mg_levels", ctypes.c_int), ("mg_nu", ctypes.c_int), ("mg_omega", ctypes.c_double),
        ("mg_coarse_sweeps", ctypes.c_int),
    ]


class Report(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int),
        ("F", ctypes.c_double * (MAX_REPORT + 1)),
        ("nll", ctypes.c_double * (MAX_REPORT + 1)),
        ("jtv", ctypes.c_double * (MAX_REPORT + 1)),
        ("cg_rel", ctypes.c_double * MAX_REPORT),
        ("cg_done", ctypes.c_int * MAX_REPORT),
    ]


class Projection(ctypes.Structure):
    _fields_ = [
        ("dims", (ctypes.c_int * 3) * MAX_CONTRASTS),
        ("affine", (ctypes.c_double * 12) * MAX_CONTRASTS),
    ]


# Exported symbols and their prototypes (restype, argtypes).
_P = ctypes.POINTER(Problem)
_O = ctypes.POINTER(Opts)
_V = ctypes.c_void_p
_S = ctypes.c_size_t
_Q = ctypes.POINTER(Projection)
_VA = ctypes.POINTER(ctypes.c_void_p)
PROTOTYPES = {
    "mpm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "mpm_last_error": (ctypes.c_char_p, []),
    "mpm_workspace_size": (ctypes.c_int, [_P, _O, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    "mpm_forward": (ctypes.c_int, [_P, _V, _V, _V, _V, _V]),
    "mpm_grad_hess": (ctypes.c_int, [_P, _V, _V, _V, _V, _V, _V, _V, _V, _S, _V]),
    "mpm_jtv_weights": (ctypes.c_int, [_P, _V, _V, _V, _V, _S, _V]),
    "mpm_solve": (ctypes.c_int, [_P, _O, _V, _V, _V, _V, _V, _V, _V, _S, _V]),
    "mpm_solve_static": (ctypes.c_int, [_P, _O, _V, _V, _V, _V, _V, _V, _V]),
    "mpm_uncertainty": (ctypes.c_int, [_P, _V, _V, _V, _V, _V, _V, _V]),
    "mpm_fit": (ctypes.c_int, [_P, _O, _V, _V, _V, _V, _V, _V, _S, ctypes.POINTER(Report), _V]),
    "mpm_fit_batch": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_P), _O, ctypes.POINTER(_V),
                                     ctypes.POINTER(_V), ctypes.POINTER(_V), ctypes.POINTER(_V),
                                     ctypes.POINTER(_V), ctypes.POINTER(_V),
                                     ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(Report), _V]),
    "mpm_workspace_status": (ctypes.c_int, [_V, _S, _V]),
    "mpm_workspace_size_proj": (ctypes.c_int, [_P, _Q, _O, ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_size_t)]),
    "mpm_pull": (ctypes.c_int, [_P, _Q, ctypes.c_int, ctypes.c_int, _V, _V, _V]),
    "mpm_push": (ctypes.c_int, [_P, _Q, ctypes.c_int, ctypes.c_int, _V, _V, ctypes.c_int, _V]),
    "mpm_grad_hess_proj": (ctypes.c_int, [_P, _Q, _VA, _VA, _VA, _V, _V, _V, _V, _V, _S, _V]),
    "mpm_fit_proj": (ctypes.c_int, [_P, _Q, _O, _VA, _VA, _VA, _V, _V, _V, _S,
                                    ctypes.POINTER(Report), _V]),
    "mpm_server_create": (ctypes.c_int, [_V, _S, ctypes.c_int, _V, ctypes.POINTER(_V)]),
    "mpm_server_submit": (ctypes.c_int, [_V, _P, _O, _V, _V, _V, _V, _V,
                                         ctypes.POINTER(ctypes.c_int)]),
    "mpm_server_step": (ctypes.c_int, [_V, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "mpm_server_poll": (ctypes.c_int, [_V, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(Report)]),
    "mpm_server_release": (ctypes.c_int, [_V, ctypes.c_int]),
    "mpm_server_destroy": (ctypes.c_int, [_V]),
    "mpm_autotune": (ctypes.c_int, [_P, _O, _V, _S, _V, ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_float)]),
    "mpm_test_copy_timeout": (ctypes.c_int, [ctypes.c_int, ctypes.c_double]),
    "mpm_kernel_launches": (ctypes.c_ulonglong, []),
    "mpm_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "mpm_profile_read": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_ulonglong), ctypes.c_int]),
}

TILE_SHAPES = 3      # MPM_TILE_SHAPES

KERNEL_KINDS = ["grad_hess", "jtv", "pcg_init", "pcg_step", "pcg_final", "uncertainty",
                "forward", "init", "grad_hess_proj", "reslice", "multigrid"]

_handle = None


def load():
    """Load ``libmpm.so`` (raises if it is missing) and declare prototypes."""
    global _handle
    if _handle is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in PROTOTYPES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _handle = lib
    return _handle


class MPMError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        msg = lib.mpm_status_string(status).decode()
        detail = lib.mpm_last_error().decode()
        super().__init__(f"{where}: {msg} ({status}){': ' + detail if detail else ''}")
        self.status = status


def check(status: int, where: str, allow=(OK,)) -> int:
    if status not in allow:
        raise MPMError(status, where)
    return status
