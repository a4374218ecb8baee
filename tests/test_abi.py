"""The C ABI without a GPU: the library builds and loads, exports every entry
point that include/mpm.h declares, its structures have the header's layout,
and argument errors are reported on the host before anything reaches a
device."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_2102_01604_gb300 import _lib, build, phantom

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mpm.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mpm_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ("mpm_fit", "mpm_forward", "mpm_grad_hess", "mpm_jtv_weights", "mpm_solve",
                 "mpm_uncertainty", "mpm_workspace_size"):
        assert need in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _lib.PROTOTYPES, name


def test_struct_layout_matches_header(lib):
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "mpm.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(mpm_problem), sizeof(mpm_opts), sizeof(mpm_report),
         sizeof(mpm_projection), offsetof(mpm_projection, affine));
  printf("%zu %zu %zu %zu %zu %zu\n", offsetof(mpm_problem, te), offsetof(mpm_problem, n_maps),
         offsetof(mpm_problem, lambda), offsetof(mpm_problem, echo_dtype),
         offsetof(mpm_report, cg_rel), offsetof(mpm_report, cg_done));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as tmp:
        c = os.path.join(tmp, "layout.c")
        exe = os.path.join(tmp, "layout")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-std=c11", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(v) for v in out]
    P, O, R = _lib.Problem, _lib.Opts, _lib.Report
    assert sizes[:3] == [ctypes.sizeof(P), ctypes.sizeof(O), ctypes.sizeof(R)]
    assert sizes[3:5] == [ctypes.sizeof(_lib.Projection), _lib.Projection.affine.offset]
    assert sizes[5:] == [P.te.offset, P.n_maps.offset, P.lam.offset, P.echo_dtype.offset,
                         R.cg_rel.offset, R.cg_done.offset]


def _problem(shape=(32, 32, 16), **kw):
    import paper_2102_01604_gb300 as mpm
    return mpm.make_problem(phantom.protocol(), shape, **kw)


def test_workspace_size_and_validation(lib):
    import paper_2102_01604_gb300 as mpm
    p = _problem()
    o = mpm.make_opts()
    small = mpm.mpm_workspace_size(p, o)
    big = mpm.mpm_workspace_size(_problem((64, 64, 32)), o)
    assert 0 < small < big
    # the fit workspace is enough for every other call
    for call in (_lib.CALL_SOLVE, _lib.CALL_GRAD_HESS, _lib.CALL_JTV):
        assert mpm.mpm_workspace_size(p, o, call) <= small
    n = ctypes.c_size_t()
    bad = [("n_maps", 3), ("n_contrasts", 0), ("eps", 0.0), ("precond", 7), ("echo_dtype", 2),
           ("nx", -1)]
    for field, val in bad:
        q = _problem()
        setattr(q, field, val)
        st = lib.mpm_workspace_size(ctypes.byref(q), ctypes.byref(o), 0, ctypes.byref(n))
        assert st == _lib.ERR_INVALID_ARG, field
        assert lib.mpm_last_error().decode()
    q = _problem()
    q.alpha[1] = 0.0
    assert lib.mpm_workspace_size(ctypes.byref(q), ctypes.byref(o), 0, ctypes.byref(n)) == _lib.ERR_INVALID_ARG
    q = _problem()
    q.sigma2[2] = -1.0
    assert lib.mpm_workspace_size(ctypes.byref(q), ctypes.byref(o), 0, ctypes.byref(n)) == _lib.ERR_INVALID_ARG
    o2 = mpm.make_opts(cg_iters=0)
    assert lib.mpm_workspace_size(ctypes.byref(p), ctypes.byref(o2), 0, ctypes.byref(n)) == _lib.ERR_INVALID_ARG
    assert lib.mpm_workspace_size(None, ctypes.byref(o), 0, ctypes.byref(n)) == _lib.ERR_INVALID_ARG


def test_host_pointers_are_refused(lib):
    """A host pointer would fault inside a kernel: the call refuses it first."""
    import numpy as np
    p = _problem((4, 4, 2))
    y = np.zeros((4, 32), dtype=np.float32)
    s = np.zeros((22, 32), dtype=np.float32)
    st = lib.mpm_forward(ctypes.byref(p), y.ctypes.data, None, None, s.ctypes.data, None)
    assert st == _lib.ERR_INVALID_ARG
    msg = lib.mpm_last_error().decode()
    assert "y" in msg


def test_status_strings(lib):
    for s in (0, 1, -1, -2, -3, -4, -5):
        assert lib.mpm_status_string(s).decode()


def _eye_proj(mpm, dims, C=3):
    return mpm.make_projection([dims] * C, [[[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]]] * C)


def test_projection_validation(lib):
    """Spatial projection: singular or non-finite affines, empty grids and host
    pointers are refused before anything is enqueued; the workspace grows with
    the acquisition grids."""
    import numpy as np
    import paper_2102_01604_gb300 as mpm
    p = _problem((16, 12, 8))
    o = mpm.make_opts()
    q = _eye_proj(mpm, (16, 12, 8))
    base = mpm.mpm_workspace_size_proj(p, q, o)
    assert base > mpm.mpm_workspace_size(p, o)
    q2 = _eye_proj(mpm, (32, 24, 8))
    assert mpm.mpm_workspace_size_proj(p, q2, o) > base
    n = ctypes.c_size_t()
    for mutate in ("singular", "nan", "dims", "fine"):
        qb = _eye_proj(mpm, (16, 12, 8))
        if mutate == "singular":
            for k in range(12):
                qb.affine[1][k] = 0.0
        elif mutate == "nan":
            qb.affine[2][5] = float("nan")
        elif mutate == "fine":
            for r in range(3):
                qb.affine[1][5 * r] = 0.2           # 5x smaller acquisition voxels
        else:
            qb.dims[0][2] = 0
        st = lib.mpm_workspace_size_proj(ctypes.byref(p), ctypes.byref(qb), ctypes.byref(o), 0,
                                         ctypes.byref(n))
        assert st == _lib.ERR_INVALID_ARG, mutate
        assert lib.mpm_last_error().decode()
    # a host pointer among the per-contrast images
    x = np.zeros((8, 16 * 12 * 8), dtype=np.float32)
    xs = (ctypes.c_void_p * 3)(x.ctypes.data, x.ctypes.data, x.ctypes.data)
    y = np.zeros((4, 16 * 12 * 8), dtype=np.float32)
    st = lib.mpm_grad_hess_proj(ctypes.byref(p), ctypes.byref(q), xs, None, None, y.ctypes.data,
                                y.ctypes.data, y.ctypes.data, y.ctypes.data, None, 0, None)
    assert st == _lib.ERR_INVALID_ARG
    assert "x[0]" in lib.mpm_last_error().decode()


def test_every_compute_call_refuses_host_memory_and_null_problems(lib):
    """Each entry point that takes device arrays names the first host array it
    is given, and a NULL problem, before it enqueues anything."""
    import numpy as np
    import paper_2102_01604_gb300 as mpm
    shape = (8, 8, 4)
    p = _problem(shape)
    o = mpm.make_opts(gn_iters=2, cg_iters=4)
    q = _eye_proj(mpm, shape)
    N = 8 * 8 * 4
    host = np.zeros(64 * N, dtype=np.float32)        # large enough for any array here
    hp = host.ctypes.data
    d = ctypes.c_double()
    rep = _lib.Report()
    arr = (ctypes.c_void_p * 3)(hp, hp, hp)
    P, O, Q = ctypes.byref(p), ctypes.byref(o), ctypes.byref(q)
    calls = {
        "mpm_forward": lambda pp: lib.mpm_forward(pp, hp, None, None, hp, None),
        "mpm_grad_hess": lambda pp: lib.mpm_grad_hess(pp, hp, hp, None, None, hp, hp,
                                                      ctypes.addressof(d), hp, 1 << 20, None),
        "mpm_jtv_weights": lambda pp: lib.mpm_jtv_weights(pp, hp, hp, ctypes.addressof(d), hp,
                                                          1 << 20, None),
        "mpm_solve": lambda pp: lib.mpm_solve(pp, O, hp, hp, hp, hp, hp, None, hp, 1 << 20, None),
        "mpm_solve_static": lambda pp: lib.mpm_solve_static(pp, O, hp, hp, hp, hp, hp, None, None),
        "mpm_uncertainty": lambda pp: lib.mpm_uncertainty(pp, hp, hp, hp, hp, None, None, None),
        "mpm_fit": lambda pp: lib.mpm_fit(pp, O, hp, None, None, hp, None, hp, 1 << 20,
                                          ctypes.byref(rep), None),
        "mpm_pull": lambda pp: lib.mpm_pull(pp, Q, 0, 4, hp, hp, None),
        "mpm_push": lambda pp: lib.mpm_push(pp, Q, 0, 4, hp, hp, 0, None),
        "mpm_grad_hess_proj": lambda pp: lib.mpm_grad_hess_proj(pp, Q, arr, None, None, hp, hp,
                                                                hp, ctypes.addressof(d), hp,
                                                                1 << 20, None),
        "mpm_fit_proj": lambda pp: lib.mpm_fit_proj(pp, Q, O, arr, None, None, hp, None, hp,
                                                    1 << 20, ctypes.byref(rep), None),
    }
    for name, call in calls.items():
        assert call(P) == _lib.ERR_INVALID_ARG, name
        assert lib.mpm_last_error().decode(), name
        assert call(None) == _lib.ERR_INVALID_ARG, name + " (NULL problem)"
    # batched fit: a host image array of the second subject
    pa = (ctypes.POINTER(_lib.Problem) * 2)(ctypes.pointer(p), ctypes.pointer(p))
    V2 = ctypes.c_void_p * 2
    st = lib.mpm_fit_batch(2, pa, O, V2(hp, hp), None, None, V2(hp, hp), None, V2(hp, hp),
                           (ctypes.c_size_t * 2)(1 << 20, 1 << 20), None, None)
    assert st == _lib.ERR_INVALID_ARG and lib.mpm_last_error().decode()
    # an empty batch is a no-op; negative or oversized batches are refused
    assert lib.mpm_fit_batch(0, None, O, None, None, None, None, None, None, None, None,
                             None) == _lib.OK
    for bad in (-1, _lib.MAX_BATCH + 1):
        assert lib.mpm_fit_batch(bad, pa, O, V2(hp, hp), None, None, V2(hp, hp), None,
                                 V2(hp, hp), (ctypes.c_size_t * 2)(1 << 20, 1 << 20), None,
                                 None) == _lib.ERR_INVALID_ARG
    # the server: host arena, bad slot count, NULL handles
    out = ctypes.c_void_p()
    assert lib.mpm_server_create(hp, 1 << 20, 2, None, ctypes.byref(out)) == _lib.ERR_INVALID_ARG
    assert not out.value
    assert lib.mpm_server_create(hp, 1 << 20, 0, None, ctypes.byref(out)) == _lib.ERR_INVALID_ARG
    n = ctypes.c_int()
    assert lib.mpm_server_step(None, ctypes.byref(n), ctypes.byref(n), ctypes.byref(n)) == _lib.ERR_INVALID_ARG
    assert lib.mpm_server_poll(None, 1, ctypes.byref(n), ctypes.byref(n), None) == _lib.ERR_INVALID_ARG
    assert lib.mpm_server_release(None, 1) == _lib.ERR_INVALID_ARG
    assert lib.mpm_server_destroy(None) == _lib.OK            # like free(NULL)
    assert lib.mpm_workspace_status(hp, 1 << 20, None) == _lib.ERR_INVALID_ARG
