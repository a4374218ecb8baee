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
