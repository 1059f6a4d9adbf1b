"""The C-ABI library builds, loads without a GPU, and exports every function
declared in include/*.h; host-side argument checks reject bad input without
touching a GPU."""
import ctypes as C
import glob
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\**\s*(cqm_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2006_05186_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("cqm_bem_setup", "cqm_bem_solve", "cqm_bem_rhs_plane_wave", "cqm_bem_destroy",
              "cqm_bem_strerror"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2006_05186_gb300 import _lib
    so = _lib.lib_path()
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    assert set(_lib.EXPORTED) == set(declared_functions())


def test_strerror_and_defaults(lib):
    from paper_2006_05186_gb300 import _lib
    assert lib.cqm_bem_strerror(0) == b"ok"
    assert b"invalid" in lib.cqm_bem_strerror(1)
    p = _lib.default_params()
    assert p.mode == _lib.MODE_H2MACA and p.n_min == 32 and p.eta == 1.0 and p.cheb_m == 4
    assert p.tensor_cores == 1 and p.inner_fp32 == 1 and p.rank_cap == 32
    assert p.exact_ff == 1 and p.expand_near == 1 and p.expand_far == 1
    assert p.aca_eps == 1e-6 and p.g_sing == 5 and p.gmres_tol == 1e-13
    assert lib.cqm_params_default(None) == _lib.CQM_EINVAL


def test_setup_rejects_bad_arguments_on_host(lib):
    """Validation happens on the host before any device work."""
    from paper_2006_05186_gb300 import _lib
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=np.float64)
    h = C.c_void_p()
    for tri, dt, N, bdf in [
        (np.array([[0, 1, 3]], np.int32), 0.1, 4, 2),     # index out of range
        (np.array([[0, 1, 1]], np.int32), 0.1, 4, 2),     # repeated vertex
        (np.array([[0, 1, 2]], np.int32), -0.1, 4, 2),    # dt <= 0
        (np.array([[0, 1, 2]], np.int32), 0.1, 0, 2),     # N < 1
        (np.array([[0, 1, 2]], np.int32), 0.1, 4, 3),     # BDF order
    ]:
        mesh = _lib.cqm_mesh(3, xyz.ctypes.data, 1, tri.ctypes.data)
        st = lib.cqm_bem_setup(C.byref(mesh), dt, N, bdf, None, None, C.byref(h))
        assert st == _lib.CQM_EINVAL
        assert h.value is None
    assert lib.cqm_bem_setup(None, 0.1, 4, 2, None, None, C.byref(h)) == _lib.CQM_EINVAL
    tri = np.array([[0, 1, 2]], np.int32)
    mesh = _lib.cqm_mesh(3, xyz.ctypes.data, 1, tri.ctypes.data)
    for field, value in [("rank_cap", 65), ("rank_cap", 0), ("cheb_m", 5), ("cheb_m", 0),
                         ("n_min", 33), ("inner_rtol", 1.0), ("eta", 0.0), ("g_sing", 13),
                         ("tc_single_ratio", -1.0)]:
        prm = _lib.cqm_params()
        assert lib.cqm_params_default(C.byref(prm)) == 0
        setattr(prm, field, value)
        st = lib.cqm_bem_setup(C.byref(mesh), 0.1, 4, 2, C.byref(prm), None, C.byref(h))
        assert st == _lib.CQM_EINVAL, (field, value)
        assert h.value is None
    assert lib.cqm_bem_destroy(None) == 0
    assert len(lib.cqm_bem_last_error()) >= 0
    # the P1 and mixed-boundary calls check their arguments before any device work
    buf = np.zeros(4)
    p = buf.ctypes.data
    assert lib.cqm_bem_p1_matrices(None, p, p, p, 0) == _lib.CQM_EINVAL
    dm = np.zeros(1, np.int32)
    assert lib.cqm_bem_solve_mixed(None, dm.ctypes.data, p, p, p, p, 0) == _lib.CQM_EINVAL
