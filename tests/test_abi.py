"""The C ABI library builds, loads without a GPU and exports every entry
point declared in include/qbe.h; the Python binding covers them all.  CPU only
(no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qbe.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qbe_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    import __graft_entry__ as g

    g.build()
    from paper_1408_1782_gb300 import qbe

    return qbe.LIB_PATH


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("qbe_create", "qbe_set_boundary", "qbe_set_bfield", "qbe_set_state", "qbe_get_state",
                     "qbe_collide", "qbe_step", "qbe_moments", "qbe_advect", "qbe_collide_rk2", "qbe_destroy",
                     "qbe_last_error", "qbe_set_stream"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(L, name), name


def test_binding_covers_every_declared_symbol(libpath):
    from paper_1408_1782_gb300 import qbe

    assert sorted(qbe.SIGNATURES) == declared_functions()
    qbe.lib()


def test_structs_match_header_layout():
    from paper_1408_1782_gb300 import qbe

    # qbe_grid: 4 ints, 2 doubles, 2 ints; qbe_fd: 3 + 8 doubles
    assert ctypes.sizeof(qbe.QbeGrid) == 4 * 4 + 2 * 8 + 2 * 4
    assert ctypes.sizeof(qbe.QbeFD) == 11 * 8


def test_create_rejects_bad_arguments_without_touching_a_gpu(libpath):
    """Argument validation happens before any CUDA call."""
    from paper_1408_1782_gb300 import qbe

    L = qbe.lib()
    h = ctypes.c_void_p()
    for bad in (dict(N=12), dict(N=40), dict(N=16, J=5), dict(N=16, M=0), dict(N=16, Nx=0), dict(N=16, L=-1.0)):
        args = dict(N=16, Nx=4, J=8, M=8, L=12.0, R=7.5)
        args.update(bad)
        g = qbe.QbeGrid(args["N"], args["Nx"], args["J"], args["M"], args["L"], args["R"], 0, 0)
        assert L.qbe_create(ctypes.byref(g), ctypes.byref(h)) == -1
    g = qbe.QbeGrid(16, 4, 8, 8, 12.0, 7.5, 2, 0)
    assert L.qbe_create(ctypes.byref(g), ctypes.byref(h)) == -5
    assert L.qbe_create(None, ctypes.byref(h)) == -1
