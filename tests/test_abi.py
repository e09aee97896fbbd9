"""The C-ABI library loads and exports every function include/sbio.h declares
(no GPU needed: nothing here calls into a kernel)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sbio.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(sbio_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as G

    G.build()
    import paper_2506_20809_gb300.sbio as S

    return S


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("sbio_ctx_create", "sbio_geom_create", "sbio_apply_laplace", "sbio_apply_stokes_sl",
                 "sbio_apply_laplace_host", "sbio_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    import ctypes

    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(so, n)]
    assert not missing, missing
    # the binding wraps every declared function under the same name
    assert set(declared_functions()) <= set(lib.EXPORTED)


def test_version_and_error_string(lib):
    assert "sbio" in lib.sbio_version()
    assert isinstance(lib.sbio_last_error(), str)


def test_invalid_arguments_rejected_without_gpu(lib):
    """Argument validation happens before any device work."""
    import ctypes

    so = ctypes.CDLL(lib.LIB_PATH)
    so.sbio_ctx_create.argtypes = [ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p]
    assert so.sbio_ctx_create(0, 0, None) == lib.SBIO_EINVAL
    so.sbio_apply_laplace.argtypes = [ctypes.c_void_p] * 6
    assert so.sbio_apply_laplace(None, None, None, None, None, None) == lib.SBIO_EINVAL
