"""Host-side checks of the C ABI (no GPU needed): the library builds, loads
and exports every entry point that include/fs.h declares, and the binding's
structures match the header's field lists."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fs.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1907_06821_gb300 import build as b
    path = b.build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fs_[A-Za-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fs_create", "fs_apply_H", "fs_solve", "fs_destroy", "fs_npw", "fs_gvectors",
                     "fs_get_states", "fs_set_initial_states", "fs_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_null_safe_calls_without_gpu(lib):
    lib.fs_destroy.argtypes = [ctypes.c_void_p]
    lib.fs_destroy(None)                         # NULL is accepted
    lib.fs_last_error.restype = ctypes.c_char_p
    lib.fs_last_error.argtypes = [ctypes.c_void_p]
    assert lib.fs_last_error(None) == b"no context"
    lib.fs_create.restype = ctypes.c_int
    assert lib.fs_create(None, ctypes.c_double(1.0), None, None, None, None, None) == 1  # FS_ERR_ARG
    lib.fs_linear_solve.restype = ctypes.c_int
    assert lib.fs_linear_solve(None, ctypes.c_double(0.0), None, None, 0, 0, 0, ctypes.c_double(1e-8), 10,
                               None) == 1
    lib.fs_set_linear_states.restype = ctypes.c_int
    assert lib.fs_set_linear_states(None, None, None, None, 0, 0) == 1
    lib.fs_spectral_bounds.restype = ctypes.c_int
    assert lib.fs_spectral_bounds(None, 10, None, None) == 1
    lib.fs_wait_selftest.restype = ctypes.c_int
    assert lib.fs_wait_selftest(None, ctypes.c_longlong(10)) == 1


def test_binding_structs_match_header():
    import paper_1907_06821_gb300 as fs
    text = open(HEADER).read()

    blocks = {name: body for body, name in re.findall(r"typedef struct \{([^}]*)\}\s*(\w+);", text)}

    def fields(struct):
        body = re.sub(r"/\*.*?\*/", "", blocks[struct], flags=re.S)
        return re.findall(r"([A-Za-z_][A-Za-z_0-9]*)\s*(?:\[\d+\])?\s*;", body)
    for cls, name in ((fs.fs_grid, "fs_grid"), (fs.fs_projectors, "fs_projectors"),
                      (fs.fs_options, "fs_options"), (fs.fs_result, "fs_result"), (fs.fs_linres, "fs_linres"),
                      (fs.fs_chebfd_result, "fs_chebfd_result")):
        assert [f[0] for f in cls._fields_] == fields(name), name
