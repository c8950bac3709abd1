"""The C ABI library builds for sm_103a, loads without a GPU, and exports every
entry point that include/inhand.h declares; argument checks that need no GPU
reject bad input with the documented status codes."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2002_12160_gb300 import build
    return build.build()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "inhand.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:ih_status|int32_t|const char \*)\s*([a-z_0-9]+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["sim_create", "sim_destroy", "sim_set_state", "sim_step", "sim_read_sensors",
                     "cost_eval", "optimizer_update"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = C.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_export(libpath):
    from paper_2002_12160_gb300 import inhand
    assert sorted(inhand.EXPORTS) == declared_functions()


def test_null_arguments_are_rejected_without_a_gpu(libpath):
    lib = C.CDLL(libpath)
    lib.sim_create.restype = C.c_int
    lib.sim_create.argtypes = [C.c_void_p] * 3 + [C.c_void_p, C.c_void_p]
    out = C.c_void_p()
    assert lib.sim_create(None, None, None, None, C.byref(out)) == 1   # IH_ERR_ARG
    lib.sim_last_error.restype = C.c_char_p
    lib.sim_last_error.argtypes = [C.c_void_p]
    assert b"null" in lib.sim_last_error(None)
    for name in ["sim_step", "sim_sync", "sim_destroy"]:
        fn = getattr(lib, name)
        fn.restype = C.c_int
    lib.sim_step.argtypes = [C.c_void_p, C.c_int, C.c_int]
    assert lib.sim_step(None, 0, 1) == 1
    assert lib.sim_destroy(None) == 0
