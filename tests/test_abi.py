"""The C ABI library builds for sm_103a, loads, and exports every function
include/brng.h declares; host-side argument checks that need no device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "brng.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|uint32_t|uint64_t)\s+(brng_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1412_4825_gb300 import build_lib
    path = build_lib.build()
    return C.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["brng_create", "brng_destroy", "brng_uniform", "brng_normal", "brng_exponential",
                     "brng_gamma", "brng_dirichlet", "brng_mixed", "brng_gibbs_run",
                     "brng_philox_words", "brng_read_counters"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_side_argument_checks(lib):
    lib.brng_create.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.POINTER(C.c_void_p)]
    h = C.c_void_p()
    assert lib.brng_create(1, 0, 0, C.byref(h)) == 1  # no streams
    assert lib.brng_create(1, 4, 0, None) == 1        # no output slot
    assert lib.brng_create(1, 4, 48, C.byref(h)) == 1  # buffer length not a power of two
    assert lib.brng_destroy(None) == 0
    lib.brng_fp64_eval.argtypes = [C.c_uint32, C.c_size_t, C.c_void_p, C.c_void_p, C.c_void_p]
    assert lib.brng_fp64_eval(9, 1, None, None, None) == 1
    lib.brng_set_tuning.argtypes = [C.c_void_p, C.c_void_p]
    assert lib.brng_set_tuning(None, None) == 1
    lib.brng_gibbs_run.argtypes = [C.c_void_p, C.c_int, C.c_uint64, C.c_uint32, C.c_uint32,
                                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    assert lib.brng_gibbs_run(None, 0, 0, 1, 1, None, None, None, None) == 1


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    """The binding has no fallback: with the library absent the import raises."""
    import importlib.util
    src = os.path.join(ROOT, "paper_1412_4825_gb300", "brng.py")
    dst = tmp_path / "brng_copy.py"
    dst.write_text(open(src).read())
    spec = importlib.util.spec_from_file_location("brng_copy", str(dst))
    mod = importlib.util.module_from_spec(spec)
    with pytest.raises(ImportError):
        spec.loader.exec_module(mod)


def test_binding_constants_match_header():
    """The binding's copies of the header's limits agree with it."""
    from paper_1412_4825_gb300 import brng as B
    text = open(HEADER).read()
    defs = dict(re.findall(r"^#define\s+(BRNG_\w+)\s+([0-9.]+)[uf]?\s*$", text, flags=re.M))
    assert int(defs["BRNG_STATIC_MAX_STREAMS"]) == B.BRNG_STATIC_MAX_STREAMS
