"""The C-ABI library builds, loads and exports every symbol include/fbs.h declares.

No compute calls: these run without a GPU."""
import ctypes
import os
import re

import pytest

from paper_1511_03296_gb300 import build, fbs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(fbs_\w+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for required in ("fbs_grid_build", "fbs_bistochastize", "fbs_solve", "fbs_solve_robust",
                     "fbs_solve_backward"):
        assert required in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    assert sorted(fbs.EXPORTED) == declared_symbols()


def test_status_strings(lib):
    lib.fbs_status_string.restype = ctypes.c_char_p
    for s in range(8):
        assert lib.fbs_status_string(s)


def test_argument_errors_need_no_gpu(lib):
    # null / invalid arguments are rejected before any CUDA call
    lib.fbs_grid_build.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                   ctypes.c_void_p]
    out = ctypes.c_void_p(1)
    assert lib.fbs_grid_build(None, 1, None, ctypes.byref(out)) == 1
    assert out.value is None
    descs = ctypes.c_void_p(0x1000)    # never read: the image count is checked first
    assert lib.fbs_grid_build(descs, 65536, None, ctypes.byref(out)) == 1
    assert lib.fbs_grid_build(descs, 0, None, ctypes.byref(out)) == 1
    lib.fbs_bistochastize.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    assert lib.fbs_bistochastize(None, 2, None) == 1
    lib.fbs_solve.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    assert lib.fbs_solve(None, None, 25, None) == 1
    lib.fbs_grid_info.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                  ctypes.c_void_p]
    assert lib.fbs_grid_info(None, 0, None, None) == 1
    lib.fbs_autotune.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                 ctypes.c_void_p]
    assert lib.fbs_autotune(None, None, 25, None, None) == 1
    lib.fbs_solve_lowrank.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.fbs_solve_lowrank(None, None, 25, 0.01, None, None) == 1
    # the domain transform checks every argument before touching the device
    lib.fbs_domain_transform.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_int, ctypes.c_float,
                                         ctypes.c_float, ctypes.c_int, ctypes.c_void_p]
    fake = ctypes.c_void_p(0x1000)     # never dereferenced: each call fails validation first
    for args in ((None, 8, 8, fake, 1, 32.0, 64.0, 3),          # no guide
                 (fake, 8, 8, None, 1, 32.0, 64.0, 3),          # no x
                 (fake, 0, 8, fake, 1, 32.0, 64.0, 3),          # empty image
                 (fake, 8, 8, fake, 0, 32.0, 64.0, 3),          # no channels
                 (fake, 8, 8, fake, 1, 0.0, 64.0, 3),           # sigma_s
                 (fake, 8, 8, fake, 1, 32.0, float("inf"), 3),  # sigma_r
                 (fake, 8, 8, fake, 1, 32.0, 64.0, 0),          # iterations
                 (fake, 8, 8, fake, 1, 32.0, 64.0, 17),
                 (fake, 8, 28001, fake, 1, 32.0, 64.0, 3)):     # row wider than shared memory
        assert lib.fbs_domain_transform(*args, None) == 1, args


def test_autograd_function_is_exposed():
    torch = pytest.importorskip("torch")
    assert issubclass(fbs.BilateralSolve, torch.autograd.Function)


def test_binding_fails_loudly_without_library(tmp_path):
    with pytest.raises(RuntimeError, match="not built"):
        fbs._lib = None
        fbs.load(str(tmp_path / "missing.so"))
