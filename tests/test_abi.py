"""The C-ABI library loads and exports what include/kot.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2310_14087_gb300 import _build, kot

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return kot.lib()


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "kot.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kot_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("kot_create", "kot_build_features", "kot_ssn_solve", "kot_batch_solve",
                     "kot_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)
    assert sorted(kot.EXPORTS) == _declared_functions()


def test_default_options_follow_the_paper(lib):
    o = kot.default_options()
    # Sec. 5 constants and the CG cap of the Sec. 4.4 remark
    assert (o.alpha1, o.alpha2, o.beta0, o.beta1, o.beta2) == (1e-6, 1.0, 0.5, 1.2, 5.0)
    assert o.cg_max_iter == 20
    assert (o.tau, o.kappa, o.theta0) == (0.1, 1.0, 1.0)
    assert o.precision == kot.FP64 and o.use_eg == 1
    # library choices: products below 8e6 multiply-adds on the FP64 pipes, five refinement steps
    assert o.tc_min_flops == 8e6 and o.eig_refine == 5


def test_struct_layouts_match_header(lib):
    # kot_options: int, pointer, 4 ints, 13 doubles, 3 ints, 1 double, 4 ints, 1 double (natural alignment;
    # the library asserts the same sizes at compile time)
    assert ctypes.sizeof(kot.Options) == 8 * 4 + 13 * 8 + 16 + 8 + 16 + 8
    assert ctypes.sizeof(kot.Result) == 5 * 4 + 4 + 7 * 8 + 16


def test_null_arguments_are_rejected_without_gpu_work(lib):
    assert lib.kot_default_options(None) == kot.ERR_INVALID
    assert lib.kot_create(None, None) == kot.ERR_INVALID
    assert lib.kot_destroy(None) == kot.OK
    assert lib.kot_last_error(None) == b"null context"
    for fn, args in (("kot_build_features", [None, 1, 1, None, None, 1, None, None, 1.0, 1.0, 1.0]),
                     ("kot_ssn_solve", [None, 1e-6, None, None, None, None, None]),
                     ("kot_batch_solve", [None, 0, None, None])):
        assert getattr(lib, fn)(*args) == kot.ERR_INVALID


def test_invalid_options_rejected(lib):
    h = ctypes.c_void_p()
    bad = kot.default_options(tau=1.5)
    assert lib.kot_create(ctypes.byref(h), ctypes.byref(bad)) == kot.ERR_INVALID
    bad = kot.default_options(precision=7)
    assert lib.kot_create(ctypes.byref(h), ctypes.byref(bad)) == kot.ERR_INVALID
