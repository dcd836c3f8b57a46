"""The C-ABI library loads and exports every symbol include/ks.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2502_11686_gb300 import build as kbuild
from paper_2502_11686_gb300 import native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ks.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(ks_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    kbuild.build()
    return ctypes.CDLL(kbuild.LIB)


def test_header_and_binding_agree():
    assert declared_functions() == sorted(native.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_default_options(lib):
    o = native.ks_default_options()
    assert (o.device, o.precision, o.sync, o.mem_budget) == (0, native.KS_FP64, 1, 0)


def test_null_ctx_is_rejected_without_gpu(lib):
    native.load()
    assert native.load().ks_smooth(None, 1, 1, None, None, None, None, None, None, None, None,
                                   None, None, None) == native.KS_ERR_ARG
    assert native.load().ks_destroy(None) == native.KS_OK
    assert native.load().ks_release(None, None) == native.KS_ERR_ARG
