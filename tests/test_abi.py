"""The C ABI library loads on the CPU and exports every entry point that
include/csp.h declares.  No compute call is made here."""

import ctypes
import os
import re

import pytest

from paper_1511_05174_gb300 import _binding
from paper_1511_05174_gb300 import build as pkg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "csp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(csp_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    path = pkg_build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    assert set(names) == set(_binding.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_loads_and_rejects_bad_device():
    lib = _binding.load_library()
    ctx = ctypes.c_void_p()
    st = lib.csp_create(ctypes.byref(ctx), -1, 0)
    assert st != _binding.CSP_OK
    assert lib.csp_last_error(None)  # a message is set


def test_null_context_is_rejected():
    lib = _binding.load_library()
    assert lib.csp_set_geometry(None, None) == _binding.CSP_ERR_INVALID
    assert lib.csp_solve(None, None, None, 0, None, None, None, None) == _binding.CSP_ERR_INVALID
