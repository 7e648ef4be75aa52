"""The C-ABI library builds, loads and exports every symbol include/uotk.h
declares; host-side validation runs without a GPU.  CPU only."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2306_13618_gb300 import build, uotk
    build.build()
    return uotk.lib()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "uotk.h")).read()
    return sorted(set(re.findall(r"\b(uotk_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for want in ("uotk_kernel_sum", "uotk_uot_sinkhorn", "uotk_sinkhorn_divergence", "uotk_mmd2"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_names_match_header(lib):
    from paper_2306_13618_gb300 import uotk
    assert sorted(uotk.EXPORTED) == declared_symbols()


def test_null_context_is_rejected_on_host(lib):
    st = lib.uotk_kernel_sum(None, None, 3, None, 0, None, None, 0, None, 1.0, None)
    assert st == 1  # UOTK_ERR_INVALID, no device touched
    assert lib.uotk_status_string(1) == b"invalid argument"
    assert lib.uotk_status_string(6) == b"not converged"
    assert lib.uotk_launch_count(None) == 0
