"""The C ABI library builds, loads and exports every symbol that include/lt.h declares;
the Python binding covers the same set (CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "lt.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^LT_API\s+[\w\s\*]+?\b(lt_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def liblt():
    from paper_2202_02870_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lt_make_dct", "lt_make_cproduct", "lt_ctx_create", "lt_ctx_destroy",
                     "lt_workspace_size", "lt_transform", "lt_inverse", "lt_product",
                     "lt_svd", "lt_svt", "lt_pga_complete", "lt_pga_complete_batched",
                     "lt_last_device_status", "lt_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(liblt):
    for name in declared_functions():
        assert hasattr(liblt, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2202_02870_gb300 import lt
    assert sorted(lt.SIGNATURES) == declared_functions()
    for name in declared_functions():
        assert callable(getattr(lt, name)), name


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    from paper_2202_02870_gb300 import lt
    monkeypatch.setattr(lt, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(lt, "_lib", None)
    with pytest.raises(RuntimeError):
        lt.lib()
