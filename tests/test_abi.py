"""The C-ABI library loads and exports every symbol include/stroke_expand.h declares
(no GPU needed: only symbol lookup, no compute call)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "stroke_expand.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(se_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def so():
    from paper_2405_00127_gb300 import build
    return build.build()


def test_header_declares_the_api():
    syms = declared_symbols()
    assert "se_expand" in syms and "se_encode" in syms and "se_ctx_create" in syms


def test_library_exports_every_declared_symbol(so):
    lib = ctypes.CDLL(so)
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol(so):
    from paper_2405_00127_gb300 import binding
    assert sorted(binding.EXPORTED) == declared_symbols()
    for name in binding.EXPORTED:
        assert callable(getattr(binding, name))
