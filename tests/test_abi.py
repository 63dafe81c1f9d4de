"""The C-ABI library loads and exports every entry point include/meg.h
declares (no compute call: no GPU needed)."""
import ctypes
import re
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2012_10469_gb300 import build, binding
    build.build()
    return binding.load()


def test_header_declares_the_boundary():
    from paper_2012_10469_gb300 import binding
    names = set(binding.exported_symbols())
    for need in ("meg_create", "meg_set_objective", "meg_step", "meg_solve", "meg_certificate",
                 "meg_destroy", "meg_get_iterate", "meg_last_error"):
        assert need in names


def test_library_exports_every_declared_symbol(built_lib):
    from paper_2012_10469_gb300 import binding
    for name in binding.exported_symbols():
        assert hasattr(built_lib, name), name
        assert isinstance(getattr(built_lib, name), ctypes._CFuncPtr)


def test_header_has_no_torch_types():
    with open(os.path.join(ROOT, "include", "meg.h")) as f:
        text = f.read()
    assert not re.search(r"\b(at::|torch|Tensor)\b", text)


def test_footprint_is_host_only(built_lib):
    from paper_2012_10469_gb300 import binding
    small = binding.meg_footprint(200, 5, 4, binding.MEG_FP64, binding.MEG_DENSE_QUAD)
    big = binding.meg_footprint(4096, 10, 6, binding.MEG_MIXED_BF16, binding.MEG_DENSE_QUAD)
    assert 0 < small < big
    assert binding.meg_footprint(0, 5, 4, 0, 0) < 0


def test_options_struct_matches_header():
    from paper_2012_10469_gb300 import binding
    with open(os.path.join(ROOT, "include", "meg.h")) as f:
        text = f.read()
    body = text[text.index("typedef struct {\n    int n, r, p, q;"):]
    body = body[: body.index("} meg_options;")]
    fields = re.findall(r"\b(\w+)\s*[,;]", body.replace("typedef struct {", ""))
    py = [f for f, _ in binding.meg_options._fields_]
    assert fields == py
