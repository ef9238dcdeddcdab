"""The C-ABI library loads and exports every symbol include/lpa.h declares (no GPU)."""
import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(lpa_[a-z0-9_]+)\s*\(", text):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2411_11468_gb300 import build
    path = build.build()
    return ct.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "lpa_create" in names and "lpa_run" in names and "lpa_modularity" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert missing == []


def test_binding_symbol_list_matches_header():
    from paper_2411_11468_gb300 import lpa
    assert set(lpa.SYMBOLS) <= set(declared_functions())


def test_struct_layout_matches_binding(lib):
    from paper_2411_11468_gb300 import lpa
    lib.lpa_struct_size.restype = ct.c_size_t
    assert lib.lpa_struct_size(0) == ct.sizeof(lpa.Stats)
    assert lib.lpa_struct_size(1) == ct.sizeof(lpa.Tuning)


def test_strerror_without_gpu(lib):
    lib.lpa_strerror.restype = ct.c_char_p
    assert lib.lpa_strerror(0) == b"success"
    assert lib.lpa_strerror(-1) == b"invalid argument"
    lib.lpa_kernel_name.restype = ct.c_char_p
    assert lib.lpa_kernel_name(2) == b"warp"


def test_tuning_fields_are_checked_by_name():
    from paper_2411_11468_gb300 import lpa
    t = lpa.Tuning().update(float_values=2, hub_chunk=4096)
    assert t.float_values == 2 and t.hub_chunk == 4096
    with pytest.raises(KeyError):
        t.update(float_value=2)          # a misspelt field is an error, not a no-op
    with pytest.raises(KeyError):
        t.update(reserved=1)
