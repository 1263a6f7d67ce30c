"""The C-ABI library loads on a machine without a GPU and exports every entry
point that include/*.h declares (no compute calls here)."""
import ctypes
import glob
import os
import re

import pytest

from conftest import ROOT


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \t\*]*?\b(pir_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g

    g.build_library()
    import paper_2301_10904_gb300 as pir

    return pir


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("pir_keygen", "pir_server_eval", "pir_reconstruct", "pir_server_eval_device",
                 "pir_server_eval_range"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in _declared_functions() if not hasattr(so, n)]
    assert not missing, missing


def test_key_size_and_domain(lib):
    assert lib.pir_key_bytes(20) == 32 + 1280
    assert [lib.pir_domain_bits(r) for r in (1, 2, 3, 4, 5, 1 << 20, (1 << 20) + 1)] == [1, 1, 2, 2, 3, 20, 21]
    assert lib.pir_domain_bits(0) == 0


def test_error_strings(lib):
    assert lib.pir_error_string(0) == "ok"
    assert lib.pir_error_string(-3) == "malformed key"
