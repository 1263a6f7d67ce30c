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


def test_binding_structs_match_the_header(lib, tmp_path):
    # Every public struct of include/pir.h, compiled by the host C compiler:
    # size and each field's offset equal the ctypes mirror the binding uses.
    import shutil
    import subprocess

    cc = shutil.which("cc") or shutil.which("gcc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = {name: getattr(lib, name) for name in
               ("pir_table", "pir_plan", "pir_server_config", "pir_server_stats", "pir_work_item")}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "pir.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'    printf("{name} %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'    printf("{name}.{field} %zu\\n", offsetof({name}, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(line.rsplit(" ", 1) for line in subprocess.check_output([str(exe)], text=True).splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(got[f"{name}.{field}"]) == getattr(cls, field).offset, (name, field)


def test_binding_constants_match_the_header(lib):
    """Every integer constant the binding re-exports under a header macro's
    name (engines, status bits, error codes) has the header's value."""
    defs = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        for m in re.finditer(r"^#define\s+(PIR_\w+)\s+\(?(-?\d+)u?\)?", open(h).read(), flags=re.M):
            defs[m.group(1)] = int(m.group(2))
    shared = [k for k in defs if isinstance(getattr(lib, k, None), int)]
    assert "PIR_CONTRACT_TC_F16" in shared and "PIR_CONTRACT_IMAD" in shared
    for k in shared:
        assert getattr(lib, k) == defs[k], k
