"""The C-ABI library loads on a machine without a GPU and exports every
function include/miugks.h declares; the oracle exports what oracle.h declares.
No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared(header):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b((?:miugks|oracle)_[a-z0-9_]+)\s*\(", text)))


def test_library_builds_loads_and_exports_every_declared_symbol():
    from paper_1704_03151_gb300 import build, miugks
    build.build()
    lib = ctypes.CDLL(build.LIB)
    names = declared(os.path.join(ROOT, "include", "miugks.h"))
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(miugks.exported_symbols()) <= set(names)


def test_oracle_exports_every_declared_symbol():
    import oracle
    lib = ctypes.CDLL(oracle.build())
    names = declared(os.path.join(ROOT, "oracle", "oracle.h"))
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_refuses_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_1704_03151_gb300 import miugks, workloads
    with pytest.raises(miugks.MiugksError):
        miugks.Solver(workloads.cavity(n=4, nvel=4))


def test_binding_structures_match_the_header_layout(tmp_path):
    """Every struct of include/miugks.h has, in a C compile of the header, the
    size and field offsets of its ctypes counterpart in the binding."""
    import subprocess
    import shutil
    if not shutil.which("gcc"):
        pytest.skip("no host C compiler")
    from paper_1704_03151_gb300 import miugks
    structs = {name: getattr(miugks, name) for name in
               ("miugks_mesh", "miugks_vgrid", "miugks_gas", "miugks_bc", "miugks_opts")}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "miugks.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for field, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, field, name, field))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)]).decode().splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(got["%s.%s" % (name, field)]) == getattr(cls, field).offset, (name, field)
