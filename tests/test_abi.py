"""The C-ABI library loads and exports every entry point its header declares
(no compute call is made: these run without a GPU)."""

import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w ]*?\**\s*\b(ising_\w+)\s*\(",
                                txt, flags=re.M))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["ising_create", "ising_prune", "ising_select_domain", "ising_reconstruct",
                 "ising_energy", "ising_solve", "ising_ds_create", "ising_ds_run"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2312_05837_gb300 import _lib
    lib = _lib.load()
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layouts_match_the_header(tmp_path):
    """Field offsets of the ctypes mirrors equal those a C compiler gives."""
    import shutil
    import subprocess
    from paper_2312_05837_gb300 import _lib as L
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"ising_instance": L.Instance, "ising_ds_params": L.DSParams,
               "ising_ds_stats": L.DSStats, "ising_server_cfg": L.ServerCfg,
               "ising_result": L.Result, "ising_server_stats": L.ServerStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ising_ds.h"',
             'int main(void) {']
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, str(src), "-I", os.path.join(ROOT, "include"), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                  check=True).stdout.splitlines())
    for cname, cls in structs.items():
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(cls, f).offset, (cname, f)
    assert L.load().ising_version() == 10000


def test_binding_has_no_cpu_fallback(monkeypatch, tmp_path):
    from paper_2312_05837_gb300 import _lib as L
    monkeypatch.setattr(L, "_lib", None)
    monkeypatch.setattr(L, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        L.load()
