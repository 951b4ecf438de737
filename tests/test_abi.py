"""The C-ABI library loads and exports every entry point declared in
include/*.h (no compute calls: CPU only)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names |= set(re.findall(r"^\s*(?:rl_status|const char \*)\s*(rl_[a-z0-9_]+)\s*\(", src, re.M))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("rl_context_create", "rl_forest_create_random", "rl_forest_adapt",
                 "rl_forest_update_modes", "rl_relocalise", "rl_relocalise_batch",
                 "rl_cascade_relocalise", "rl_scene_box", "rl_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1810_12163_gb300 import binding
    if not os.path.exists(binding.LIB_PATH):
        from paper_1810_12163_gb300 import build
        build.build()
    lib = ctypes.CDLL(binding.LIB_PATH)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(binding.exported_symbols()) == _declared()


def test_product_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1810_12163_gb300 import binding
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(binding, "_lib", None)
    with pytest.raises(ImportError):
        binding.lib()


def test_error_path_without_gpu():
    """Argument validation happens before any device work."""
    from paper_1810_12163_gb300 import binding
    if not os.path.exists(binding.LIB_PATH):
        pytest.skip("library not built")
    L = binding.lib()
    assert L.rl_context_create(0, None, 0, None) == 1
    assert b"null" in L.rl_last_error()
    assert L.rl_forest_destroy(None) == 1
    assert L.rl_reloc_destroy(None) == 1


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the public structs have the C compiler's sizes
    and field offsets (gcc on the header itself)."""
    import ctypes
    import subprocess

    from paper_1810_12163_gb300 import binding as B
    structs = {"rl_intrinsics": B.Intrinsics, "rl_forest_params": B.ForestParams,
               "rl_icp_params": B.IcpParams, "rl_ransac_params": B.RansacParams,
               "rl_result": B.Result, "rl_tuning": B.Tuning, "rl_server_params": B.ServerParams,
               "rl_server_stats": B.ServerStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "relocgb.h"', 'int main(void) {']
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in cls._fields_:
            lines.append(f'printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        name, field, v = ln.split()
        got[(name, field)] = int(v)
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for f in cls._fields_:
            assert got[(cname, f[0])] == getattr(cls, f[0]).offset, (cname, f[0])
