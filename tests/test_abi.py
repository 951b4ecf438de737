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
