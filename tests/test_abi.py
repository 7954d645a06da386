"""The C-ABI library loads and exports every function that include/*.h
declares (no compute calls: runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(drk_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_render_entry_points():
    names = declared_functions()
    for req in ("drk_render", "drk_render_backward", "drk_ctx_create", "drk_ctx_destroy", "drk_sort_pairs"):
        assert req in names


def test_library_exports_every_declared_symbol():
    from paper_2412_11752_gb300 import build as B
    path = B.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads_and_reports_defaults():
    from paper_2412_11752_gb300 import drk
    o = drk.default_options()
    assert o.kbuf_capacity in (8, 16) and o.cull_level == 2
    assert abs(o.alpha_min - 1.2340980e-4) < 1e-9
    assert drk.lib().drk_version().startswith(b"libdrk")


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2412_11752_gb300 import build as B, drk
    monkeypatch.setattr(B, "LIB", str(tmp_path / "nope.so"))
    monkeypatch.setattr(drk, "_lib", None)
    with pytest.raises(RuntimeError):
        drk.lib()


def test_context_calls_reject_null_arguments_before_any_cuda_call():
    # the host-side argument checks come first, so they run without a GPU:
    # each returns DRK_ERR_INVALID_ARG and leaves its message
    from paper_2412_11752_gb300 import drk
    L = drk.lib()
    calls = (("drk_stats_enable", (None, 0)), ("drk_timing_enable", (None, 1)), ("drk_get_stats", (None, None)),
             ("drk_ctx_create", (0, None)))
    for name, args in calls:
        assert getattr(L, name)(*args) == 1, name
        assert L.drk_last_error(), name
