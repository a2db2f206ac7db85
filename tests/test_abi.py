"""The C-ABI library builds, loads and exports every entry point that
include/mlmc.h declares (CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mlmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(mlmc_[a-z0-9_]+)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ("mlmc_level_sums", "mlmc_estimate", "mlmc_multilevel_sums",
                 "mlmc_workspace_bytes", "mlmc_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1612_07717_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points():
    import paper_1612_07717_gb300 as M
    p = M.make_params()
    assert p.H == 600.0 and p.M0 == 8 and p.c_f == 15.0
    assert M.lib().mlmc_workspace_bytes(ctypes.byref(p), 1) >= 4 << 20
    assert "invalid" in M.strerror(M.EINVAL)
    assert "unstable" in M.strerror(M.EUNSTABLE)


def test_package_import_does_not_need_the_library(monkeypatch):
    import importlib
    import paper_1612_07717_gb300 as M
    monkeypatch.setattr(M, "LIB_PATH", "/nonexistent/libmlmc.so")
    M._lib = None
    with pytest.raises(RuntimeError, match="not built"):
        M.lib()
    # the reload defines the ctypes classes anew and leaves the library
    # unloaded, so the next lib() binds its argument types to them
    importlib.reload(M)
