"""The C-ABI library loads and exports every function include/hydro.h declares
(no GPU call is made)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "hydro.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hydro_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hydro_create", "hydro_set_state", "hydro_cfl_dt", "hydro_step", "hydro_get_state",
                     "hydro_batch_create", "hydro_batch_run", "hydro_mlp_train", "hydro_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2503_04428_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2503_04428_gb300 import hydro
    monkeypatch.setattr(hydro, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(hydro, "_lib", None)
    try:
        hydro.lib()
    except ImportError as e:
        assert "no CPU fallback" in str(e)
    else:
        raise AssertionError("binding loaded a missing library")
