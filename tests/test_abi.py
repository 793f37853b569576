"""The C-ABI library builds, loads without a GPU, and exports every function
include/mdlg.h declares (no compute calls)."""

import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"^\s*(?:int|void|const char\s*\*)\s*\**\s*(\w+)\s*\(", txt, flags=re.M)
    return names


def test_header_declares_boundary():
    names = set(_declared())
    for f in ("md_init", "md_init_batch", "md_step", "mdlg_bin", "feq_measured", "feq_gaussian",
              "wsg_lambda", "feq_wsg", "md_get_state", "md_set_state", "md_energy", "md_destroy",
              "md_last_error"):
        assert f in names, f


def test_library_exports_every_declared_symbol():
    from paper_2101_01160_gb300 import build

    so = build.build()
    lib = ctypes.CDLL(so)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2101_01160_gb300 import mdlg

    monkeypatch.setattr(mdlg, "_SO", str(tmp_path / "missing.so"))
    monkeypatch.setattr(mdlg, "_lib", None)
    try:
        mdlg.load()
    except ImportError:
        return
    raise AssertionError("load() must raise when the library is missing")
