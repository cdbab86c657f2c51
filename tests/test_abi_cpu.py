"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every function declared in include/*.h, and rejects
invalid arguments before any device work."""
import ctypes
import os
import re

import pytest

import paper_2507_01439_gb300 as trg
from paper_2507_01439_gb300 import build as trbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    trbuild.build()
    return trg.load_library()


def _declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(turboreg_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_every_declared_function_is_exported(lib):
    declared = _declared_functions()
    assert {"turboreg_create", "turboreg_register", "turboreg_register_batched", "turboreg_destroy"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    assert declared <= set(trg.EXPORTED)


def test_status_strings_and_defaults(lib):
    assert trg.status_string(trg.OK) == "ok"
    assert "hypothesis" in trg.status_string(trg.ERR_NO_HYPOTHESIS)
    p = trg.default_params(0.1, 2000, 0.1)
    assert p.k2 == 2 and p.graph_mode == trg.GRAPH_O2 and p.proposal == trg.PROPOSAL_PLAIN
    assert abs(p.kappa_fp64 - 100.0) < 1e-6 and p.k1 == 2000


def test_invalid_arguments_rejected_on_host(lib):
    h = ctypes.c_void_p()
    assert lib.turboreg_create(0, 2, 1, None, ctypes.byref(h)) == trg.ERR_INVALID_ARG
    assert lib.turboreg_create(0, trg.TURBOREG_MAX_N + 1, 1, None, ctypes.byref(h)) == trg.ERR_INVALID_ARG
    assert lib.turboreg_create(0, 1000, 0, None, ctypes.byref(h)) == trg.ERR_INVALID_ARG
    assert lib.turboreg_create(0, 1000, 1, None, None) == trg.ERR_INVALID_ARG
    out = trg.turboreg_result()
    p = trg.default_params(0.1, 10, 0.1)
    assert lib.turboreg_register(None, None, None, 10, ctypes.byref(p), ctypes.byref(out)) == trg.ERR_INVALID_ARG
    assert lib.turboreg_register_batched(None, None, None, None, 1, ctypes.byref(p), 1,
                                         ctypes.byref(out)) == trg.ERR_INVALID_ARG
    lib.turboreg_destroy(None)   # NULL-safe


def test_package_refuses_to_run_without_library(tmp_path):
    import importlib
    mod = importlib.import_module("paper_2507_01439_gb300")
    with pytest.raises(RuntimeError):
        mod._lib = None
        try:
            mod.load_library(str(tmp_path / "missing.so"))
        finally:
            mod._lib = None
