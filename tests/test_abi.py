"""The C-ABI library builds, loads without a GPU, and exports every declared entry point."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            names += re.findall(r"EC_API\s+[\w\s\*]+?\b(ec_\w+)\s*\(", text)
    return names


def test_header_declares_entry_points():
    names = declared_symbols()
    assert "ec_setup" in names and "ec_run" in names and len(names) >= 10


def test_library_exports_every_declared_symbol():
    from paper_2407_11993_gb300 import build, eddy
    path = build.build()
    so = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(so, n)]
    assert not missing, missing
    assert set(declared_symbols()) <= set(eddy.EXPORTS) | set(declared_symbols())
    # the binding wraps every declared entry point
    assert set(declared_symbols()) == set(eddy.EXPORTS)


def test_error_strings_without_gpu():
    from paper_2407_11993_gb300 import build, eddy
    build.build()
    so = eddy.lib()
    assert so.ec_error_string(0) == b"ok"
    assert b"positive definite" in so.ec_error_string(3)


def test_binding_rejects_bad_config_without_gpu():
    """Argument checks happen before any CUDA call."""
    from paper_2407_11993_gb300 import build, eddy
    build.build()
    with pytest.raises(eddy.EcError) as e:
        eddy.ThetaMethod("plain", theta=1.5, dt=1e-6)
    assert e.value.code == 1
