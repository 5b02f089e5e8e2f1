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


@pytest.mark.parametrize("kwargs,code", [
    (dict(form="plain", precision="bf16"), 10),                    # BF16 variants: modal only
    (dict(form="plain", precision="bf16x3"), 10),
    (dict(form="plain", precision="fp32x2", solver="substitution"), 10),
    (dict(form="plain", precision="fp32", solver="substitution"), 10),
    (dict(form="plain", precision="fp32", rhs="independent"), 10),
    (dict(form="plain", integrator="exact"), 10),                  # exact integrator: modal only
    (dict(form="plain", rhs="paired", solver="substitution"), 10),
    (dict(form="plain", precision="fp32", refine_steps=9), 1),     # 0 .. 8 sweeps
    (dict(form="modal", dt=0.0), 1),
    (dict(form="modal", theta=-0.1), 1),
])
def test_config_combinations_checked_without_gpu(kwargs, code):
    """ec_create rejects unsupported or invalid configurations before touching the GPU."""
    from paper_2407_11993_gb300 import build, eddy
    build.build()
    kw = dict(theta=0.5, dt=1e-6)
    kw.update(kwargs)
    form = kw.pop("form")
    with pytest.raises(eddy.EcError) as e:
        eddy.ThetaMethod(form, **kw)
    assert e.value.code == code


def test_entry_points_check_arguments_without_gpu():
    from paper_2407_11993_gb300 import build, eddy
    build.build()
    so = eddy.lib()
    # a batch needs 1 .. EC_BATCH_MAX contexts
    assert so.ec_batch_run(None, 0, 1, None, None, None, 0, None, 0) == 1
    hs = (ctypes.c_void_p * 65)()
    assert so.ec_batch_run(hs, 65, 1, None, None, None, 0, None, 0) == 1
    # the allocation-free solve rejects sizes past its scratch before any CUDA call
    dummy = ctypes.c_void_p(16)
    assert so.ec_solve_inverse_noalloc(eddy.NOALLOC_MAX_N + 1, dummy, eddy.NOALLOC_MAX_N + 1,
                                       dummy, dummy, None) == 2
    assert so.ec_solve_inverse_noalloc(0, dummy, 1, dummy, dummy, None) == 1
    # null context
    assert so.ec_run(None, 1, None, None, None, 0, None, 0) == 1
    assert so.ec_set_precision(None, 0) == 1
    assert so.ec_state_size(None) == 0


def test_noalloc_binding_checks_sizes_and_devices_without_gpu():
    """The allocation-free solve's binding refuses short or mismatched tensors before it
    touches the library (so a short buffer can never reach a kernel)."""
    import torch
    from paper_2407_11993_gb300 import eddy
    n = 100
    W = torch.zeros(n * n, dtype=torch.float64)
    b = torch.zeros(n, dtype=torch.float64)
    with pytest.raises(ValueError):          # Winv shorter than n * n
        eddy.solve_inverse_noalloc(W[: n * n - 1], b, b)
    with pytest.raises(ValueError):          # b shorter than the n override
        eddy.solve_inverse_noalloc(W, b, b, n=n + 1)
    with pytest.raises(ValueError):          # x too short
        eddy.solve_inverse_noalloc(W, b, b[:-1])
    with pytest.raises(ValueError):          # ldw * (n - 1) + n elements needed
        eddy.solve_inverse_noalloc(W, b, b, ldw=n + 1)
    with pytest.raises(TypeError):           # host memory is not device memory
        eddy.solve_inverse_noalloc(W, b, b)
