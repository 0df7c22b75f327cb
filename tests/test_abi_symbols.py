"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every function
include/dmpc.h declares; the ctypes binding declares the same names."""
import ctypes
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dmpc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dmpc_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("dmpc_create_problem_batch", "dmpc_solve", "dmpc_vjp", "dmpc_destroy"):
        assert required in names


def test_library_loads_and_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_06179_gb300 import _lib
    lib = ctypes.CDLL(_lib.LIB_PATH)
    for name in _declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(dmpc_[a-z0-9_]+)\b", out))
    assert set(_declared()) <= exported
    assert set(_lib.SIGNATURES) == set(_declared())


def test_library_reports_version_and_default_options_without_gpu():
    from paper_2510_06179_gb300 import _lib
    lib = _lib.load()
    assert b"sm_103a" in lib.dmpc_version()
    o = _lib.dmpc_options()
    lib.dmpc_default_options(ctypes.byref(o))
    assert o.n_alpha == 5 and abs(o.alpha[4] - 0.01) < 1e-9 and abs(o.ls_eta - 0.4) < 1e-7
    assert o.sqp_iters == 1 and o.warm_start == 1


def test_create_rejects_bad_arguments_before_touching_the_gpu():
    from paper_2510_06179_gb300 import _lib
    lib = _lib.load()
    h = ctypes.c_void_p()
    assert lib.dmpc_create_problem_batch(None, 1, None, None, ctypes.byref(h)) == 1
    assert h.value is None
    assert lib.dmpc_vjp(None, None, None, None, None, None, None) == 1


def test_product_path_fails_loudly_without_the_library():
    """No CPU fallback: with the CUDA library absent, creating a batch raises at once."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("from paper_2510_06179_gb300.solver import OCPBatch\n"
            "OCPBatch(('cartpole', 4, 1, 10, 0.05), batch=2, device='cpu')\n")
    env = dict(os.environ, DMPC_LIB=os.path.join(root, "_no_such_dir", "libdmpc.so"))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode != 0
    assert "CUDA library not built" in r.stderr


def test_reference_requiring_grad_is_rejected():
    """The backward returns gradients for x_s and theta only, so a reference that asks for one
    is refused before any solve (checked without a GPU: the batch is never touched)."""
    import pytest
    import torch
    from paper_2510_06179_gb300.solver import DiffMPCFunction
    x_s = torch.zeros(4)
    theta = torch.zeros(7, requires_grad=True)
    x_ref = torch.zeros(8, requires_grad=True)
    with pytest.raises(ValueError, match="x_ref"):
        DiffMPCFunction.apply(x_s, theta, object(), x_ref, None)
