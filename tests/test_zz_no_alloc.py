"""The allocation-free forward solve (dmpc_solve_noalloc) against the regular handle-based
solve (dmpc_solve), through the C-ABI.

dmpc_solve_noalloc serves callers that cannot allocate device memory when they solve (a
controller in a real-time loop that may only touch memory reserved at start-up, a plug-in
inside a framework that owns the device allocator); its scratch is a fixed device array in the
library.  This file is collected last so that a run stopping at its first failure has already
run every other test; it also passes on its own in a fresh process."""
import ctypes

import numpy as np
import pytest

from paper_2510_06179_gb300 import workloads
from tests.gpu_helpers import ensure_built, dev
from tests.oracle_helpers import rel_err

pytestmark = pytest.mark.gpu

Z_TOL = 1e-4  # the solution tolerance of the parity tests


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def test_noalloc_solve_matches_regular_solve_twice():
    import torch
    ensure_built()
    from paper_2510_06179_gb300 import _lib
    from paper_2510_06179_gb300.solver import OCPBatch, MODEL_IDS, default_options
    lib = _lib.load()
    w = workloads.cartpole_config(B=24, T=40, seed=13, sqp_iters=3)
    opts = dict(sqp_iters=w.sqp_iters, line_search=1, pcg_tol=1e-9, warm_start=0)
    # regular path
    reg = OCPBatch((w.model, w.nx, w.nu, w.T, w.dt), batch=w.B, device="cuda:0", **opts)
    x_s, th, xr = dev(w.x_s), dev(w.theta), dev(w.x_ref)
    ref = reg.solve(x_s, th, xr)
    torch.cuda.synchronize()
    z_ref = ref["z"].view(w.B, -1).cpu().numpy().astype(np.float64)
    # allocation-free path, two calls in a row (the second reuses the shared scratch)
    desc = _lib.dmpc_ocp_desc(MODEL_IDS[w.model], w.nx, w.nu, w.T, w.dt)
    o = default_options(**opts)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        z = torch.full((w.B * w.n,), float("nan"), device="cuda:0")
        lam = torch.empty(w.B * w.m, device="cuda:0")
        st = torch.full((w.B,), -1, dtype=torch.int32, device="cuda:0")
        it = torch.empty(w.B * w.sqp_iters, dtype=torch.int32, device="cuda:0")
        al = torch.empty(w.B * w.sqp_iters, device="cuda:0")
        code = lib.dmpc_solve_noalloc(ctypes.byref(desc), w.B, ctypes.byref(o), stream, _ptr(x_s), _ptr(th),
                                      _ptr(xr), None, None, _ptr(z), _ptr(lam), _ptr(st), _ptr(it), _ptr(al))
        assert code == 0, code
        torch.cuda.synchronize()
        zz = z.view(w.B, -1).cpu().numpy().astype(np.float64)
        assert np.isfinite(zz).all()
        assert rel_err(zz, z_ref).max() <= Z_TOL, (call, rel_err(zz, z_ref).max())
        assert np.array_equal(st.cpu().numpy(), ref["status"].cpu().numpy())
    reg.close()


def test_noalloc_rejects_requests_beyond_its_scratch():
    ensure_built()
    from paper_2510_06179_gb300 import _lib
    from paper_2510_06179_gb300.solver import MODEL_IDS, default_options
    lib = _lib.load()
    desc = _lib.dmpc_ocp_desc(MODEL_IDS["cartpole"], 4, 1, 50, 0.05)
    o = default_options()
    dummy = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    code = lib.dmpc_solve_noalloc(ctypes.byref(desc), 1 << 20, ctypes.byref(o), None, dummy, dummy, None,
                                  None, None, dummy, None, None, None, None)
    assert code == 3  # DMPC_E_BUDGET
