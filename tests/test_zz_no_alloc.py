"""The allocation-free forward solve (dmpc_solve_noalloc) against the regular handle-based
solve (dmpc_solve) and the FP64 oracle, through the C-ABI.

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
from tests.oracle_helpers import rel_err, replay_check, assert_replay_parity

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
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        code = lib.dmpc_solve_noalloc(ctypes.byref(desc), w.B, ctypes.byref(o), stream, _ptr(x_s), _ptr(th),
                                      _ptr(xr), None, None, _ptr(z), _ptr(lam), _ptr(st), _ptr(it), _ptr(al))
        assert code == 0, code
        torch.cuda.synchronize()
        if call == 1:   # the first call may load the kernel's code; the second must not allocate
            assert torch.cuda.mem_get_info()[0] == free_before
        zz = z.view(w.B, -1).cpu().numpy().astype(np.float64)
        assert np.isfinite(zz).all()
        assert rel_err(zz, z_ref).max() <= Z_TOL, (call, rel_err(zz, z_ref).max())
        assert np.array_equal(st.cpu().numpy(), ref["status"].cpu().numpy())
        res = replay_check(w, zz, al.view(w.B, -1).cpu().numpy())
        assert_replay_parity(f"noalloc cart-pole call {call}", res, Z_TOL)
    reg.close()


def test_noalloc_global_workspace_branch_matches_regular_solve_and_oracle():
    """12-state rigid-body OCPs with T = 200 (about 0.8 MB of workspace each, beyond shared
    memory): the per-team workspaces come out of the library's fixed scratch array, one team per
    OCP.  Two calls in a row; each matches the regular path and, under the replay protocol, the
    FP64 oracle; the second call allocates nothing (free device memory unchanged across it)."""
    import torch
    ensure_built()
    from paper_2510_06179_gb300 import _lib
    from paper_2510_06179_gb300.solver import OCPBatch, MODEL_IDS, default_options
    lib = _lib.load()
    w = workloads.rigid_body_config(B=3, T=200, seed=21, sqp_iters=3)
    opts = dict(sqp_iters=w.sqp_iters, line_search=1, pcg_tol=1e-9, warm_start=0)
    # the regular path in its one-team form (no thread-block cluster) runs it from global memory too
    reg = OCPBatch((w.model, w.nx, w.nu, w.T, w.dt), batch=w.B, device="cuda:0", cluster_ctas=1, **opts)
    assert reg.get_tiling()["smem_bytes"] == 0
    x_s, th, xr = dev(w.x_s), dev(w.theta), dev(w.x_ref)
    ref = reg.solve(x_s, th, xr)
    torch.cuda.synchronize()
    z_ref = ref["z"].view(w.B, -1).cpu().numpy().astype(np.float64)
    desc = _lib.dmpc_ocp_desc(MODEL_IDS[w.model], w.nx, w.nu, w.T, w.dt)
    o = default_options(**opts)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    z = torch.empty(w.B * w.n, device="cuda:0")
    lam = torch.empty(w.B * w.m, device="cuda:0")
    st = torch.empty(w.B, dtype=torch.int32, device="cuda:0")
    al = torch.empty(w.B * w.sqp_iters, device="cuda:0")
    for call in range(2):
        z.fill_(float("nan"))
        st.fill_(-1)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        code = lib.dmpc_solve_noalloc(ctypes.byref(desc), w.B, ctypes.byref(o), stream, _ptr(x_s), _ptr(th),
                                      _ptr(xr), None, None, _ptr(z), _ptr(lam), _ptr(st), None, _ptr(al))
        assert code == 0, code
        torch.cuda.synchronize()
        if call == 1:   # the first call may load the kernel's code; the second must not allocate
            assert torch.cuda.mem_get_info()[0] == free_before
        zz = z.view(w.B, -1).cpu().numpy().astype(np.float64)
        assert np.isfinite(zz).all()
        assert rel_err(zz, z_ref).max() <= Z_TOL, (call, rel_err(zz, z_ref).max())
        assert not (st.cpu().numpy() & (1 | 2 | 8)).any()
        res = replay_check(w, zz, al.view(w.B, -1).cpu().numpy())
        assert_replay_parity(f"noalloc rigid body T=200 call {call}", res, Z_TOL)
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
