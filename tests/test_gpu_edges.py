"""Edge cases on the GPU: the maximum horizon the boundary accepts (T = 4096, workspace in
global memory), a large batch (100 000 OCPs in one launch, sampled against the oracle), a
one-OCP batch with an implicit integrator and T = 1, and an empty subset launch of the serving
entry point (a no-op that leaves the resident state alone)."""
import ctypes

import numpy as np
import pytest

from paper_2510_06179_gb300 import workloads
from oracle.sqp import sqp as oracle_sqp
from tests.gpu_helpers import gpu_solve, alpha_paths_agree, dev
from tests.oracle_helpers import to_ocp, rel_err

pytestmark = pytest.mark.gpu


def test_maximum_horizon_matches_oracle():
    w = workloads.pendulum_config(B=2, T=4096, seed=3, sqp_iters=2)
    b, g = gpu_solve(w)
    assert b.get_tiling()["smem_bytes"] == 0            # global-memory workspace
    ref = oracle_sqp(to_ocp(w), w.sqp_iters, line_search_on=True)
    agree = alpha_paths_agree(g["alpha"], ref["alpha"])
    e = rel_err(g["z"], ref["z"])
    print(f"T=4096: agree {agree.sum()}/2 err {e}")
    assert agree.any() and e[agree].max() <= 1e-4
    assert not (g["status"] & (1 | 2 | 8)).any()
    b.close()


def test_large_batch_sampled_against_oracle():
    w = workloads.pendulum_config(B=100_000, T=8, seed=11, sqp_iters=2)
    b, g = gpu_solve(w)
    t = b.get_tiling()
    print(f"B=100000: tiling {t}")
    assert t["grid"] * t["teams_per_block"] >= w.B
    assert not (g["status"] & (1 | 2 | 8)).any()
    idx = np.concatenate([np.arange(3), np.random.default_rng(2).choice(w.B, size=5, replace=False), [w.B - 1]])
    sub = w.subset(idx)
    ref = oracle_sqp(to_ocp(sub), w.sqp_iters, line_search_on=True)
    agree = alpha_paths_agree(g["alpha"][idx], ref["alpha"])
    e = rel_err(g["z"][idx], ref["z"])
    print(f"B=100000: sampled {len(idx)}, agree {agree.sum()}, errors {e}")
    assert agree.sum() >= 6 and e[agree].max() <= 1e-4
    b.close()


def test_single_ocp_implicit_horizon_one():
    w = workloads.cartpole_config(B=1, T=1, seed=5, sqp_iters=2, integrator="trapezoid")
    b, g = gpu_solve(w)
    ref = oracle_sqp(to_ocp(w), w.sqp_iters, line_search_on=True)
    if alpha_paths_agree(g["alpha"], ref["alpha"]).all():
        assert rel_err(g["z"], ref["z"]).max() <= 1e-4
    b.close()


def test_empty_subset_is_a_no_op():
    import torch
    from paper_2510_06179_gb300 import _lib
    w = workloads.cartpole_config(B=4, T=20, seed=7, sqp_iters=2)
    b, g = gpu_solve(w)
    z_before = torch.from_numpy(g["z"].astype(np.float32).reshape(-1)).to("cuda:0")
    z_out = z_before.clone()
    idx = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    code = b.lib.dmpc_solve_subset(b.h, ptr(idx), 0, ptr(dev(w.x_s)), ptr(dev(w.theta)), ptr(dev(w.x_ref)),
                                   ptr(z_out), None, None, None, None)
    _lib.check(code, b.h)
    torch.cuda.synchronize()
    assert torch.equal(z_out, z_before)
    b.close()
