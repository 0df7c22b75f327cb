"""Parity at the benchmark's full sizes and launch configuration, on sampled OCPs the oracle
solves one by one: cart-pole (256 OCPs, T 50, 10 SQP iterations, tolerance 1e-7, default tiling,
solution and gradient) and the single-track vehicle (1024 OCPs, T 100).  Replay protocol: every
sampled OCP's step sizes are consistent with the oracle's tests and its solution is within the
gate of the FP64 oracle replaying them."""
import numpy as np
import pytest

from paper_2510_06179_gb300 import workloads
from oracle.backward import vjp as oracle_vjp
from tests.gpu_helpers import gpu_solve, gpu_vjp
from tests.oracle_helpers import to_ocp, rel_err, replay_check, assert_replay_parity

pytestmark = pytest.mark.gpu


def _sampled(name, w, g, idx):
    res = replay_check(w.subset(idx), g["z"][idx], g["alpha"][idx])
    assert_replay_parity(name, res, 1e-4)
    return res


def test_cartpole_bench_configuration_sampled():
    w = workloads.cartpole_config(B=256, T=50, seed=1000, sqp_iters=10)
    b, g = gpu_solve(w, pcg_tol=1e-7, warm_start=0)
    idx = np.random.default_rng(0).choice(256, size=24, replace=False)
    _sampled("cart-pole 256", w, g, idx)
    sub = w.subset(idx)
    # gradient at the GPU's solution (the backward isolated from the forward's error)
    dl = w.dl_dz(g["z"])
    gv = gpu_vjp(b, w, dl)
    gref = oracle_vjp(to_ocp(sub), g["z"][idx], g["lam"][idx], dl[idx])
    ge = rel_err(gv["dtheta"][idx], gref["dtheta"])
    print(f"cart-pole 256: sampled gradient max err {ge.max():.2e}")
    assert ge.max() <= 1e-3
    b.close()


def test_vehicle_full_batch_sampled():
    w = workloads.vehicle_config(B=1024, T=100, seed=0, sqp_iters=10)
    b, g = gpu_solve(w, pcg_tol=1e-7, warm_start=0)
    idx = np.random.default_rng(1).choice(1024, size=12, replace=False)
    _sampled("vehicle 1024", w, g, idx)
    assert not (g["status"] & (1 | 2 | 8)).any()
    b.close()
