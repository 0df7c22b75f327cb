"""Implicit (trapezoidal) integrator on the GPU: A^+ != I in the linearisation, the Schur blocks
and gamma (Eq. 4, 10), the FP64 and double-float operators, the line search's constraint
residual and the theta contraction.  Checked against the FP64 oracle's implicit path: the QP
building blocks at a random point, SQP solutions under the step-size path protocol, gradients
at the GPU's own solution, and the plain form against the fused one."""
import numpy as np
import pytest

from paper_2510_06179_gb300 import workloads
from tests.gpu_helpers import gpu_solve, dev
from tests.oracle_helpers import rel_err
from tests.test_gpu_parity import _check_inspect, _nonlinear_forward, _grad_check

pytestmark = pytest.mark.gpu


def test_inspect_implicit_cartpole_blocks():
    w = workloads.cartpole_config(B=16, T=40, seed=3, integrator="trapezoid")
    rng = np.random.default_rng(1)
    z = (0.3 * rng.standard_normal((w.B, w.n))).astype(np.float32)
    lam = (0.1 * rng.standard_normal((w.B, w.m))).astype(np.float32)
    _check_inspect(w, z, lam, 2e-5)


@pytest.mark.parametrize("maker", [workloads.pendulum_config, workloads.cartpole_config])
def test_implicit_forward_and_gradient_parity(maker):
    w = maker(B=32, T=40, seed=4, sqp_iters=6, integrator="trapezoid")
    b, g, ref = _nonlinear_forward(w)
    _grad_check(w, b, g)
    b.close()


@pytest.mark.parametrize("team", [32, 128])
def test_implicit_tilings_and_double_float_agree(team):
    """Register (single warp) and multi-warp paths, and the double-float PCG, on the same OCPs."""
    w = workloads.cartpole_config(B=16, T=50, seed=6, sqp_iters=4, integrator="trapezoid")
    b0, g0 = gpu_solve(w, team_threads=team)
    b1, g1 = gpu_solve(w, team_threads=team, pcg_precision=1)
    same = np.all(g0["alpha"] == g1["alpha"], axis=1)
    assert same.mean() >= 0.75
    assert rel_err(g0["z"][same], g1["z"][same]).max() <= 1e-4
    b0.close()
    b1.close()


def test_implicit_plain_form_matches_fused_form():
    import torch
    w = workloads.pendulum_config(B=16, T=30, seed=8, sqp_iters=3, integrator="trapezoid")
    b, g = gpu_solve(w, warm_start=0)
    zp = b.solve(dev(w.x_s), dev(w.theta), dev(w.x_ref), plain=True)
    torch.cuda.synchronize()
    zz = zp["z"].view(w.B, -1).cpu().numpy().astype(np.float64)
    assert np.array_equal(zp["alpha"].view(w.B, -1).cpu().numpy(), g["alpha"])
    assert rel_err(zz, g["z"]).max() <= 1e-5
    b.close()


def test_implicit_rejected_with_exact_hessian():
    from paper_2510_06179_gb300 import _lib
    w = workloads.pendulum_config(B=2, T=10, seed=1, integrator="trapezoid")
    with pytest.raises(_lib.DMPCError):
        gpu_solve(w, exact_hessian=1)
