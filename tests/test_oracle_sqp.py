"""Pins of the oracle's SQP (Algorithm 2) and line search (Algorithm 5): closed-form merit
decrease on feasible convex problems, convergence to a KKT point (Eq. 1), and the
special cases the reading of the penalty parameter fixes."""
import numpy as np

from paper_2510_06179_gb300 import workloads
from oracle import ocp as O
from oracle.sqp import sqp, line_search, cold_start, LS_ALPHAS, solve_to_convergence
from tests.oracle_helpers import to_ocp


def _feasible_rollout(ocp, rng):
    """A dynamically feasible z: roll the dynamics forward from x_s with random inputs."""
    u = 0.3 * rng.standard_normal((ocp.B, ocp.T, ocp.nu))
    x = np.zeros((ocp.B, ocp.K, ocp.nx))
    x[:, 0] = ocp.x_s
    for t in range(ocp.T):
        x[:, t + 1] = O.dynamics_values(ocp, x[:, t:t + 1], u[:, t:t + 1], t0=t)[:, 0]
    return O.join_z(x, u)


def test_line_search_closed_form_on_feasible_lq():
    """At a feasible point of a convex LQ problem the penalty is 0 and, with the exact QP step
    Delta, num = -Delta^T G Delta, so Delta phi_alpha = alpha num (1 - alpha/2 - 0.4);
    every alpha in (0, 1] decreases the merit and the full step is taken."""
    w = workloads.lq_config(B=3, T=15, seed=11, c_var=0.01)
    ocp = to_ocp(w)
    rng = np.random.default_rng(3)
    z = _feasible_rollout(ocp, rng)
    qp = O.linearise(ocp, z)
    zp = np.stack([O.solve_qp(qp, b)[0] for b in range(ocp.B)])
    alpha, diag = line_search(ocp, z, zp)
    assert np.all(diag["mu"] == 0.0)
    num = np.einsum("bn,bn->b", O.cost_gradient(ocp, z), zp - z)
    assert np.all(num < 0)
    expect = np.array([[a * nb * (1 - a / 2 - 0.4) for a in LS_ALPHAS] for nb in num])
    np.testing.assert_allclose(diag["delta"], expect, rtol=1e-7, atol=1e-9)
    assert np.all(alpha == 1.0)


def test_line_search_penalty_formula_on_infeasible_start():
    """Away from feasibility mu = num / (0.5 ||g||_1) (Nocedal 18.33 with rho = 0.5) when num > 0,
    giving D_mu = -num; when num <= 0, mu = 0 and D_mu = num."""
    w = workloads.cartpole_config(B=8, T=20, seed=2)
    ocp = to_ocp(w)
    z, _ = cold_start(ocp)
    qp = O.linearise(ocp, z)
    zp = np.stack([O.solve_qp(qp, b)[0] for b in range(ocp.B)])
    _, diag = line_search(ocp, z, zp)
    num = np.einsum("bn,bn->b", O.cost_gradient(ocp, z), zp - z)
    g1 = np.abs(O.constraint_residual(ocp, z)).reshape(ocp.B, -1).sum(1)
    assert np.all(g1 > 1e-3)
    mu_expect = np.where(num > 0, num / (0.5 * g1), 0.0)
    np.testing.assert_allclose(diag["mu"], mu_expect, rtol=1e-12)
    np.testing.assert_allclose(diag["D"], np.where(num > 0, -num, num), rtol=1e-9, atol=1e-12)


def test_line_search_takes_smallest_step_when_nothing_decreases():
    """Algorithm 5: if no candidate passes, alpha = min(alpha set).  An ascent 'step' z+ = z - Delta."""
    w = workloads.lq_config(B=2, T=10, seed=4)
    ocp = to_ocp(w)
    z = _feasible_rollout(ocp, np.random.default_rng(0))
    qp = O.linearise(ocp, z)
    zp = np.stack([O.solve_qp(qp, b)[0] for b in range(ocp.B)])
    alpha, diag = line_search(ocp, z, 2 * z - zp)
    assert np.all(alpha == min(LS_ALPHAS))
    assert np.all(diag["delta"] >= 0)


def test_sqp_converges_to_kkt_point_cartpole():
    """SQP iterates reach F(z, lambda) = 0 (Eq. 1) on the nonlinear cart-pole."""
    w = workloads.cartpole_config(B=4, T=25, seed=5)
    w.x_s[:, 2] *= 0.3  # moderate initial angles so that every instance converges
    ocp = to_ocp(w)
    z, lam = solve_to_convergence(ocp, tol=1e-12, warm_iters=30)
    Fz, Fl = O.kkt_residual(ocp, z, lam)
    assert np.abs(Fz).max() < 1e-9
    assert np.abs(Fl).max() < 1e-11


def test_sqp_lq_fixed_point():
    """A second SQP step on an LQ problem does not move the solution (z, lambda)."""
    w = workloads.lq_config(B=2, T=10, seed=8, c_var=0.01)
    ocp = to_ocp(w)
    one = sqp(ocp, 1, line_search_on=False)
    two = sqp(ocp, 2, line_search_on=False)
    np.testing.assert_allclose(two["z"], one["z"], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(two["lam"], one["lam"], rtol=1e-9, atol=1e-11)
    three = sqp(ocp, 2, line_search_on=True)
    np.testing.assert_allclose(three["z"], one["z"], rtol=1e-10, atol=1e-12)
