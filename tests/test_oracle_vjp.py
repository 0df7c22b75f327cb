"""Pins of the oracle's backward pass (Eq. 3, Eq. 7, Algorithm 3) against central finite
differences of the loss: exact for affine dynamics (LQ) with the Gauss-Newton KKT matrix,
and exact on nonlinear dynamics with the exact-Hessian KKT matrix; the Gauss-Newton gap on
nonlinear dynamics (Sec. 3.4) is measured, not gated."""
import numpy as np
import pytest

from paper_2510_06179_gb300 import workloads
from oracle import ocp as O
from oracle.backward import vjp
from oracle.fd import fd_gradient
from oracle.sqp import sqp, solve_to_convergence, newton_kkt
from tests.oracle_helpers import to_ocp


def _loss_factory(ocp, rng):
    wz = rng.standard_normal(ocp.n)

    def loss(z):
        return 0.5 * np.sum(wz * z * z) + np.sum(np.sin(z[: ocp.nx + ocp.nu]))

    def grad(z):
        g = wz * z
        g[: ocp.nx + ocp.nu] += np.cos(z[: ocp.nx + ocp.nu])
        return g
    return loss, grad


def test_vjp_matches_fd_lq_all_parameters():
    """LQ: dl/dtheta over Q, R, Q_T, A_t, B_t, c_t, and dl/dx_s, vs central differences."""
    w = workloads.lq_config(B=1, T=6, nx=3, nu=2, seed=21, c_var=0.01)
    ocp = to_ocp(w)
    rng = np.random.default_rng(0)
    loss, grad = _loss_factory(ocp, rng)
    out = sqp(ocp, 1, line_search_on=False)
    z, lam = out["z"], out["lam"]
    res = vjp(ocp, z, lam, grad(z[0])[None])
    fd = fd_gradient(ocp, loss, z, lam, rel_step=1e-5)
    scale = np.abs(fd).max()
    np.testing.assert_allclose(res["dtheta"][0], fd, atol=1e-7 * scale, rtol=1e-6)
    fdx = fd_gradient(ocp, loss, z, lam, rel_step=1e-5, wrt="x_s")
    np.testing.assert_allclose(res["dxs"][0], fdx, rtol=1e-6, atol=1e-8 * np.abs(fdx).max())


def test_vjp_exact_hessian_matches_fd_cartpole():
    """Nonlinear cart-pole at a converged solution: the IFT gradient with the exact Lagrangian
    Hessian equals finite differences (validates dF/dtheta, incl. the mixed lambda^T d2f term)."""
    w = workloads.cartpole_config(B=1, T=12, seed=3)
    w.x_s[:, 2] *= 0.2
    ocp = to_ocp(w)
    z, lam = solve_to_convergence(ocp, tol=1e-14, warm_iters=30)
    rng = np.random.default_rng(1)
    loss, grad = _loss_factory(ocp, rng)
    ex = vjp(ocp, z, lam, grad(z[0])[None], hessian="exact")
    gn = vjp(ocp, z, lam, grad(z[0])[None], hessian="gn")
    fd = fd_gradient(ocp, loss, z, lam, rel_step=1e-6, tol=1e-15)
    scale = np.abs(fd).max()
    np.testing.assert_allclose(ex["dtheta"][0], fd, atol=2e-6 * scale, rtol=1e-5)
    fdx = fd_gradient(ocp, loss, z, lam, rel_step=1e-6, wrt="x_s", tol=1e-15)
    np.testing.assert_allclose(ex["dxs"][0], fdx, rtol=1e-5, atol=2e-6 * np.abs(fdx).max())
    # Gauss-Newton gradients differ (Sec. 3.4), but only by the dynamics-curvature term.
    gap = np.linalg.norm(gn["dtheta"][0] - fd) / np.linalg.norm(fd)
    assert 0.0 < gap < 1.0


def _fiala_kink_distance(ocp, z):
    """Smallest distance (rad) of a front or rear slip angle from the Fiala full-slide angle
    alpha_sl = atan(3 mu Fz / C_alpha), over the knots of the single-track OCP."""
    mdl = ocp.model
    x, u = O.split_z(ocp, z)
    x, u = x[0], u[0]
    mu, ca = ocp.theta[0, :2]
    a, b, m, g = mdl.a, mdl.b, mdl.m, 9.81
    af = np.arctan((x[:-1, 4] + a * x[:-1, 3]) / x[:-1, 5]) - u[:, 0]
    ar = np.arctan((x[:-1, 4] - b * x[:-1, 3]) / x[:-1, 5])
    sl_f = np.arctan(3 * mu * m * g * b / (a + b) / ca)
    sl_r = np.arctan(3 * mu * m * g * a / (a + b) / ca)
    return min(np.abs(sl_f - np.abs(af)).min(), np.abs(sl_r - np.abs(ar)).min())


@pytest.mark.parametrize("seed", [1, 2])
def test_vjp_exact_hessian_matches_fd_vehicle(seed):
    """Single-track vehicle with Fiala tyres (the vehicle workload, T 20): at a KKT point (SQP
    with the line search, then Newton-KKT to machine precision) whose slip angles stay away from
    the Fiala full-slide kink, the exact-Hessian IFT gradient over every theta entry (friction,
    cornering stiffness, cost weights) and x_s equals central differences.  Differences use
    steps relative to each entry (the drive-force weight is ~1e-6) and Newton-KKT re-solves (the
    Gauss-Newton iteration does not contract at these points).  The Gauss-Newton gradient's gap
    to the differences (Sec. 3.4 leaves the dynamics curvature out) is printed, not gated."""
    w = workloads.vehicle_config(B=1, T=20, seed=seed)
    ocp = to_ocp(w)
    out = sqp(ocp, 60)
    z, lam, step, _ = newton_kkt(ocp, out["z"], out["lam"])
    Fz, Fl = O.kkt_residual(ocp, z, lam)
    assert max(np.abs(Fz).max(), np.abs(Fl).max()) <= 1e-10
    assert _fiala_kink_distance(ocp, z) >= 1e-3     # sample away from the non-differentiable kink
    rng = np.random.default_rng(1)
    loss, grad = _loss_factory(ocp, rng)
    ex = vjp(ocp, z, lam, grad(z[0])[None], hessian="exact")
    gn = vjp(ocp, z, lam, grad(z[0])[None], hessian="gn")
    fd = fd_gradient(ocp, loss, z, lam, rel_step=1e-5, step="relative", solver="newton")
    scale = np.maximum(np.abs(fd), 1e-3 * np.abs(fd).max())
    assert (np.abs(ex["dtheta"][0] - fd) / scale).max() <= 1e-5
    fdx = fd_gradient(ocp, loss, z, lam, rel_step=1e-6, wrt="x_s", solver="newton")
    np.testing.assert_allclose(ex["dxs"][0], fdx, rtol=1e-5, atol=1e-6 * np.abs(fdx).max())
    gap = np.linalg.norm(gn["dtheta"][0] - fd) / np.linalg.norm(fd)
    print(f"vehicle seed {seed}: exact-Hessian vs FD max {(np.abs(ex['dtheta'][0] - fd) / scale).max():.1e}, "
          f"Gauss-Newton vs FD {gap:.2f} (relative)")
    assert gap > 0.0


def test_vjp_gn_equals_exact_for_affine_dynamics():
    w = workloads.lq_config(B=2, T=8, seed=5, c_var=0.01)
    ocp = to_ocp(w)
    out = sqp(ocp, 1, line_search_on=False)
    g = np.random.default_rng(2).standard_normal((2, ocp.n))
    a = vjp(ocp, out["z"], out["lam"], g, hessian="gn")
    b = vjp(ocp, out["z"], out["lam"], g, hessian="exact")
    np.testing.assert_allclose(a["dtheta"], b["dtheta"], rtol=1e-10, atol=1e-12)


_DF_CASES = {
    "cartpole": lambda: workloads.cartpole_config(B=1, T=5, seed=9),
    "kin_bicycle": lambda: workloads.bicycle_config(B=1, T=5, seed=9),
    "pendulum": lambda: workloads.pendulum_config(B=1, T=5, seed=9),
    "attitude": lambda: workloads.attitude_config(B=1, T=5, seed=9),
    "rigid_body12": lambda: workloads.rigid_body_config(B=1, T=5, seed=9),
    "single_track": lambda: workloads.vehicle_config(B=1, T=5, seed=9),
}


@pytest.mark.parametrize("name", list(_DF_CASES))
def test_dF_dtheta_matches_differenced_residual(name):
    """dF/dtheta (assembled from jets) vs central differences of F(z, lambda, theta) (Eq. 1), at
    a point near the workload's reference (random perturbation) with random multipliers; the
    bicycle and the vehicle track nonzero references, which enter the cost-weight columns, and
    the vehicle's friction and cornering-stiffness columns come from the Fiala tyre curve."""
    from oracle.backward import dF_dtheta
    w = _DF_CASES[name]()
    ocp = to_ocp(w)
    rng = np.random.default_rng(4)
    x_ref = np.asarray(w.x_ref[0], np.float64)
    u0 = np.zeros((ocp.T, ocp.nu))
    z = O.join_z(x_ref[None], u0[None]) + 0.05 * rng.standard_normal((1, ocp.n))
    if name not in ("single_track",):
        z = z + 0.45 * rng.standard_normal((1, ocp.n))
    lam = rng.standard_normal((1, ocp.m))
    M = dF_dtheta(ocp, z, lam, 0)
    for j in range(ocp.p):
        h = 1e-6 * max(1.0, abs(ocp.theta[0, j]))
        tp, tm = ocp.theta.copy(), ocp.theta.copy()
        tp[0, j] += h
        tm[0, j] -= h
        Fp = np.concatenate(O.kkt_residual(O.OCPBatch(ocp.model, ocp.T, ocp.x_s, tp, ocp.x_ref), z, lam), 1)
        Fm = np.concatenate(O.kkt_residual(O.OCPBatch(ocp.model, ocp.T, ocp.x_s, tm, ocp.x_ref), z, lam), 1)
        fd = (Fp - Fm)[0] / (2 * h)
        np.testing.assert_allclose(M[:, j], fd, atol=1e-6 * max(1.0, np.abs(fd).max()))
