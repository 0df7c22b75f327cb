"""Pins of the oracle's implicit (trapezoidal) dynamics, the general-A^+ case of Eq. 4 and 10:
second-order convergence of the rule itself, the linearisation (A, B, A^+, C) against central
differences of the constraint residual, KKT stationarity at a converged SQP solution, the
Schur/preconditioner path with A^+ != I against the direct KKT solve, and the implicit-function
gradient (with dF/dtheta of the implicit constraint) against finite differences of the
converged solution, the exact KKT matrix being formed by differencing the KKT residual."""
import numpy as np
import pytest

from paper_2510_06179_gb300 import workloads
from oracle import ocp as O
from oracle import schur as S
from oracle.backward import dF_dtheta
from oracle.models import make_model, rk4
from oracle.sqp import sqp, solve_to_convergence
from tests.oracle_helpers import to_ocp


def _trap_solve(model, x, u, ths):
    """x_{t+1} from f_t(x, u, x_{t+1}) = 0 by Newton's method with the oracle's A^+ = df/dx_{t+1}."""
    from oracle.jet import Jet
    xn = np.array(x, dtype=float)
    for _ in range(30):
        k = model.nx
        xs = [Jet.seed(np.array([xn[i]]), i, k) for i in range(k)]
        out = model.residual([np.array([v]) for v in x], [np.array([v]) for v in u], xs,
                             [np.array([v]) for v in ths], [])
        r = np.array([o.v[0] for o in out])
        J = np.array([o.g[0] for o in out])
        step = np.linalg.solve(J, r)
        xn = xn - step
        if np.abs(step).max() < 1e-14:
            break
    return xn


def test_trapezoid_rule_is_second_order():
    """Pendulum over 1 s: the trapezoidal trajectory's error against a fine RK4 reference drops
    by ~4x when dt halves (a dropped term or sign in the residual breaks the order)."""
    m_ref = make_model("pendulum", dt=1e-4)
    ths, x0, u = [1.0, 0.8], np.array([0.9, -0.3]), [0.2]

    def run(model, n):
        x = x0.copy()
        for _ in range(n):
            if model.implicit:
                x = _trap_solve(model, list(x), u, ths)
            else:
                x = np.array([v for v in rk4(model.fc, list(x), u, ths, model.dt)])
        return x
    ref = run(m_ref, 10000)
    errs = []
    for dt in (0.05, 0.025, 0.0125):
        m = make_model("pendulum", dt=dt, integrator="trapezoid")
        errs.append(np.linalg.norm(run(m, int(round(1.0 / dt))) - ref))
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(3.6 < r < 4.4 for r in ratios), (errs, ratios)


@pytest.mark.parametrize("maker", [workloads.pendulum_config, workloads.cartpole_config])
def test_implicit_linearisation_matches_differences(maker):
    """A_t, B_t, A_t^+ are the Jacobians of f_t, and C_t = A^+ x_{t+1} + A x_t + B u_t - f_t."""
    w = maker(B=1, T=4, seed=2, integrator="trapezoid")
    ocp = to_ocp(w)
    rng = np.random.default_rng(0)
    z = rng.standard_normal((1, ocp.n)) * 0.5
    qp = O.linearise(ocp, z)
    nx, nu, T = ocp.nx, ocp.nu, ocp.T
    g0 = O.constraint_residual(ocp, z)[0]
    h = 1e-6
    for t in range(T):
        for kind, idx, mat in (("x", O.x_index(nx, nu, t), qp.A[0, t]), ("u", O.u_index(nx, nu, t), qp.Bm[0, t]),
                               ("xn", O.x_index(nx, nu, t + 1), qp.Ap[0, t])):
            for j, col in enumerate(idx):
                zp, zm = z.copy(), z.copy()
                zp[0, col] += h
                zm[0, col] -= h
                d = (O.constraint_residual(ocp, zp)[0, t + 1] - O.constraint_residual(ocp, zm)[0, t + 1]) / (2 * h)
                np.testing.assert_allclose(mat[:, j], d, rtol=1e-6, atol=1e-8)
    assert np.abs(qp.Ap[0] - np.eye(nx)).max() > 1e-3        # a genuinely general A^+
    x, u = O.split_z(ocp, z)
    C = (np.einsum("tij,tj->ti", qp.Ap[0], x[0, 1:]) + np.einsum("tij,tj->ti", qp.A[0], x[0, :-1])
         + np.einsum("tij,tj->ti", qp.Bm[0], u[0]) - g0[1:])
    np.testing.assert_allclose(qp.C[0], C, rtol=1e-12, atol=1e-12)


def test_implicit_schur_pcg_matches_direct_solve():
    """With A^+ != I the Schur blocks, gamma, the stair preconditioner, PCG and the recovery
    reproduce the direct KKT solution of the QP."""
    w = workloads.cartpole_config(B=2, T=8, seed=4, integrator="trapezoid")
    ocp = to_ocp(w)
    z = sqp(ocp, 2)["z"]
    qp = O.linearise(ocp, z)
    D, Ob = S.schur_blocks(qp)
    Pd, Po = S.preconditioner_blocks(D, Ob)
    gam = S.gamma_spd(qp)
    lam, it, _, _ = S.pcg(D, Ob, Pd, Po, gam, np.zeros_like(gam), 1e-28, 5000)
    zr = S.recover_primal(qp, lam)
    for b in range(ocp.B):
        zd, ld = O.solve_qp(qp, b)
        np.testing.assert_allclose(O.join_z(*zr)[b] if isinstance(zr, tuple) else zr[b], zd, rtol=1e-7, atol=1e-9)
        np.testing.assert_allclose(lam[b].ravel(), ld, rtol=1e-7, atol=1e-9)


def test_implicit_sqp_converges_to_a_kkt_point():
    w = workloads.pendulum_config(B=3, T=12, seed=5, integrator="trapezoid")
    w.x_s[:, 0] *= 0.3
    ocp = to_ocp(w)
    z, lam = solve_to_convergence(ocp, tol=1e-13, warm_iters=30)
    Fz, Fl = O.kkt_residual(ocp, z, lam)
    assert np.abs(Fl).max() < 1e-10
    assert np.abs(Fz).max() < 1e-8


def test_implicit_ift_gradient_matches_differences():
    """dl/dtheta = -(dF/dtheta)^T K^-1 [dl/dz; 0] with the exact KKT matrix (differenced from the
    KKT residual), against central differences of the loss of the re-converged solution."""
    w = workloads.pendulum_config(B=1, T=8, seed=7, integrator="trapezoid")
    w.x_s[:, 0] *= 0.3
    ocp = to_ocp(w)
    z, lam = solve_to_convergence(ocp, tol=1e-14, warm_iters=30)
    n, m = ocp.n, ocp.m
    rng = np.random.default_rng(3)
    wz = rng.standard_normal(n)
    loss = lambda zz: 0.5 * np.sum(wz * zz * zz)
    # exact KKT matrix by central differences of F(z, lambda)
    K = np.zeros((n + m, n + m))
    h = 1e-6
    v0 = np.concatenate([z[0], lam[0]])
    for j in range(n + m):
        vp, vm = v0.copy(), v0.copy()
        vp[j] += h
        vm[j] -= h
        Fp = np.concatenate(O.kkt_residual(ocp, vp[None, :n], vp[None, n:]), axis=1)[0]
        Fm = np.concatenate(O.kkt_residual(ocp, vm[None, :n], vm[None, n:]), axis=1)[0]
        K[:, j] = (Fp - Fm) / (2 * h)
    sol = np.linalg.solve(K, np.concatenate([wz * z[0], np.zeros(m)]))
    grad = -dF_dtheta(ocp, z, lam, 0).T @ sol
    fd = np.zeros(ocp.p)
    for i in range(ocp.p):
        hh = 1e-6 * max(1.0, abs(ocp.theta[0, i]))
        vals = []
        for sgn in (1.0, -1.0):
            th = ocp.theta.copy()
            th[0, i] += sgn * hh
            pert = O.OCPBatch(ocp.model, ocp.T, ocp.x_s, th, ocp.x_ref)
            zz, _ = solve_to_convergence(pert, z, lam, tol=1e-14)
            vals.append(loss(zz[0]))
        fd[i] = (vals[0] - vals[1]) / (2 * hh)
    np.testing.assert_allclose(grad, fd, rtol=2e-5, atol=2e-6 * np.abs(fd).max())
