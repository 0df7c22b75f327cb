"""Forward pass of the FP64 oracle: SQP (Algorithm 2) with the line search of App. A.3
(Algorithm 5, merit Eq. 12-15), each QP solved DIRECTLY from its KKT system (Eq. 6).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Readings where the paper leaves a detail open:
  * penalty mu (App. A.3, Nocedal Eq. 18.33 with rho = 0.5): mu = max(num, 0) / (0.5 ||g||_1),
    num = sum_t grad c^T (z^+ - z); the point counts as feasible, mu = 0, when
    ||g||_1 <= FEAS_TOL (m + ||x||_1) (the formula divides by ||g||_1, which is 0, or
    rounding noise, once the constraints hold);
  * ||g||_1 includes the initial-state row x_0 - x_s;
  * the step is accepted when Delta phi_alpha < 0, scanning alpha in decreasing order;
    if none passes the smallest alpha is taken (Algorithm 5);
  * the multipliers take the same step: lambda <- lambda + alpha (lambda^+ - lambda).
"""
import numpy as np

from .ocp import (linearise, solve_qp, split_z, join_z, cost_value, cost_gradient,
                  constraint_residual, kkt_residual)

LS_ALPHAS = (1.0, 0.7, 0.3, 0.1, 0.01)
LS_ETA = 0.4
FEAS_TOL = 1e-5


def cold_start(ocp):
    """x_t = x_s for every knot, u_t = 0, lambda = 0."""
    x = np.repeat(ocp.x_s[:, None, :], ocp.K, axis=1)
    u = np.zeros((ocp.B, ocp.T, ocp.nu))
    return join_z(x, u), np.zeros((ocp.B, ocp.m))


def merit_parts(ocp, z):
    """(cost, ||g(z)||_1) per OCP."""
    return cost_value(ocp, z), np.abs(constraint_residual(ocp, z)).reshape(ocp.B, -1).sum(axis=1)


def line_search(ocp, z, z_plus, alphas=LS_ALPHAS, eta=LS_ETA):
    """Algorithm 5.  Returns (alpha (B,), diagnostics dict)."""
    dz = z_plus - z
    c0, g0 = merit_parts(ocp, z)
    num = np.einsum("bn,bn->b", cost_gradient(ocp, z), dz)
    x, _ = split_z(ocp, z)
    feasible = g0 <= FEAS_TOL * (ocp.m + np.abs(x).reshape(ocp.B, -1).sum(axis=1))
    mu = np.where(feasible, 0.0, np.maximum(num, 0.0) / np.where(feasible, 1.0, 0.5 * g0))
    D = num - mu * g0
    phi0 = c0 + mu * g0
    delta = np.empty((ocp.B, len(alphas)))
    for j, a in enumerate(alphas):
        ca, ga = merit_parts(ocp, z + a * dz)
        delta[:, j] = (ca + mu * ga) - phi0 - eta * a * D
    alpha = np.full(ocp.B, min(alphas))
    chosen = np.full(ocp.B, len(alphas) - 1 if min(alphas) == alphas[-1] else int(np.argmin(alphas)))
    for b in range(ocp.B):
        for j, a in enumerate(alphas):
            if delta[b, j] < 0.0:
                alpha[b] = a
                chosen[b] = j
                break
    return alpha, dict(delta=delta, phi0=phi0, mu=mu, D=D, chosen=chosen)


def sqp(ocp, iters, line_search_on=True, alphas=LS_ALPHAS, eta=LS_ETA, z0=None, lam0=None,
        dense=False, alpha_seq=None):
    """Algorithm 2 for a batch, a fixed number of iterations.

    Each iteration: linearise (Eq. 4), solve the QP exactly (Eq. 6), line search
    (Algorithm 5) or a full step, then z <- z + alpha (z^+ - z), lambda likewise.

    alpha_seq (B, iters), optional: take these step sizes instead of the line search's choice
    (a replay of another run's path); the line search's test values are still evaluated at
    every iterate and returned, with the oracle's own choice in "alpha_own"."""
    z, lam = cold_start(ocp)
    if z0 is not None:
        z = np.array(z0, dtype=np.float64)
    if lam0 is not None:
        lam = np.array(lam0, dtype=np.float64)
    hist_alpha = np.ones((ocp.B, iters))
    hist_own = np.ones((ocp.B, iters))
    hist_delta = np.zeros((ocp.B, iters, len(alphas)))
    hist_phi0 = np.zeros((ocp.B, iters))
    for k in range(iters):
        qp = linearise(ocp, z)
        zp = np.empty_like(z)
        lp = np.empty_like(lam)
        for b in range(ocp.B):
            zp[b], lp[b] = solve_qp(qp, b, dense=dense)
        if line_search_on:
            alpha, diag = line_search(ocp, z, zp, alphas, eta)
            hist_delta[:, k] = diag["delta"]
            hist_phi0[:, k] = diag["phi0"]
        else:
            alpha = np.ones(ocp.B)
        hist_own[:, k] = alpha
        if alpha_seq is not None:
            alpha = np.asarray(alpha_seq, dtype=np.float64)[:, k]
        z = z + alpha[:, None] * (zp - z)
        lam = lam + alpha[:, None] * (lp - lam)
        hist_alpha[:, k] = alpha
    return dict(z=z, lam=lam, alpha=hist_alpha, alpha_own=hist_own, delta=hist_delta, phi0=hist_phi0)


def solve_to_convergence(ocp, z0=None, lam0=None, tol=1e-13, max_iters=400, warm_iters=40):
    """Run SQP with the line search for `warm_iters` iterations, then full steps until
    max |z^+ - z| <= tol (used by the finite-difference checks)."""
    if z0 is None:
        out = sqp(ocp, warm_iters, line_search_on=True)
        z, lam = out["z"], out["lam"]
    else:
        z, lam = np.array(z0, dtype=np.float64), np.array(lam0, dtype=np.float64)
    for _ in range(max_iters):
        qp = linearise(ocp, z)
        zp = np.empty_like(z)
        lp = np.empty_like(lam)
        for b in range(ocp.B):
            zp[b], lp[b] = solve_qp(qp, b)
        step = np.abs(zp - z).max()
        z, lam = zp, lp
        if step <= tol:
            break
    return z, lam


def newton_kkt(ocp, z0, lam0, tol=1e-13, max_iters=50):
    """Newton's method on the KKT conditions F(z, lambda) = 0 of Eq. 1 (the textbook Newton-KKT
    iteration, Nocedal and Wright Alg. 18.1): K [dz; dlambda] = -F with K the KKT matrix of the
    EXACT Lagrangian Hessian (dynamics curvature included).  Converges quadratically from a point
    near a strict local minimum, where full-step Gauss-Newton SQP need not converge at all (its
    fixed-point map is not a contraction when the dynamics curvature weighted by the multipliers
    is large against the cost Hessian).  Used to re-solve perturbed OCPs for finite differences;
    not the paper's method.  Returns (z, lambda, final step, iterations)."""
    from .backward import exact_hessian_blocks
    z = np.array(z0, dtype=np.float64)
    lam = np.array(lam0, dtype=np.float64)
    step = np.inf
    for it in range(1, max_iters + 1):
        qp = linearise(ocp, z)
        Fz, Fl = kkt_residual(ocp, z, lam)
        dz = np.empty_like(z)
        dl = np.empty_like(lam)
        for b in range(ocp.B):
            G = exact_hessian_blocks(ocp, z, lam, b)
            dz[b], dl[b] = solve_qp(qp, b, rhs=-np.concatenate([Fz[b], Fl[b]]), G_blocks=G)
        z = z + dz
        lam = lam + dl
        step = np.abs(dz).max()
        if step <= tol:
            break
    return z, lam, step, it
