"""Central finite differences of a loss of the OCP solution with respect to theta and x_s
(Eq. 3 checked numerically).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

For each coordinate i: (l(z*(theta + h e_i)) - l(z*(theta - h e_i))) / (2 h), the forward
re-solved to tight convergence each time (warm-started from the unperturbed solution).

step="max1": h = rel_step * max(1, |theta_i|); step="relative": h = rel_step * |theta_i| (for
parameters far below 1, such as a drive-force weight of 1e-6, where max(1, .) would change the
parameter by many times its own size).  solver="gn": full-step Gauss-Newton SQP (the method's
own QP); solver="newton": Newton's method on the KKT conditions with the exact Hessian, for
models where the Gauss-Newton fixed-point map does not contract at the solution."""
import numpy as np

from .ocp import OCPBatch
from .sqp import solve_to_convergence, newton_kkt


def fd_gradient(ocp, loss, z_star, lam_star, indices=None, rel_step=1e-6, wrt="theta",
                tol=1e-14, max_iters=400, step="max1", solver="gn"):
    """ocp: single-OCP batch.  loss: z (n,) -> float.  Returns gradient entries at `indices`."""
    base = ocp.theta[0] if wrt == "theta" else ocp.x_s[0]
    idx = range(base.size) if indices is None else indices
    out = []
    for i in idx:
        h = rel_step * (abs(base[i]) if step == "relative" and base[i] != 0 else max(1.0, abs(base[i])))
        vals = []
        for sgn in (1.0, -1.0):
            th = ocp.theta.copy()
            xs = ocp.x_s.copy()
            if wrt == "theta":
                th[0, i] += sgn * h
            else:
                xs[0, i] += sgn * h
            pert = OCPBatch(ocp.model, ocp.T, xs, th, ocp.x_ref)
            if solver == "newton":
                z, _, _, _ = newton_kkt(pert, z_star, lam_star, tol=tol, max_iters=min(max_iters, 50))
            else:
                z, _ = solve_to_convergence(pert, z_star, lam_star, tol=tol, max_iters=max_iters)
            vals.append(loss(z[0]))
        out.append((vals[0] - vals[1]) / (2.0 * h))
    return np.array(out)
