"""Re-check of the OCPs whose step-size path branched from the oracle's.  Swing-up OCPs are
nonconvex and the line search's tests can sit within rounding of zero, so FP32 and FP64 runs may
take different step sizes and reach different local minima, all of them correct results.  For
every branched OCP both sides run on to convergence from their own iterates (full SQP steps);
the GPU's converged point must then be a KKT point of the OCP (Eq. 1): the FP64 oracle's
full-step SQP, started there, stays within the solution gate of it.  Where both sides end at
the same minimum the gate applies directly; the counts of same and other minima, and the costs,
are printed."""
import numpy as np
import pytest

from paper_2510_06179_gb300 import workloads
from oracle.ocp import cost_value, kkt_residual
from oracle.sqp import sqp as oracle_sqp, solve_to_convergence
from tests.gpu_helpers import gpu_solve, make_batch, dev, alpha_paths_agree
from tests.oracle_helpers import to_ocp, rel_err

pytestmark = pytest.mark.gpu

CASES = {
    "cartpole": lambda: workloads.cartpole_config(B=64, T=50, seed=1000, sqp_iters=10),
    "pendulum": lambda: workloads.pendulum_config(B=64, T=40, seed=7, sqp_iters=10),
    "kin_bicycle": lambda: workloads.bicycle_config(B=64, T=40, seed=7, sqp_iters=10),
    "attitude": lambda: workloads.attitude_config(B=64, seed=7, sqp_iters=10),
}


@pytest.mark.parametrize("name", list(CASES))
def test_branched_ocps_end_at_kkt_points(name):
    w = CASES[name]()
    B = w.B
    b10, g10 = gpu_solve(w, pcg_tol=5e-8, warm_start=0)
    b10.close()
    ocp_all = to_ocp(w)
    ref10 = oracle_sqp(ocp_all, w.sqp_iters, line_search_on=True)
    br = np.where(~alpha_paths_agree(g10["alpha"], ref10["alpha"]))[0]
    print(f"{name} {B}: {len(br)} OCPs branched after {w.sqp_iters} SQP iterations")
    if len(br) == 0:
        return
    # the GPU on from its own iterate: 100 full SQP steps (Gauss-Newton converges linearly)
    bc = make_batch(w, sqp_iters=100, line_search=0, pcg_tol=5e-8, warm_start=0)
    out = bc.solve(dev(w.x_s), dev(w.theta), dev(w.x_ref), z_init=dev(g10["z"]), lam_init=dev(g10["lam"]))
    z_g = out["z"].view(B, -1).cpu().numpy().astype(np.float64)[br]
    lam_g = out["lam"].view(B, -1).cpu().numpy().astype(np.float64)[br]
    st = out["status"].cpu().numpy()[br]
    bc.close()
    assert not (st & (2 | 8)).any()
    # the oracle on from its own iterate, and from the GPU's converged point
    ocp = to_ocp(w, br)
    z_or, _ = solve_to_convergence(ocp, ref10["z"][br], ref10["lam"][br], tol=1e-12)
    z_pol, lam_pol = solve_to_convergence(ocp, z_g, lam_g, tol=1e-12)
    Fz, Fl = kkt_residual(ocp, z_pol, lam_pol)
    polished_res = np.maximum(np.abs(Fz).max(1), np.abs(Fl).max(1))
    e_pol = rel_err(z_g, z_pol)
    same = rel_err(z_g, z_or) <= 1e-4
    c_g, c_or = cost_value(ocp, z_g), cost_value(ocp, z_or)
    for i, b in enumerate(br):
        print(f"  OCP {b}: {'same minimum' if same[i] else 'other minimum'}; GPU point to its FP64 KKT "
              f"point {e_pol[i]:.1e} (residual there {polished_res[i]:.1e}); cost GPU {c_g[i]:.6g} "
              f"oracle {c_or[i]:.6g}")
    print(f"branched: {same.sum()} same minimum, {(~same).sum()} other minimum")
    assert polished_res.max() <= 1e-8
    assert e_pol.max() <= 1e-4
