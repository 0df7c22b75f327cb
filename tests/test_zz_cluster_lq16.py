"""LQ with nx 16, nu 8 at a horizon longer than one CTA's share of the cluster's shared memory
holds at the ~40-knot rule: the automatic shape grows to the fewest CTAs whose share fits, and
the forward and adjoint solves on that cluster match the oracle's direct KKT solves.

Like the allocation-free tests this file is collected near the end, so that a run stopping at
its first failure has run the other parity files first."""
import numpy as np
import pytest

from paper_2510_06179_gb300 import workloads
from tests.gpu_helpers import gpu_solve, gpu_vjp
from tests.oracle_helpers import to_ocp, rel_err

pytestmark = pytest.mark.gpu

Z_GATE = 1e-4
G_GATE = 1e-3
BAD = 1 | 2 | 8 | 256   # PCG cap, non-finite, bad input, cluster wait timeout


def test_lq_nx16_t120_cluster_forward_and_adjoint_match_the_oracle():
    """T 120 (121 knots): one CTA holds at most 25 knots of a 16-state OCP, so the shape is 5 CTAs
    of 25 knots (the last owns 21), not the 4 of 31 the ~40-knot rule alone would give.  One SQP
    step solves the QP exactly (Eq. 8-11 with Algorithm 4), compared with the oracle's direct KKT
    solve; the backward's adjoint multipliers (Algorithm 3's linear solve with the same Schur
    complement) are compared with the oracle's direct solve of the KKT system with right-hand side
    (dl/dz, 0) at the GPU's solution, and dl/dx_s is their first knot."""
    from oracle.sqp import sqp as oracle_sqp
    from oracle.ocp import linearise, solve_qp
    w = workloads.lq_config(B=6, T=120, nx=16, nu=8, seed=4, c_var=0.01)
    b, g = gpu_solve(w, pcg_tol=1e-8)
    cl = b.get_cluster()
    assert (cl["ctas_per_cluster"], cl["knots_per_cta"]) == (5, 25), cl
    assert not (g["status"] & BAD & ~4).any(), g["status"]
    ocp = to_ocp(w)
    ref = oracle_sqp(ocp, 1, line_search_on=False)
    ez = rel_err(g["z"], ref["z"])
    dl = w.dl_dz(g["z"])
    gv = gpu_vjp(b, w, dl)
    assert not (gv["status"] & BAD).any(), gv["status"]
    qp = linearise(ocp, g["z"])
    lt = np.stack([solve_qp(qp, i, rhs=np.concatenate([dl[i], np.zeros(ocp.m)]))[1] for i in range(w.B)])
    el = rel_err(gv["lamt"], lt)
    ex = rel_err(gv["dxs"], lt[:, :w.nx])
    print(f"LQ nx 16 T 120 cluster {cl}: z err {ez.max():.2e}, adjoint err {el.max():.2e}, "
          f"dl/dx_s err {ex.max():.2e}")
    assert ez.max() <= Z_GATE
    assert el.max() <= G_GATE and ex.max() <= G_GATE
    b.close()
