"""Algorithm 4 distributed over a thread-block cluster (12-state rigid body with horizons whose
workspace does not fit in one CTA's shared memory: each OCP runs on a cluster of CTAs holding its
S and Phi^-1 blocks in their shared memory during the PCG solves).  Checked against the FP64
oracle: the QP solution of one SQP iteration against the oracle's direct KKT solve, multi-iteration
runs under the replay protocol, gradients against the oracle's VJP at the GPU's own (z, lambda),
ragged knot partitions (including CTAs that own no knot), every cluster size, and the handle's
choice of the cluster form."""
import numpy as np
import pytest

from paper_2510_06179_gb300 import workloads
from oracle import ocp as O
from oracle.backward import vjp as oracle_vjp
from oracle.sqp import cold_start
from tests.gpu_helpers import make_batch, gpu_solve, gpu_vjp, dev, ensure_built
from tests.oracle_helpers import to_ocp, rel_err, replay_check, assert_replay_parity

pytestmark = pytest.mark.gpu

Z_GATE = 1e-4
G_GATE = 1e-3
BAD = 1 | 2 | 8 | 256   # PCG cap, non-finite, bad input, cluster wait timeout


def test_cluster_form_is_chosen_when_the_workspace_exceeds_shared_memory():
    w = workloads.rigid_body_config(B=3, T=200, seed=21, sqp_iters=1)
    b = make_batch(w)
    # about 40 knots per CTA: 201 knots on 6 CTAs of 34
    assert b.get_cluster() == dict(ctas_per_cluster=6, knots_per_cta=34, clusters=3)
    assert b.get_tiling()["team_threads"] == 256
    b.close()
    b = make_batch(w, cluster_ctas=1)          # opt-out: one team per OCP from global memory
    assert b.get_cluster()["ctas_per_cluster"] == 0
    assert b.get_tiling()["smem_bytes"] == 0
    b.close()
    b = make_batch(w, cluster_ctas=8)
    assert b.get_cluster()["ctas_per_cluster"] == 8 and b.get_cluster()["knots_per_cta"] == 26
    b.close()
    b = make_batch(w, cluster_ctas=4)          # 51 knots per CTA: more than a CTA holds
    assert b.get_cluster()["ctas_per_cluster"] == 0
    b.close()
    short = workloads.rigid_body_config(B=2, T=24, seed=2, sqp_iters=1)
    b = make_batch(short)                      # fits in one CTA's shared memory
    assert b.get_cluster()["ctas_per_cluster"] == 0 and b.get_tiling()["smem_bytes"] > 0
    b.close()


@pytest.mark.parametrize("T,seed", [(255, 7), (100, 3)])
def test_cluster_qp_solution_matches_direct_kkt(T, seed):
    """One QP per OCP at the cold start (dmpc_qp_inspect): the distributed PCG's solution and
    multipliers against the oracle's banded direct KKT solve."""
    import torch
    w = workloads.rigid_body_config(B=4, T=T, seed=seed, sqp_iters=1)
    b = make_batch(w)
    assert b.get_cluster()["ctas_per_cluster"] > 0
    ocp = to_ocp(w)
    z0, lam0 = cold_start(ocp)
    rec, off = b.inspect(dev(w.x_s), dev(w.theta), dev(z0), x_ref=dev(w.x_ref), lam=dev(lam0))
    torch.cuda.synchronize()
    qp = O.linearise(ocp, z0.astype(np.float32).astype(np.float64))
    ez, el = [], []
    for bi in range(w.B):
        r = b.parse_inspect(rec, off, bi)
        zex, lex = O.solve_qp(qp, bi)
        ez.append(rel_err(r["z"], zex))
        el.append(rel_err(r["lam"].reshape(-1), lex))
    print(f"cluster inspect T={T}: z+ err {max(ez):.2e}, lambda+ err {max(el):.2e}")
    assert max(ez) <= Z_GATE and max(el) <= 1e-3
    b.close()


def test_cluster_forward_replay_parity():
    w = workloads.rigid_body_config(B=6, T=200, seed=21, sqp_iters=3)
    b, g = gpu_solve(w)
    assert b.get_cluster()["ctas_per_cluster"] == 6
    assert not (g["status"] & BAD).any(), g["status"]
    res = replay_check(w, g["z"], g["alpha"])
    assert_replay_parity("cluster rigid body T=200", res, Z_GATE)
    b.close()


@pytest.mark.parametrize("ctas", [2, 3, 5, 8])
def test_every_cluster_size_matches_the_oracle(ctas):
    """The knot partition changes with the cluster size (T = 80: 81 knots over 2..8 CTAs,
    ragged last CTA); every size solves to the oracle's replay."""
    w = workloads.rigid_body_config(B=3, T=80, seed=11, sqp_iters=2)
    b, g = gpu_solve(w, cluster_ctas=ctas)
    assert b.get_cluster()["ctas_per_cluster"] == ctas
    assert not (g["status"] & BAD).any(), g["status"]
    assert_replay_parity(f"cluster of {ctas} CTAs", replay_check(w, g["z"], g["alpha"]), Z_GATE)
    b.close()


def test_ragged_horizons_in_one_handle_with_empty_ctas():
    """One handle, horizons 200, 97, 40 and 6 on clusters of 8 CTAs (the count follows the longest
    horizon), so the short OCPs leave trailing CTAs with no knot (T = 40: 41 knots as 6 per CTA,
    CTA 7 empty; T = 6: one knot per CTA)."""
    import torch
    from paper_2510_06179_gb300.solver import OCPBatch
    ensure_built()
    items = [workloads.rigid_body_config(B=1, T=T, seed=30 + T, sqp_iters=2) for T in (200, 97, 40, 6)]
    descs = [(w.model, w.nx, w.nu, w.T, w.dt) for w in items]
    b = OCPBatch(descs, device="cuda:0", sqp_iters=2, line_search=1, pcg_tol=1e-9, cluster_ctas=8)
    assert b.get_cluster()["ctas_per_cluster"] == 8
    cat = lambda f: np.concatenate([getattr(w, f).ravel() for w in items])
    out = b.solve(dev(cat("x_s")), dev(cat("theta")), dev(cat("x_ref")))
    torch.cuda.synchronize()
    z = out["z"].cpu().numpy().astype(np.float64)
    al = out["alpha"].view(len(items), -1).cpu().numpy()
    st = out["status"].cpu().numpy()
    assert not (st & BAD).any(), st
    for i, w in enumerate(items):
        res = replay_check(w, z[b.z_off[i]:b.z_off[i + 1]][None], al[i][None])
        assert_replay_parity(f"ragged T={w.T}", res, Z_GATE)
    b.close()


def test_cluster_gradient_parity():
    """Backward (Algorithm 3): the adjoint PCG on the cluster; dl/dtheta and dl/dx_s against the
    oracle's Gauss-Newton VJP linearised at the GPU's own (z, lambda)."""
    w = workloads.rigid_body_config(B=4, T=150, seed=5, sqp_iters=2)
    b, g = gpu_solve(w)
    assert b.get_cluster()["ctas_per_cluster"] > 0
    dl = w.dl_dz(g["z"])
    gv = gpu_vjp(b, w, dl)
    ref = oracle_vjp(to_ocp(w), g["z"], g["lam"], dl)
    e = rel_err(gv["dtheta"], ref["dtheta"])
    ex = rel_err(gv["dxs"], ref["dxs"])
    print(f"cluster grad: dtheta {e.max():.2e}, dxs {ex.max():.2e}, adjoint PCG {gv['iters'].tolist()}")
    assert not (gv["status"] & BAD).any()
    assert e.max() <= G_GATE and ex.max() <= G_GATE
    b.close()


def test_cluster_and_single_team_forms_agree():
    """Same inputs through the cluster form and the one-team global-memory form: both within the
    gate of the oracle's replay of their own step sizes; where the step sizes agree, the two
    solutions agree to the gate."""
    w = workloads.rigid_body_config(B=4, T=128, seed=13, sqp_iters=2)
    b1, g1 = gpu_solve(w)
    b2, g2 = gpu_solve(w, cluster_ctas=1)
    assert b1.get_cluster()["ctas_per_cluster"] > 0 and b2.get_cluster()["ctas_per_cluster"] == 0
    for name, g in (("cluster", g1), ("one team", g2)):
        assert_replay_parity(name, replay_check(w, g["z"], g["alpha"]), Z_GATE)
    same = np.all(g1["alpha"] == g2["alpha"], axis=1)
    if same.any():
        assert rel_err(g1["z"][same], g2["z"][same]).max() <= Z_GATE
    b1.close(); b2.close()


def test_double_float_rescue_on_the_cluster():
    """OCPs whose FP32 iteration stagnates are finished by the double-float PCG on the cluster
    (status bit 64); those solutions match the FP64 oracle's replay like the others."""
    w = workloads.rigid_body_config(B=64, T=128, seed=3, sqp_iters=5)
    b, g = gpu_solve(w, pcg_tol=1e-7)
    assert b.get_cluster()["ctas_per_cluster"] > 0
    assert not (g["status"] & BAD).any(), g["status"]
    rescued = np.where(g["status"] & 64)[0]
    assert rescued.size > 0, "no OCP of this batch needed the rescue"
    pick = np.concatenate([rescued[:4], np.setdiff1d(np.arange(w.B), rescued)[:2]])
    sub = w.subset(pick)
    res = replay_check(sub, g["z"][pick], g["alpha"][pick])
    assert_replay_parity(f"cluster rescue ({rescued.size} rescued)", res, Z_GATE)
    b.close()


def test_cluster_stored_blocks_backward_matches_recompute():
    """Stored-Schur mode on a cluster handle: the forward keeps the blocks at the returned z and
    the vjp's cluster PCG reads them instead of forming them; the gradient equals the recompute
    mode's."""
    w = workloads.rigid_body_config(B=3, T=90, seed=17, sqp_iters=2)
    b1, g1 = gpu_solve(w, store_schur=0)
    b2, g2 = gpu_solve(w, store_schur=1)
    assert b2.get_cluster()["ctas_per_cluster"] > 0
    assert np.array_equal(g1["z"], g2["z"])
    dl = w.dl_dz(g1["z"])
    v1, v2 = gpu_vjp(b1, w, dl), gpu_vjp(b2, w, dl)
    assert not ((v1["status"] | v2["status"]) & BAD).any()
    assert rel_err(v2["dtheta"], v1["dtheta"]).max() <= 1e-5
    ref = oracle_vjp(to_ocp(w), g2["z"], g2["lam"], dl)
    assert rel_err(v2["dtheta"], ref["dtheta"]).max() <= G_GATE
    b1.close(); b2.close()


def test_cluster_exact_hessian_backward():
    """Exact-Hessian backward (Riccati on CTA 0; OCPs whose reduced Hessian is not positive
    definite take the Gauss-Newton path, whose PCG runs on the cluster) after a cluster forward."""
    w = workloads.rigid_body_config(B=3, T=70, seed=19, sqp_iters=3)
    b, g = gpu_solve(w, exact_hessian=1)
    assert b.get_cluster()["ctas_per_cluster"] > 0
    dl = w.dl_dz(g["z"])
    gv = gpu_vjp(b, w, dl)
    ocp = to_ocp(w)
    exact = oracle_vjp(ocp, g["z"], g["lam"], dl, hessian="exact")
    gn = oracle_vjp(ocp, g["z"], g["lam"], dl, hessian="gn")
    flagged = (gv["status"] & 128) != 0
    ref = np.where(flagged[:, None], gn["dtheta"], exact["dtheta"])
    assert not (gv["status"] & BAD).any()
    assert rel_err(gv["dtheta"], ref).max() <= G_GATE
    b.close()


def test_lq_nx16_cluster_matches_the_oracle():
    """LQ with nx 16, nu 8, T 30 (the RL table's problems 5 and 6) runs on a cluster (a one-warp team
    would carry four 16 x 16 blocks per lane); one SQP step solves the QP exactly, compared with the
    oracle's direct KKT solve, and the gradient with the oracle's VJP."""
    from oracle.sqp import sqp as oracle_sqp
    w = workloads.lq_config(B=6, T=30, nx=16, nu=8, seed=4, c_var=0.01)
    b, g = gpu_solve(w, pcg_tol=1e-8)
    assert b.get_cluster()["ctas_per_cluster"] == 2
    assert not (g["status"] & BAD & ~4).any(), g["status"]
    ref = oracle_sqp(to_ocp(w), 1, line_search_on=False)
    ez = rel_err(g["z"], ref["z"])
    dl = w.dl_dz(g["z"])
    gv = gpu_vjp(b, w, dl)
    gr = oracle_vjp(to_ocp(w), g["z"], g["lam"], dl)
    eg = rel_err(gv["dtheta"], gr["dtheta"])
    print(f"LQ nx 16 cluster: z err {ez.max():.2e}, dtheta err {eg.max():.2e}, {b.get_cluster()}")
    assert ez.max() <= Z_GATE and eg.max() <= G_GATE
    b.close()


def test_autotuner_keeps_the_cluster_form():
    """The automatic tiling is the autotuner's first candidate, so a rigid-body batch with a long
    horizon keeps the cluster form (every explicit tiling runs one team from global memory); an
    explicit tiling and then (0, 0) restore the automatic choice."""
    import torch
    from paper_2510_06179_gb300 import autotune
    w = workloads.rigid_body_config(B=4, T=100, seed=23, sqp_iters=1)
    b = make_batch(w, pcg_tol=1e-7)
    auto = b.get_cluster()
    assert auto["ctas_per_cluster"] > 0
    b.set_tiling(256, 1)
    assert b.get_cluster()["ctas_per_cluster"] == 0
    b.set_tiling(0, 0)
    assert b.get_cluster() == auto
    inp = (dev(w.x_s), dev(w.theta), dev(w.x_ref))
    res = autotune.tune(b, inp, reps=1, use_cache=False, teams=(128, 256), tpbs=(1,))
    assert res["table"][0]["team_threads"] == 0
    print("autotune table (ms):", [(r["team_threads"], r["teams_per_block"], round(r["ms"], 2)) for r in res["table"]])
    assert (res["team_threads"], res["teams_per_block"]) == (0, 0)
    assert b.get_cluster() == auto
    b.close()
