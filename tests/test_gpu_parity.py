"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle on the same seeded
float32 inputs.  Gates: solution ||z - z*|| / ||z*|| <= 1e-4 per OCP, gradient relative
error <= 1e-3 per OCP; QP building blocks (Eq. 4, 8-10) element by element within FP32
tolerances.  Runs with the line search follow the replay protocol (oracle/protocol.py): every
step size the GPU took must be one the oracle's own tests allow up to rounding, and every OCP's
solution is gated against the FP64 oracle replaying that step-size path."""
import numpy as np
import pytest

from paper_2510_06179_gb300 import workloads
from oracle import ocp as O
from oracle import schur as S
from oracle.backward import vjp as oracle_vjp
from oracle.sqp import sqp as oracle_sqp, cold_start
from tests.gpu_helpers import make_batch, gpu_solve, gpu_vjp, dev
from tests.oracle_helpers import to_ocp, rel_err, replay_check, assert_replay_parity

pytestmark = pytest.mark.gpu

Z_GATE = 1e-4
G_GATE = 1e-3


def _report(name, **kv):
    print(name, " ".join(f"{k}={v}" for k, v in kv.items()))


# ---------------------------------------------------------------------- building blocks
def _check_inspect(w, z, lam, tol_blocks):
    import torch
    b = make_batch(w)
    rec, off = b.inspect(dev(w.x_s), dev(w.theta), dev(z), x_ref=dev(w.x_ref), lam=dev(lam))
    torch.cuda.synchronize()
    ocp = to_ocp(w)
    qp = O.linearise(ocp, z.astype(np.float64))
    D, Off = S.schur_blocks(qp)
    Pd, Po = S.preconditioner_blocks(D, Off)
    gam = S.gamma_spd(qp)
    g = O.constraint_residual(ocp, z.astype(np.float64))
    worst = {}
    for bi in range(w.B):
        r = b.parse_inspect(rec, off, bi)
        zex, lex = O.solve_qp(qp, bi)
        pairs = {"A": (r["A"], qp.A[bi]), "B": (r["B"], qp.Bm[bi]), "C": (r["C"], qp.C[bi]),
                 "g": (r["g"], g[bi]), "D": (r["D"], D[bi]), "O": (r["O"][1:], Off[bi][1:]),
                 "Pd": (r["Pd"], Pd[bi]), "Po": (r["Po"][1:], Po[bi][1:]), "gamma": (r["gamma"], gam[bi])}
        for k, (a, e) in pairs.items():
            # relative to the block's magnitude; quantities that are exactly zero in the
            # oracle (C_t of LQ without offsets) are compared on the scale of 1
            scale = max(np.abs(e).max(), 1.0 if k in ("C", "g") else 1e-30)
            err = np.abs(a - e).max() / scale
            worst[k] = max(worst.get(k, 0.0), err)
        worst["z+"] = max(worst.get("z+", 0.0), rel_err(r["z"], zex))
        worst["lam+"] = max(worst.get("lam+", 0.0), rel_err(r["lam"].reshape(-1), lex))
    _report(f"inspect[{w.name}]", **{k: f"{v:.2e}" for k, v in worst.items()})
    for k in ("A", "B", "C", "D", "O", "Pd", "Po", "gamma", "g"):
        assert worst[k] <= tol_blocks, (k, worst[k])
    assert worst["z+"] <= Z_GATE
    b.close()
    return worst


def test_inspect_lq_blocks_and_qp_solution():
    w = workloads.lq_config()
    ocp = to_ocp(w)
    z0, lam0 = cold_start(ocp)
    _check_inspect(w, z0.astype(np.float32), lam0.astype(np.float32), 1e-5)


def test_inspect_cartpole_blocks_random_point():
    w = workloads.cartpole_config(B=16, T=50, seed=3)
    rng = np.random.default_rng(0)
    z = (0.3 * rng.standard_normal((w.B, w.n))).astype(np.float32)
    lam = (0.1 * rng.standard_normal((w.B, w.m))).astype(np.float32)
    _check_inspect(w, z, lam, 2e-5)


# ---------------------------------------------------------------------- forward parity
def test_lq_config_forward_parity():
    """LQ, nx 4, nu 1, T 20, batch 16, seed 0, one SQP step, PCG tol 1e-8 (relative residual)."""
    w = workloads.lq_config()
    b, g = gpu_solve(w, pcg_tol=1e-8)
    ref = oracle_sqp(to_ocp(w), 1, line_search_on=False)
    e = rel_err(g["z"], ref["z"])
    el = rel_err(g["lam"], ref["lam"])
    _report("lq", zerr_max=f"{e.max():.2e}", lamerr_max=f"{el.max():.2e}", pcg_iters=g["iters"].ravel().tolist())
    assert (g["status"] & ~4 == 0).all(), g["status"]
    assert e.max() <= Z_GATE
    b.close()


def _nonlinear_forward(w, **opt):
    b, g = gpu_solve(w, **opt)
    res = replay_check(w, g["z"], g["alpha"])
    _report(f"forward[{w.name}]", B=w.B, own_path=f"{res['agree'].sum()}/{w.B}",
            zerr_median=f"{np.median(res['ez']):.2e}", pcg_mean=f"{g['iters'].mean():.1f}",
            pcg_max=int(g["iters"].max()), status=np.unique(g["status"]).tolist())
    assert_replay_parity(w.name, res, Z_GATE)
    assert not (g["status"] & (1 | 2 | 8)).any()
    return b, g, res["rep"]


def test_cartpole_forward_parity():
    """Cart-pole, nx 4, nu 1, T 50, dt 0.05, RK4, 10 SQP iterations with line search."""
    w = workloads.cartpole_config(B=64, T=50, seed=0)
    b, g, ref = _nonlinear_forward(w)
    b.close()


def test_cartpole_one_reduction_pcg_parity():
    """pcg_variant = 1 (Algorithm 4 reorganised with one fused reduction per iteration) meets the
    same solution and gradient gates under the replay protocol."""
    w = workloads.cartpole_config(B=64, T=50, seed=0)
    b, g, ref = _nonlinear_forward(w, pcg_variant=1, pcg_tol=5e-8)
    _grad_check(w, b, g)
    b.close()


def test_cartpole_double_float_pcg_parity():
    """pcg_precision = 1: the whole PCG solve in double-float arithmetic (single-warp teams)
    meets the same solution and gradient gates, and no OCP needs the rescue."""
    w = workloads.cartpole_config(B=32, T=50, seed=3)
    b, g, ref = _nonlinear_forward(w, pcg_precision=1, team_threads=32)
    assert not (g["status"] & 64).any()
    _grad_check(w, b, g)
    b.close()


@pytest.mark.parametrize("maker", [workloads.pendulum_config, workloads.bicycle_config])
def test_other_small_models_forward_parity(maker):
    w = maker(B=32, T=40, seed=1, sqp_iters=6)
    b, g, ref = _nonlinear_forward(w)
    b.close()


def test_attitude_forward_parity():
    """Attitude stabilisation (App. B.1): nx = nu = 3, Euler dt 0.1, T 25, batch 16."""
    w = workloads.attitude_config()
    b, g, ref = _nonlinear_forward(w)
    b.close()


def test_vehicle_forward_parity_small():
    w = workloads.vehicle_config(B=16, T=40, seed=2, sqp_iters=4)
    b, g, ref = _nonlinear_forward(w)
    b.close()


def test_vehicle_control_rate_forward_and_gradient_parity():
    """The vehicle with control-rate augmentation (App. B.3): state (x, delta, F_x), input their
    rates; nx 8 runs the shared-memory PCG."""
    w = workloads.vehicle_rate_config(B=16, T=40, seed=3, sqp_iters=4)
    b, g, ref = _nonlinear_forward(w)
    _grad_check(w, b, g)
    b.close()


def test_rigid_body_forward_parity_small():
    w = workloads.rigid_body_config(B=8, T=24, seed=2, sqp_iters=3)
    b, g, ref = _nonlinear_forward(w)
    b.close()


# ---------------------------------------------------------------------- gradients
def _grad_check(w, b, g):
    """GPU vjp vs the oracle's Gauss-Newton VJP linearised at the GPU's own (z, lambda)."""
    dl = w.dl_dz(g["z"])
    gv = gpu_vjp(b, w, dl)
    ref = oracle_vjp(to_ocp(w), g["z"], g["lam"], dl)
    e = rel_err(gv["dtheta"], ref["dtheta"])
    ex = rel_err(gv["dxs"], ref["dxs"])
    _report(f"grad[{w.name}]", dtheta_err_max=f"{e.max():.2e}", dxs_err_max=f"{ex.max():.2e}",
            pcg_mean=f"{gv['iters'].mean():.1f}", status=np.unique(gv["status"]).tolist())
    assert e.max() <= G_GATE and ex.max() <= G_GATE
    return gv


def test_lq_gradient_parity():
    w = workloads.lq_config(c_var=0.01)
    b, g = gpu_solve(w, pcg_tol=1e-8)
    _grad_check(w, b, g)
    b.close()


def test_cartpole_gradient_parity():
    w = workloads.cartpole_config(B=64, T=50, seed=0)
    b, g = gpu_solve(w)
    _grad_check(w, b, g)
    b.close()


@pytest.mark.parametrize("maker", [workloads.pendulum_config, workloads.bicycle_config,
                                   workloads.attitude_config])
def test_other_models_gradient_parity(maker):
    w = maker(B=16, seed=4)
    b, g = gpu_solve(w)
    _grad_check(w, b, g)
    b.close()


def test_vehicle_and_rigid_body_gradient_parity():
    for w in (workloads.vehicle_config(B=8, T=40, seed=5, sqp_iters=3),
              workloads.rigid_body_config(B=4, T=24, seed=5, sqp_iters=2)):
        b, g = gpu_solve(w)
        _grad_check(w, b, g)
        b.close()


def test_store_mode_matches_recompute():
    w = workloads.cartpole_config(B=16, T=30, seed=7, sqp_iters=4)
    b1, g1 = gpu_solve(w, store_schur=0)
    b2, g2 = gpu_solve(w, store_schur=1)
    dl = w.dl_dz(g1["z"])
    v1, v2 = gpu_vjp(b1, w, dl), gpu_vjp(b2, w, dl)
    assert np.array_equal(g1["z"], g2["z"])
    assert rel_err(v1["dtheta"], v2["dtheta"]).max() <= 1e-5
    b1.close(); b2.close()


# ---------------------------------------------------------------------- structure / edges
@pytest.mark.parametrize("team,tpb", [(32, 1), (32, 3), (64, 2), (128, 1), (256, 1)])
def test_tiling_variants_agree(team, tpb):
    """Several knots per thread (K > team), several OCPs per block, a ragged last block."""
    w = workloads.cartpole_config(B=7, T=90, seed=11, sqp_iters=3)
    base_b, base = gpu_solve(w, team_threads=32, teams_per_block=1)
    b, g = gpu_solve(w, team_threads=team, teams_per_block=tpb)
    assert_replay_parity(f"tiling {team}x{tpb}", replay_check(w, g["z"], g["alpha"]), Z_GATE)
    same = np.array_equal(g["alpha"], base["alpha"])
    if same:
        assert rel_err(g["z"], base["z"]).max() <= 1e-4
    base_b.close(); b.close()


def test_horizon_one_and_two():
    for T in (1, 2):
        w = workloads.cartpole_config(B=3, T=T, seed=2, sqp_iters=2)
        b, g = gpu_solve(w)
        assert_replay_parity(f"T={T}", replay_check(w, g["z"], g["alpha"]), Z_GATE)
        b.close()


def test_mixed_batch_one_launch_matches_oracle():
    """Uneven batch (pendulum / cart-pole / bicycle, T ~ U{16..128}) in one launch."""
    import torch
    from paper_2510_06179_gb300.solver import OCPBatch
    from tests.gpu_helpers import ensure_built
    ensure_built()
    items = workloads.uneven_mix(n_ocps=18, T_lo=16, T_hi=128, seed=3, sqp_iters=4)
    descs = [(w.model, w.nx, w.nu, w.T, w.dt) for w in items]
    b = OCPBatch(descs, device="cuda:0", sqp_iters=4, line_search=1, pcg_tol=1e-9)
    x_s = np.concatenate([w.x_s.ravel() for w in items])
    th = np.concatenate([w.theta.ravel() for w in items])
    xr = np.concatenate([w.x_ref.ravel() for w in items])
    out = b.solve(dev(x_s), dev(th), dev(xr))
    torch.cuda.synchronize()
    z = out["z"].cpu().numpy().astype(np.float64)
    al = out["alpha"].view(len(items), -1).cpu().numpy()
    own = 0
    for i, w in enumerate(items):
        zi = z[b.z_off[i]:b.z_off[i + 1]][None]
        res = replay_check(w, zi, al[i][None])
        own += int(res["agree"][0])
        assert res["consistent"][0], (i, w.model, w.T, res["first_bad"][0])
        assert res["ez"][0] <= Z_GATE, (i, w.model, w.T, res["ez"][0])
    print(f"uneven: {len(items)} OCPs, {own} on the oracle's own path, all consistent and within the gate")
    b.close()


def test_nonfinite_input_is_flagged_not_fatal():
    w = workloads.cartpole_config(B=4, T=20, seed=1, sqp_iters=2)
    w.theta[2, 0] = np.nan
    b, g = gpu_solve(w)
    assert g["status"][2] & (8 | 2)
    assert np.isfinite(g["z"][[0, 1, 3]]).all()
    b.close()


def test_vjp_before_solve_is_state_error():
    from paper_2510_06179_gb300._lib import DMPCError
    w = workloads.cartpole_config(B=2, T=10)
    b = make_batch(w)
    with pytest.raises(DMPCError) as ei:
        b.vjp(dev(np.zeros((w.B, w.n))))
    assert ei.value.code == 5
    b.close()


def test_warm_start_reduces_pcg_iterations():
    w = workloads.lq_config(B=16, T=20, seed=5)
    b, g1 = gpu_solve(w, pcg_tol=1e-8)
    b2, g2 = gpu_solve(w, batch=b)          # warm start from the resident solution
    assert g2["iters"].sum() < g1["iters"].sum()
    assert rel_err(g2["z"], g1["z"]).max() <= 1e-5
    b.close()


def test_autograd_function_matches_vjp():
    import torch
    from paper_2510_06179_gb300.solver import diffmpc
    w = workloads.cartpole_config(B=8, T=30, seed=9, sqp_iters=3)
    b = make_batch(w)
    x_s = dev(w.x_s).requires_grad_(True)
    th = dev(w.theta).requires_grad_(True)
    z = diffmpc(x_s, th, b, x_ref=dev(w.x_ref)).view(w.B, -1)
    ut = dev(w.u_target).view(w.B, -1)
    loss = ((z[:, w.nx:w.nx + w.nu] - ut) ** 2).sum()
    loss.backward()
    zn = z.detach().cpu().numpy().astype(np.float64)
    g2 = gpu_vjp(b, w, w.dl_dz(zn))
    np.testing.assert_allclose(th.grad.view(w.B, -1).cpu().numpy(), g2["dtheta"], rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(x_s.grad.view(w.B, -1).cpu().numpy(), g2["dxs"], rtol=1e-5, atol=1e-6)
    b.close()
