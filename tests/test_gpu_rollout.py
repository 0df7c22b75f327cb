"""Closed-loop rollout (the RL benchmark shape): the episode reward's gradient with respect to
the MPC cost weights, back-propagated through H solves of ONE batch handle (each backward step
restores its solve's solution), against central finite differences of the same closed loop run
with the FP64 oracle's solves.  LQ dynamics make one SQP iteration exact, and the Gauss-Newton
KKT matrix is the exact one, so the IFT gradient and the differences agree to rounding."""
import numpy as np
import pytest

from paper_2510_06179_gb300 import workloads
from oracle.models import make_model
from oracle.ocp import OCPBatch as OracleBatch
from oracle.sqp import sqp as oracle_sqp
from tests.gpu_helpers import ensure_built

pytestmark = pytest.mark.gpu


def _oracle_reward(prob, q):
    """FP64 closed loop with the oracle's direct KKT solves; returns the per-OCP rewards."""
    nx, nu, T = prob.nx, prob.nu, prob.T
    knot = prob.knot_theta().astype(np.float64)
    theta = np.concatenate([knot, 2.0 * q, np.full((prob.B, nu), 2.0), 2.0 * q], axis=1)
    x = prob.x0.astype(np.float64)
    A, Bm, b = (a.astype(np.float64) for a in (prob.A, prob.Bm, prob.b))
    R = np.zeros(prob.B)
    model = make_model("lq", nx, nu)
    for _ in range(prob.H):
        ocp = OracleBatch(model, T, x, theta, np.zeros((prob.B, T + 1, nx)))
        z = oracle_sqp(ocp, 1, line_search_on=False)["z"]
        u = z[:, nx:nx + nu]
        R -= (x * x).sum(1) + (u * u).sum(1)
        x = np.einsum("bij,bj->bi", A, x) + np.einsum("bij,bj->bi", Bm, u) + b
    return R


@pytest.mark.parametrize("problem", [2, 5])
def test_rollout_gradient_matches_oracle_finite_differences(problem):
    """Problem 2 (nx 8, nu 4) and problem 5 (nx 16, nu 8) of the RL table, shortened."""
    import torch
    from paper_2510_06179_gb300.rollout import make_batch, closed_loop_reward
    ensure_built()
    prob = workloads.rl_lq_problem(problem, seed=3, B=3, H=4, T=12)
    prob.x0 = (prob.x0 / 5.0).astype(np.float32)     # keep the closed loop well scaled
    batch = make_batch(prob, "cuda:0")
    q = torch.from_numpy(prob.q0.copy()).to("cuda:0").requires_grad_(True)
    R = closed_loop_reward(batch, prob, q)
    R.backward()
    g_gpu = q.grad.cpu().numpy().astype(np.float64)
    q0 = prob.q0.astype(np.float64)
    g_fd = np.zeros_like(q0)
    for i in range(prob.nx):
        h = 1e-5 * np.maximum(1.0, np.abs(q0[:, i]))
        qp, qm = q0.copy(), q0.copy()
        qp[:, i] += h
        qm[:, i] -= h
        g_fd[:, i] = (_oracle_reward(prob, qp) - _oracle_reward(prob, qm)) / (2 * h)
    r_gpu = float(R.item())
    r_or = float(_oracle_reward(prob, q0).sum())
    err = np.linalg.norm(g_gpu - g_fd, axis=1) / np.linalg.norm(g_fd, axis=1)
    print(f"rollout: reward gpu {r_gpu:.6e} oracle {r_or:.6e}; grad rel err per OCP {err}")
    assert abs(r_gpu - r_or) <= 1e-4 * abs(r_or)
    assert err.max() <= 1e-3
    batch.close()


def test_one_handle_for_many_solves_equals_separate_handles():
    """Backward through two solves of one handle equals the same graph on two handles."""
    import torch
    from paper_2510_06179_gb300.rollout import make_batch, policy_theta, env_tensors
    from paper_2510_06179_gb300.solver import DiffMPCFunction
    ensure_built()
    prob = workloads.rl_lq_problem(2, seed=4, B=4, H=2, T=10)
    A, Bm, b, x0, knot = env_tensors(prob, "cuda:0")

    def two_steps(b1, b2, q):
        th = policy_theta(prob, knot, q)
        z1, _ = DiffMPCFunction.apply(x0.reshape(-1), th, b1, None, None)
        x1 = torch.einsum("bij,bj->bi", A, x0) + torch.einsum("bij,bj->bi", Bm, z1.view(prob.B, -1)[:, 8:12]) + b
        z2, _ = DiffMPCFunction.apply(x1.reshape(-1), th, b2, None, None)
        return (z1 ** 2).sum() + (z2 ** 3).sum()

    grads = []
    one = make_batch(prob, "cuda:0")
    two = (make_batch(prob, "cuda:0"), make_batch(prob, "cuda:0"))
    for b1, b2 in ((one, one), two):
        q = torch.from_numpy(prob.q0.copy()).to("cuda:0").requires_grad_(True)
        two_steps(b1, b2, q).backward()
        grads.append(q.grad.cpu().numpy())
    assert np.allclose(grads[0], grads[1], rtol=1e-5, atol=1e-6 * np.abs(grads[1]).max())
    for b in (one,) + two:
        b.close()


def test_graph_captured_rollout_matches_eager():
    import torch
    from paper_2510_06179_gb300.rollout import make_batch, closed_loop_reward, RolloutGraph, env_tensors
    ensure_built()
    prob = workloads.rl_lq_problem(2, seed=5, B=8, H=6, T=12)
    dev = "cuda:0"
    env = env_tensors(prob, dev)
    b1 = make_batch(prob, dev)
    q = torch.from_numpy(prob.q0.copy()).to(dev)
    with torch.no_grad():
        r_eager = float(closed_loop_reward(b1, prob, q, env).item())
    b2 = make_batch(prob, dev)
    g = RolloutGraph(b2, prob, q, env)
    q2 = q * 1.1
    with torch.no_grad():
        r_eager2 = float(closed_loop_reward(b1, prob, q2, env).item())
    r_graph2 = float(g.replay(q2).item())
    r_graph = float(g.replay(q).item())
    assert abs(r_graph - r_eager) <= 1e-5 * abs(r_eager)
    assert abs(r_graph2 - r_eager2) <= 1e-5 * abs(r_eager2)
    b1.close()
    b2.close()
