"""Closed-loop rollout of an MPC policy with gradients through every solve (the RL benchmark
shape of the paper's timing experiments): at each environment step h the batch of OCPs is
solved from the current state (one SQP iteration, full step: exact for LQ), the first control
is applied to the environment, and the episode reward is differentiated with respect to the
cost weights through the implicit-function gradient of every solve (Algorithm 3).

One OCPBatch serves all H solves: DiffMPCFunction restores each solve's solution before its
backward step (dmpc_set_solution), and the forward solves warm-start from the previous one."""
import torch

from .solver import DiffMPCFunction, OCPBatch


def make_batch(prob, device, pcg_tol=1e-9, **options):
    """OCPBatch for the MPC of an RLProblem: LQ OCPs (nx, nu, T), one SQP iteration, alpha = 1."""
    return OCPBatch(("lq", prob.nx, prob.nu, prob.T, 1.0), batch=prob.B, device=device, sqp_iters=1,
                    line_search=0, pcg_tol=pcg_tol, warm_start=1, **options)


def policy_theta(prob, knot, q):
    """theta of the LQ OCPs from the learnable diag(Q) (B, nx): the paper's costs x^T Q x and
    ||u||^2 in the library's 1/2-weighted form (Q -> 2Q, R = 2I, terminal 2Q)."""
    B = prob.B
    r = torch.full((B, prob.nu), 2.0, device=q.device)
    return torch.cat([knot, 2.0 * q, r, 2.0 * q], dim=1).reshape(-1)


def closed_loop_reward(batch, prob, q, env=None):
    """Episode reward R = -sum_{h<H} (||x_h||^2 + ||u_h||^2) summed over the batch, with
    x_{h+1} = A x_h + B u_h + b and u_h the first control of the MPC solve at x_h.
    q: (B, nx) cost weights (may require grad).  env: device tensors (A, Bm, b, x0, knot)."""
    dev = q.device
    if env is None:
        env = env_tensors(prob, dev)
    A, Bm, b, x, knot = env
    theta = policy_theta(prob, knot, q)
    nx, nu = prob.nx, prob.nu
    R = torch.zeros((), device=dev)
    for _ in range(prob.H):
        z, _ = DiffMPCFunction.apply(x.reshape(-1), theta, batch, None, None)
        u = z.view(prob.B, -1)[:, nx:nx + nu]
        R = R - (x * x).sum() - (u * u).sum()
        x = torch.einsum("bij,bj->bi", A, x) + torch.einsum("bij,bj->bi", Bm, u) + b
    return R


def env_tensors(prob, device):
    t = lambda a: torch.from_numpy(a).to(device)
    return t(prob.A), t(prob.Bm), t(prob.b), t(prob.x0), t(prob.knot_theta())


class RolloutGraph:
    """The forward closed-loop rollout (no gradients) captured once as a CUDA graph: the H solves
    and the environment steps between them replay with a single graph launch, removing the
    per-step host dispatch that bounds the eager rollout.  replay(q) copies new cost weights into
    the captured input and returns the reward tensor (valid after synchronisation)."""

    def __init__(self, batch, prob, q, env=None, warmup=2):
        self.batch, self.prob = batch, prob
        self.env = env if env is not None else env_tensors(prob, q.device)
        self.q = q.detach().clone()
        s = torch.cuda.Stream(q.device)
        s.wait_stream(torch.cuda.current_stream(q.device))
        with torch.cuda.stream(s), torch.no_grad():
            for _ in range(warmup):
                closed_loop_reward(batch, prob, self.q, self.env)
        torch.cuda.current_stream(q.device).wait_stream(s)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph), torch.no_grad():
            self.reward = closed_loop_reward(batch, prob, self.q, self.env)

    def replay(self, q=None):
        if q is not None:
            self.q.copy_(q)
        self.graph.replay()
        return self.reward
