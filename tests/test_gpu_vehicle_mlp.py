"""Vehicle OCPs with learned cost weights: features -> MLP -> theta -> GPU solve -> loss,
back-propagated through DiffMPCFunction into the MLP's parameters.  Checked against the chain
rule assembled independently: the oracle's FP64 Gauss-Newton VJP dl/dtheta at the GPU's
(z, lambda), pulled back through an FP64 CPU copy of the MLP by torch autograd."""
import numpy as np
import pytest

from paper_2510_06179_gb300 import workloads
from oracle.backward import vjp as oracle_vjp
from tests.gpu_helpers import ensure_built
from tests.oracle_helpers import to_ocp

pytestmark = pytest.mark.gpu


def test_mlp_cost_weights_gradient_through_the_solve():
    import copy
    import torch
    from paper_2510_06179_gb300.cost_mlp import CostMLP, vehicle_theta
    from paper_2510_06179_gb300.solver import OCPBatch, DiffMPCFunction
    ensure_built()
    torch.manual_seed(0)
    w = workloads.vehicle_config(B=8, T=30, seed=6, sqp_iters=6)
    dev = "cuda:0"
    mlp = CostMLP().to(dev)
    feats = torch.from_numpy(w.extra["features"]).to(dev)
    shared = torch.from_numpy(w.theta[:, :2].copy()).to(dev)
    b = OCPBatch(("single_track", 6, 2, w.T, w.dt), batch=w.B, device=dev, sqp_iters=w.sqp_iters,
                 line_search=1, pcg_tol=1e-9, warm_start=0)
    q, r = mlp(feats)
    theta = vehicle_theta(shared, q, r)
    x_s = torch.from_numpy(w.x_s.reshape(-1).copy()).to(dev)
    x_ref = torch.from_numpy(w.x_ref.reshape(-1).copy()).to(dev)
    z, lam = DiffMPCFunction.apply(x_s, theta, b, x_ref, None)
    u0 = z.view(w.B, -1)[:, 6:8]
    loss = (u0[:, 0] ** 2).sum() + 1e-6 * (u0[:, 1] ** 2).sum()
    loss.backward()
    g_gpu = {n: p.grad.detach().cpu().double().numpy() for n, p in mlp.named_parameters()}
    # independent chain: oracle dl/dtheta at the GPU's (z, lambda), pulled back through the MLP
    zz = z.detach().view(w.B, -1).cpu().numpy().astype(np.float64)
    ll = lam.detach().view(w.B, -1).cpu().numpy().astype(np.float64)
    dl = np.zeros_like(zz)
    dl[:, 6] = 2.0 * zz[:, 6]
    dl[:, 7] = 2e-6 * zz[:, 7]
    wt = copy.copy(w)
    wt.theta = theta.detach().view(w.B, -1).cpu().numpy()
    g_th = oracle_vjp(to_ocp(wt), zz, ll, dl)["dtheta"]
    mlp64 = copy.deepcopy(mlp).cpu().double()
    q64, r64 = mlp64(feats.cpu().double())
    th64 = vehicle_theta(shared.cpu().double(), q64, r64).view(w.B, -1)
    params = list(mlp64.parameters())
    ref = torch.autograd.grad((th64 * torch.from_numpy(g_th)).sum(), params)
    names = [n for n, _ in mlp64.named_parameters()]
    for n, gr in zip(names, ref):
        gr = gr.numpy()
        err = np.linalg.norm(g_gpu[n] - gr) / max(np.linalg.norm(gr), 1e-30)
        print(f"mlp grad {n}: rel err {err:.2e}")
        assert err <= 1e-3
    b.close()
