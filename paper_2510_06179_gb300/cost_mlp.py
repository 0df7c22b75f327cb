"""Learned cost weights for the vehicle OCPs: a 2-layer, 64-wide tanh MLP maps a 16-dim
feature per OCP to positive diagonal weights (Q over the 6 states, R over the 2 inputs), which
enter theta next to the tyre parameters (mu, C_alpha); the terminal weight is 10 Q.  Trained
end to end through the differentiable solve (torch autograd -> DiffMPCFunction -> Algorithm 3).
Outputs are softplus + 1e-3 (positive), scaled per component by a nominal tracking tune so that
steering (rad) and drive force (N) weights start at sensible magnitudes."""
import torch

NOMINAL_Q = (1.0, 1.0, 10.0, 1.0, 1.0, 1.0)
NOMINAL_R = (10.0, 1e-6)


class CostMLP(torch.nn.Module):
    def __init__(self, n_feat=16, width=64, nx=6, nu=2, nominal_q=NOMINAL_Q, nominal_r=NOMINAL_R):
        super().__init__()
        self.nx, self.nu = nx, nu
        self.net = torch.nn.Sequential(torch.nn.Linear(n_feat, width), torch.nn.Tanh(),
                                       torch.nn.Linear(width, width), torch.nn.Tanh(),
                                       torch.nn.Linear(width, nx + nu))
        self.register_buffer("scale", torch.tensor(tuple(nominal_q) + tuple(nominal_r)))

    def forward(self, feats):
        w = (torch.nn.functional.softplus(self.net(feats)) + 1e-3) * self.scale
        return w[:, :self.nx], w[:, self.nx:]


def vehicle_theta(shared, q, r, terminal=10.0):
    """theta of single-track OCPs, flat: per OCP [mu, C_alpha | diag Q | diag R | terminal * Q]."""
    return torch.cat([shared, q, r, terminal * q], dim=1).reshape(-1)
