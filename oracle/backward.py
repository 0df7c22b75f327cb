"""Backward pass of the FP64 oracle: the VJP of Eq. 3 through the KKT system of Eq. 7
(Algorithm 3), solved DIRECTLY, with dF/dtheta assembled explicitly from Eq. 1.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

  [z~; lambda~] = K^-1 [dl/dz; 0],   dl/dtheta = -(dF/dtheta)^T [z~; lambda~],
  F(z, lambda, theta) = [grad_z c + (dg/dz)^T lambda ; g],  g = (x_0 - x_s, f_0, ..., f_{T-1}).

K is the Gauss-Newton KKT matrix of the forward QP (Sec. 3.4: the dynamics curvature is
left out of G), linearised at the returned z.  hessian="exact" instead uses
G = grad^2_zz L including sum_t lambda_{t+1}^T grad^2 f_t; it is used only to validate the
dF/dtheta machinery against finite differences on nonlinear dynamics.
dl/dx_s = lambda~_0, because dg_0/dx_s = -I.
"""
import numpy as np

from .ocp import (linearise, solve_qp, split_z, split_theta, theta_offsets,
                  dynamics_jet, constraint_jet, x_index, u_index)


def _phi_jets(ocp, z):
    """Explicit integrators: Phi_t as Jets over (x_t, u_t, theta); implicit ones: f_t over
    (x_t, u_t, x_{t+1}, theta).  Returns (g, h) first and second derivative arrays."""
    x, u = split_z(ocp, z)
    if ocp.model.implicit:
        jets, k = constraint_jet(ocp, x, u, with_theta=True)
    else:
        jets, k = dynamics_jet(ocp, x[:, :-1], u, with_theta=True)
    g = np.stack([j.g for j in jets], axis=-2)    # (B, T, nx, k)
    h = np.stack([j.h for j in jets], axis=-3)    # (B, T, nx, k, k)
    return g, h


def dF_dtheta(ocp, z, lam, b, g=None, h=None):
    """Dense dF/dtheta, shape (n + m, p), for OCP b."""
    nx, nu, T = ocp.nx, ocp.nu, ocp.T
    mdl = ocp.model
    ps, pk = mdl.p_shared, mdl.p_knot
    n, m, p = ocp.n, ocp.m, ocp.p
    o_sh, o_kn, o_q, o_r, o_qt, _ = theta_offsets(mdl, T)
    if g is None:
        g, h = _phi_jets(ocp.one(b), z[b:b + 1])
        bb = 0
    else:
        bb = b
    x, u = split_z(ocp, z[b:b + 1])
    x, u = x[0], u[0]
    L = lam[b].reshape(T + 1, nx)
    M = np.zeros((n + m, p))
    if ocp.model.implicit:
        # f_t(x_t, u_t, x_{t+1}; theta): F_z rows of (x_t, u_t, x_{t+1}) get
        # (d^2 f_t / dz dtheta)^T lambda_{t+1}; the F_lambda row block of f_t gets df_t/dtheta
        zs = slice(0, 2 * nx + nu)
        for t in range(T):
            cols = np.concatenate([o_sh + np.arange(ps), o_kn + t * pk + np.arange(pk)]).astype(int)
            th = slice(2 * nx + nu, 2 * nx + nu + ps + pk)
            mixed = np.einsum("i,izj->zj", L[t + 1], h[bb, t][:, zs, th])
            rows = np.concatenate([x_index(nx, nu, t), u_index(nx, nu, t), x_index(nx, nu, t + 1)])
            M[np.ix_(rows, cols)] += mixed
            M[np.ix_(n + (t + 1) * nx + np.arange(nx), cols)] += g[bb, t][:, th]
    zs = slice(0, nx + nu)                 # seeds of (x_t, u_t)
    for t in range(T if not ocp.model.implicit else 0):
        cols = np.concatenate([o_sh + np.arange(ps), o_kn + t * pk + np.arange(pk)]).astype(int)
        th = slice(nx + nu, nx + nu + ps + pk)
        # F_z rows of (x_t, u_t): -(d^2 Phi_t / d(x,u) dtheta)^T lambda_{t+1}
        mixed = -np.einsum("i,izj->zj", L[t + 1], h[bb, t][:, zs, th])
        rows = np.concatenate([x_index(nx, nu, t), u_index(nx, nu, t)])
        M[np.ix_(rows, cols)] += mixed
        # F_lambda rows of f_t = x_{t+1} - Phi_t: -dPhi_t/dtheta
        M[np.ix_(n + (t + 1) * nx + np.arange(nx), cols)] += -g[bb, t][:, th]
    # cost gradient rows: grad c^x_t = Q (x_t - xref_t), grad c^u_t = R u_t
    dx = x - ocp.x_ref[b]
    for t in range(T):
        M[x_index(nx, nu, t), o_q + np.arange(nx)] += dx[t]
        M[u_index(nx, nu, t), o_r + np.arange(nu)] += u[t]
    M[x_index(nx, nu, T), o_qt + np.arange(nx)] += dx[T]
    return M


def exact_hessian_blocks(ocp, z, lam, b, h=None):
    """Per-stage blocks of grad^2_zz L over (x_t, u_t): diag(Q, R) + sum_i lambda_{t+1,i} grad^2 f_{t,i}
    with f_t = x_{t+1} - Phi_t, so grad^2 f_t = -grad^2 Phi_t.  True (unprojected) weights."""
    nx, nu, T = ocp.nx, ocp.nu, ocp.T
    if ocp.model.implicit:
        raise NotImplementedError("implicit integrators couple knots in the Lagrangian Hessian")
    _, _, qd, rd, qtd = split_theta(ocp.one(b))
    if h is None:
        _, h = _phi_jets(ocp.one(b), z[b:b + 1])
        bb = 0
    else:
        bb = b
    L = lam[b].reshape(T + 1, nx)
    blocks = []
    for t in range(T):
        Gt = np.diag(np.concatenate([qd[0], rd[0]]))
        Gt = Gt - np.einsum("i,ijk->jk", L[t + 1], h[bb, t][:, :nx + nu, :nx + nu])
        blocks.append(Gt)
    blocks.append(np.diag(qtd[0]))
    return blocks


def vjp(ocp, z, lam, dl_dz, hessian="gn", lam_fwd=None):
    """Algorithm 3 with a direct solve.  Returns dict(dtheta (B,p), dxs (B,nx), z_t, lam_t)."""
    qp = linearise(ocp, z)
    g, h = _phi_jets(ocp, z)
    B, n, m, nx = ocp.B, ocp.n, ocp.m, ocp.nx
    dtheta = np.zeros((B, ocp.p))
    dxs = np.zeros((B, nx))
    zt = np.zeros((B, n))
    lt = np.zeros((B, m))
    for b in range(B):
        Gb = exact_hessian_blocks(ocp, z, lam, b, h) if hessian == "exact" else None
        rhs = np.concatenate([dl_dz[b], np.zeros(m)])
        zt[b], lt[b] = solve_qp(qp, b, rhs=rhs, G_blocks=Gb)
        Mth = dF_dtheta(ocp, z, lam, b, g, h)
        dtheta[b] = -Mth.T @ np.concatenate([zt[b], lt[b]])
        dxs[b] = lt[b][:nx]
    return dict(dtheta=dtheta, dxs=dxs, z_t=zt, lam_t=lt)
