"""OCP batch, QP linearisation (Eq. 4) and KKT system (Eq. 5-6) for the FP64 oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Conventions (shared with the C-ABI by specification, not by code):
  z      = (x_0, u_0, x_1, u_1, ..., x_{T-1}, u_{T-1}, x_T)   (Sec. 3.1), n = (T+1) nx + T nu
  lambda = (lambda_0, ..., lambda_T), lambda_0 the multiplier of x_0 = x_s,
           lambda_{t+1} the multiplier of f_t = 0;                   m = (T+1) nx
  theta  = [shared model params (p_s) | per-knot model params (T x p_k) |
            diag Q (nx) | diag R (nu) | diag Q_T (nx)]
  costs  c_t^x(x) = 1/2 (x - xref_t)^T diag(Q) (x - xref_t)  for t < T, diag(Q_T) at t = T,
         c_t^u(u) = 1/2 u^T diag(R) u.
The Lagrangian is L = sum c + lambda^T g with g = (x_0 - x_s, f_0, ..., f_{T-1}) (Eq. 1).
"""
from dataclasses import dataclass

import numpy as np
import scipy.linalg

from .jet import Jet, value

PD_EPS = 1e-6  # PD projection floor, relative to max(1, largest diagonal entry)


@dataclass
class OCPBatch:
    model: object
    T: int
    x_s: np.ndarray     # (B, nx)
    theta: np.ndarray   # (B, p)
    x_ref: np.ndarray   # (B, T+1, nx)

    @property
    def B(self):
        return self.x_s.shape[0]

    @property
    def nx(self):
        return self.model.nx

    @property
    def nu(self):
        return self.model.nu

    @property
    def K(self):
        return self.T + 1

    @property
    def n(self):
        return self.K * self.nx + self.T * self.nu

    @property
    def m(self):
        return self.K * self.nx

    @property
    def p(self):
        return theta_size(self.model, self.T)

    def one(self, b):
        return OCPBatch(self.model, self.T, self.x_s[b:b + 1], self.theta[b:b + 1], self.x_ref[b:b + 1])


def theta_size(model, T):
    return model.p_shared + T * model.p_knot + 2 * model.nx + model.nu


def theta_offsets(model, T):
    """Offsets of the theta blocks: shared, knot, Q, R, Q_T, end."""
    o_sh = 0
    o_kn = model.p_shared
    o_q = o_kn + T * model.p_knot
    o_r = o_q + model.nx
    o_qt = o_r + model.nu
    return o_sh, o_kn, o_q, o_r, o_qt, o_qt + model.nx


def split_theta(ocp):
    o_sh, o_kn, o_q, o_r, o_qt, end = theta_offsets(ocp.model, ocp.T)
    th = ocp.theta
    B = th.shape[0]
    ths = th[:, o_sh:o_kn]
    thk = th[:, o_kn:o_q].reshape(B, ocp.T, ocp.model.p_knot)
    return ths, thk, th[:, o_q:o_r], th[:, o_r:o_qt], th[:, o_qt:end]


def split_z(ocp, z):
    """Interleaved z (B, n) -> x (B, T+1, nx), u (B, T, nu)."""
    B, nx, nu, T = z.shape[0], ocp.nx, ocp.nu, ocp.T
    head = z[:, :T * (nx + nu)].reshape(B, T, nx + nu)
    x = np.concatenate([head[:, :, :nx], z[:, None, T * (nx + nu):]], axis=1)
    return x, head[:, :, nx:]


def join_z(x, u):
    B, K, nx = x.shape
    T = K - 1
    head = np.concatenate([x[:, :T], u], axis=2).reshape(B, -1)
    return np.concatenate([head, x[:, T]], axis=1)


def pd_project_diag(d):
    """Project a diagonal Hessian onto the PD cone (Sec. 3.1): clamp each eigenvalue
    (diagonal entry) below at PD_EPS * max(1, largest entry)."""
    floor = PD_EPS * np.maximum(1.0, d.max(axis=-1, keepdims=True))
    return np.maximum(d, floor)


def dynamics_values(ocp, x, u, t0=0):
    """Phi_t(x_t, u_t), plain values, for knots t = t0 .. t0 + x.shape[1] - 1 (all t < T by
    default).  x: (B, k, nx), u: (B, k, nu)."""
    ths, thk, _, _, _ = split_theta(ocp)
    thk = thk[:, t0:t0 + x.shape[1]]
    mdl = ocp.model
    xs = [x[..., i] for i in range(mdl.nx)]
    us = [u[..., i] for i in range(mdl.nu)]
    sh = [ths[:, None, i] for i in range(mdl.p_shared)]
    kn = [thk[..., i] for i in range(mdl.p_knot)]
    out = mdl.step(xs, us, sh, kn)
    return np.stack([np.broadcast_to(value(o), x.shape[:2]) for o in out], axis=-1)


def constraint_residual(ocp, z):
    """g(z) = (x_0 - x_s, f_0, ..., f_{T-1}), f_t = x_{t+1} - Phi_t(x_t, u_t) (or the implicit
    trapezoidal residual).  (B, T+1, nx)."""
    x, u = split_z(ocp, z)
    g = np.empty_like(x)
    g[:, 0] = x[:, 0] - ocp.x_s
    if ocp.model.implicit:
        ths, thk, _, _, _ = split_theta(ocp)
        mdl = ocp.model
        xs = [x[:, :-1, i] for i in range(mdl.nx)]
        xn = [x[:, 1:, i] for i in range(mdl.nx)]
        us = [u[..., i] for i in range(mdl.nu)]
        sh = [ths[:, None, i] for i in range(mdl.p_shared)]
        out = mdl.residual(xs, us, xn, sh, [thk[..., i] for i in range(mdl.p_knot)])
        g[:, 1:] = np.stack([np.broadcast_to(value(o), x[:, 1:].shape[:2]) for o in out], axis=-1)
        return g
    phi = dynamics_values(ocp, x[:, :-1], u)
    g[:, 1:] = x[:, 1:] - phi
    return g


def dynamics_jet(ocp, x, u, with_theta=False):
    """Phi_t as Jets seeded on (x_t, u_t[, theta_shared, theta_knot_t]); x: (B,T,nx), u: (B,T,nu).

    Returns (list of nx Jets over (B, T), k, index slices)."""
    mdl = ocp.model
    ths, thk, _, _, _ = split_theta(ocp)
    nx, nu, ps, pk = mdl.nx, mdl.nu, mdl.p_shared, mdl.p_knot
    k = nx + nu + ((ps + pk) if with_theta else 0)
    shape = x.shape[:2]
    xs = [Jet.seed(x[..., i], i, k) for i in range(nx)]
    us = [Jet.seed(u[..., i], nx + i, k) for i in range(nu)]
    if with_theta:
        sh = [Jet.seed(np.broadcast_to(ths[:, None, i], shape), nx + nu + i, k) for i in range(ps)]
        kn = [Jet.seed(thk[..., i], nx + nu + ps + i, k) for i in range(pk)]
    else:
        sh = [ths[:, None, i] for i in range(ps)]
        kn = [thk[..., i] for i in range(pk)]
    out = mdl.step(xs, us, sh, kn)
    out = [o if isinstance(o, Jet) else Jet(np.broadcast_to(o, shape), np.zeros(shape + (k,)),
                                            np.zeros(shape + (k, k))) for o in out]
    return out, k


def constraint_jet(ocp, x, u, with_theta=False):
    """f_t as Jets seeded on (x_t, u_t, x_{t+1}[, theta_shared, theta_knot_t]) for the implicit
    integrators; x: (B, T+1, nx), u: (B, T, nu).  Returns (list of nx Jets over (B, T), k)."""
    mdl = ocp.model
    ths, thk, _, _, _ = split_theta(ocp)
    nx, nu, ps, pk = mdl.nx, mdl.nu, mdl.p_shared, mdl.p_knot
    k = 2 * nx + nu + ((ps + pk) if with_theta else 0)
    shape = u.shape[:2]
    xs = [Jet.seed(x[:, :-1, i], i, k) for i in range(nx)]
    us = [Jet.seed(u[..., i], nx + i, k) for i in range(nu)]
    xn = [Jet.seed(x[:, 1:, i], nx + nu + i, k) for i in range(nx)]
    if with_theta:
        sh = [Jet.seed(np.broadcast_to(ths[:, None, i], shape), 2 * nx + nu + i, k) for i in range(ps)]
        kn = [Jet.seed(thk[..., i], 2 * nx + nu + ps + i, k) for i in range(pk)]
    else:
        sh = [ths[:, None, i] for i in range(ps)]
        kn = [thk[..., i] for i in range(pk)]
    out = mdl.residual(xs, us, xn, sh, kn)
    return out, k


@dataclass
class QP:
    """QP data of Sec. 3.1 at the linearisation point, all (B, ...) arrays."""
    Q: np.ndarray    # (B, T+1, nx) diagonal of Q_t (Q_T at t = T)
    q: np.ndarray    # (B, T+1, nx)
    R: np.ndarray    # (B, T, nu)   diagonal of R_t
    r: np.ndarray    # (B, T, nu)
    A: np.ndarray    # (B, T, nx, nx)  A_t   = d f_t / d x_t
    Bm: np.ndarray   # (B, T, nx, nu)  B_t   = d f_t / d u_t
    Ap: np.ndarray   # (B, T, nx, nx)  A_t^+ = d f_t / d x_{t+1}
    C: np.ndarray    # (B, T, nx)      C_t = A^+ x_{t+1} + A x_t + B u_t - f_t
    x_s: np.ndarray  # (B, nx)
    f: np.ndarray    # (B, T, nx)      f_t at the linearisation point


def cost_hessians(ocp):
    _, _, qd, rd, qtd = split_theta(ocp)
    K = ocp.K
    Qd = np.repeat(pd_project_diag(qd)[:, None, :], K, axis=1)
    Qd[:, -1] = pd_project_diag(qtd)
    Rd = np.repeat(pd_project_diag(rd)[:, None, :], ocp.T, axis=1)
    return Qd, Rd


def cost_value(ocp, z):
    """sum_t c_t^x(x_t) + sum_t c_t^u(u_t) per OCP (true costs, unprojected weights)."""
    _, _, qd, rd, qtd = split_theta(ocp)
    x, u = split_z(ocp, z)
    dx = x - ocp.x_ref
    cx = 0.5 * np.einsum("btn,bn->b", dx[:, :-1] ** 2, qd) + 0.5 * np.einsum("bn,bn->b", dx[:, -1] ** 2, qtd)
    cu = 0.5 * np.einsum("btn,bn->b", u ** 2, rd)
    return cx + cu


def cost_gradient(ocp, z):
    """grad_z of the cost, laid out like z."""
    _, _, qd, rd, qtd = split_theta(ocp)
    x, u = split_z(ocp, z)
    gx = (x - ocp.x_ref) * qd[:, None, :]
    gx[:, -1] = (x[:, -1] - ocp.x_ref[:, -1]) * qtd
    gu = u * rd[:, None, :]
    return join_z(gx, gu)


def linearise(ocp, z):
    """QP matrices of Eq. 4 at z, with the Delta-form linear terms q_t = grad c - Q_t x_t
    (so that the QP is posed in absolute z as in Sec. 3.1) and C_t from its definition."""
    x, u = split_z(ocp, z)
    nx, nu, T = ocp.nx, ocp.nu, ocp.T
    if ocp.model.implicit:
        jets, _ = constraint_jet(ocp, x, u)
        f = np.stack([j.v for j in jets], axis=-1)             # (B, T, nx)
        jac = np.stack([j.g for j in jets], axis=-2)           # (B, T, nx, 2nx+nu)
        A = jac[..., :nx].copy()
        Bm = jac[..., nx:nx + nu].copy()
        Ap = jac[..., nx + nu:2 * nx + nu].copy()
    else:
        jets, _ = dynamics_jet(ocp, x[:, :-1], u)
        phi = np.stack([j.v for j in jets], axis=-1)           # (B, T, nx)
        jac = np.stack([j.g for j in jets], axis=-2)           # (B, T, nx, nx+nu)
        A = -jac[..., :nx]
        Bm = -jac[..., nx:nx + nu]
        Ap = np.broadcast_to(np.eye(nx), A.shape).copy()
        f = x[:, 1:] - phi
    C = (np.einsum("btij,btj->bti", Ap, x[:, 1:]) + np.einsum("btij,btj->bti", A, x[:, :-1])
         + np.einsum("btij,btj->bti", Bm, u) - f)
    Qd, Rd = cost_hessians(ocp)
    gz = cost_gradient(ocp, z)
    gx, gu = split_z(ocp, gz)
    q = gx - Qd * x
    r = gu - Rd * u
    return QP(Qd, q, Rd, r, A, Bm, Ap, C, ocp.x_s.copy(), f)


# ---------------------------------------------------------------------------------
# Index maps for the KKT matrix of Eq. 5 (z ordering of Sec. 3.1, then lambda).
def x_index(nx, nu, t):
    return t * (nx + nu) + np.arange(nx)


def u_index(nx, nu, t):
    return t * (nx + nu) + nx + np.arange(nu)


def kkt_triplets(qp, b, G_blocks=None):
    """Nonzeros (rows, cols, vals) of the KKT matrix [G H^T; H 0] of Eq. 5 for OCP b,
    in the ordering (z, lambda).  G is block diagonal: diag(Q_t), diag(R_t) by default,
    or the dense per-stage blocks G_blocks[t] over (x_t, u_t) (x_T alone at t = T)."""
    T, nx = qp.A.shape[1], qp.A.shape[2]
    nu = qp.Bm.shape[3]
    K = T + 1
    n = K * nx + T * nu
    rows, cols, vals = [], [], []

    def put(ri, ci, M):
        M = np.atleast_2d(M)
        rr, cc = np.meshgrid(ri, ci, indexing="ij")
        rows.append(rr.ravel()); cols.append(cc.ravel()); vals.append(M.ravel())

    for t in range(K):
        ix = x_index(nx, nu, t)
        if G_blocks is None:
            put(ix, ix, np.diag(qp.Q[b, t]))
            if t < T:
                iu = u_index(nx, nu, t)
                put(iu, iu, np.diag(qp.R[b, t]))
        else:
            idx = ix if t == T else np.concatenate([ix, u_index(nx, nu, t)])
            put(idx, idx, G_blocks[t])
    # H (rows n + constraint index) and its transpose
    hblocks = [(np.arange(nx), x_index(nx, nu, 0), np.eye(nx))]
    for t in range(T):
        r_ = (t + 1) * nx + np.arange(nx)
        hblocks += [(r_, x_index(nx, nu, t), qp.A[b, t]), (r_, u_index(nx, nu, t), qp.Bm[b, t]),
                    (r_, x_index(nx, nu, t + 1), qp.Ap[b, t])]
    for r_, c_, M in hblocks:
        put(n + r_, c_, M)
        put(c_, n + r_, np.asarray(M).T)
    return np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), n


def kkt_dense(qp, b, G_blocks=None):
    r_, c_, v_, n = kkt_triplets(qp, b, G_blocks)
    N = n + qp.A.shape[1] * qp.A.shape[2] + qp.A.shape[2]
    M = np.zeros((N, N))
    np.add.at(M, (r_, c_), v_)
    return M


def kkt_rhs(qp, b):
    """(-b, d) of Eq. 6: b = (q_0, r_0, ..., q_T), d = (x_s, C_0, ..., C_{T-1})."""
    bvec = join_z(qp.q[b:b + 1], qp.r[b:b + 1])[0]
    d = np.concatenate([qp.x_s[b], qp.C[b].reshape(-1)])
    return -bvec, d


def stage_permutation(nx, nu, T):
    """Order unknowns by time stage: (lambda_t, x_t, u_t) for t = 0..T (no u_T)."""
    n = (T + 1) * nx + T * nu
    perm = []
    for t in range(T + 1):
        perm.extend(n + t * nx + np.arange(nx))       # lambda_t
        perm.extend(x_index(nx, nu, t))               # x_t
        if t < T:
            perm.extend(u_index(nx, nu, t))           # u_t
    return np.array(perm)


def solve_kkt_banded(trip, rhs, nx, nu, T):
    """Solve the KKT system after reordering the unknowns by time stage, where the matrix
    is banded (half-bandwidth about 2 nx + nu): LAPACK banded LU with partial pivoting."""
    r_, c_, v_, _ = trip
    perm = stage_permutation(nx, nu, T)
    N = perm.size
    pos = np.empty(N, dtype=np.int64)
    pos[perm] = np.arange(N)
    pr, pc = pos[r_], pos[c_]
    lo = int(max(0, (pr - pc).max()))
    up = int(max(0, (pc - pr).max()))
    ab = np.zeros((lo + up + 1, N))
    np.add.at(ab, (up + pr - pc, pc), v_)
    sol_p = scipy.linalg.solve_banded((lo, up), ab, rhs[perm])
    return sol_p[pos]


def solve_qp(qp, b, rhs=None, G_blocks=None, dense=False):
    """Solve Eq. 6 (or Eq. 7 when rhs is given) for OCP b; returns (z, lambda).
    dense=True: brute-force LU of the dense KKT matrix (small T only)."""
    T, nx, nu = qp.A.shape[1], qp.A.shape[2], qp.Bm.shape[3]
    n = (T + 1) * nx + T * nu
    if rhs is None:
        mb, d = kkt_rhs(qp, b)
        rhs = np.concatenate([mb, d])
    if dense:
        sol = np.linalg.solve(kkt_dense(qp, b, G_blocks), rhs)
    else:
        sol = solve_kkt_banded(kkt_triplets(qp, b, G_blocks), rhs, nx, nu, T)
    return sol[:n], sol[n:]


def kkt_residual(ocp, z, lam):
    """F(z, lambda) of Eq. 1 for the OCP: (grad_z c + (dg/dz)^T lambda, g).  Returns (Fz, Fl)."""
    x, u = split_z(ocp, z)
    nx, nu, T = ocp.nx, ocp.nu, ocp.T
    L = lam.reshape(lam.shape[0], T + 1, nx)
    gz = cost_gradient(ocp, z)
    gx, gu = split_z(ocp, gz)
    if ocp.model.implicit:
        jets, _ = constraint_jet(ocp, x, u)
        jac = np.stack([j.g for j in jets], axis=-2)  # df_t/d(x_t, u_t, x_{t+1})
        gx = gx.copy()
        gx[:, 0] += L[:, 0]
        gx[:, :-1] += np.einsum("btij,bti->btj", jac[..., :nx], L[:, 1:])
        gx[:, 1:] += np.einsum("btij,bti->btj", jac[..., nx + nu:], L[:, 1:])
        gu = gu + np.einsum("btij,bti->btj", jac[..., nx:nx + nu], L[:, 1:])
        return join_z(gx, gu), constraint_residual(ocp, z).reshape(z.shape[0], -1)
    jets, _ = dynamics_jet(ocp, x[:, :-1], u)
    jac = np.stack([j.g for j in jets], axis=-2)     # dPhi/d(x,u): (B, T, nx, nx+nu)
    # g_0 = x_0 - x_s contributes lambda_0 to x_0; f_t = x_{t+1} - Phi_t contributes
    # lambda_{t+1} to x_{t+1} and -(dPhi/dx)^T lambda_{t+1}, -(dPhi/du)^T lambda_{t+1}.
    gx = gx + L
    gx[:, :-1] -= np.einsum("btij,bti->btj", jac[..., :nx], L[:, 1:])
    gu = gu - np.einsum("btij,bti->btj", jac[..., nx:], L[:, 1:])
    return join_z(gx, gu), constraint_residual(ocp, z).reshape(z.shape[0], -1)
