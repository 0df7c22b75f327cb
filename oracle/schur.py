"""Schur complement, symmetric stair preconditioner, PCG and primal recovery in FP64
(Sec. 3.3: Eq. 8-11; App. A.2: gamma; App. A.2 Algorithm 4: PCG).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper writes S := -H G^-1 H^T (negative definite).  Following the usual PCG setting
this module works with the SPD matrix S_spd = H G^-1 H^T = -S and the right-hand side
gamma_spd = -gamma, which leave lambda unchanged.  Block rows i = 0..T of S_spd:
  D_0 = Q_0^-1,  D_{t+1} = chi_t = A_t Q_t^-1 A_t^T + B_t R_t^-1 B_t^T + A_t^+ Q_{t+1}^-1 A_t^+T
  O_{t+1,t} = phi_t = A_t Q_t^-1 A_{t-1}^+T  (A_{-1}^+ = I),  O_{t,t+1} = phi_t^T
The preconditioner is Phi^-1 = D^-1 - D^-1 O D^-1 (block diagonal D, off-diagonal O),
which reproduces every block Eq. 10 displays.
All functions take a batch of OCPs: leading axis B.
"""
import numpy as np


def _inv_diag(d):
    return 1.0 / d


def _a_plus_prev(Ap, t):
    """A_{t-1}^+ with A_{-1}^+ = I."""
    if t == 0:
        return np.broadcast_to(np.eye(Ap.shape[-1]), Ap[:, 0].shape)
    return Ap[:, t - 1]


def schur_blocks(qp):
    """S_spd blocks (D: (B, T+1, nx, nx), O: (B, T+1, nx, nx), O[:,0] unused = 0) of Eq. 10."""
    Bn, T, nx = qp.A.shape[0], qp.A.shape[1], qp.A.shape[2]
    Qi = _inv_diag(qp.Q)            # (B, T+1, nx)
    Ri = _inv_diag(qp.R)            # (B, T, nu)
    D = np.zeros((Bn, T + 1, nx, nx))
    O = np.zeros((Bn, T + 1, nx, nx))
    D[:, 0] = np.einsum("bi,ij->bij", Qi[:, 0], np.eye(nx))
    for t in range(T):
        A, Bm, Ap = qp.A[:, t], qp.Bm[:, t], qp.Ap[:, t]
        chi = (np.einsum("bik,bk,bjk->bij", A, Qi[:, t], A)
               + np.einsum("bik,bk,bjk->bij", Bm, Ri[:, t], Bm)
               + np.einsum("bik,bk,bjk->bij", Ap, Qi[:, t + 1], Ap))
        phi = np.einsum("bik,bk,bjk->bij", A, Qi[:, t], _a_plus_prev(qp.Ap, t))
        D[:, t + 1] = chi
        O[:, t + 1] = phi
    return D, O


def gamma_spd(qp, q=None, r=None, d=None):
    """gamma_spd = -(d + (Q_0^-1 q_0, zeta_0, ..., zeta_{T-1})), App. A.2,
    zeta_t = A_t Q_t^-1 q_t + B_t R_t^-1 r_t + A_t^+ Q_{t+1}^-1 q_{t+1}.
    Defaults: q, r from the QP and d = (x_s, C_0..C_{T-1}) (Eq. 6)."""
    q = qp.q if q is None else q
    r = qp.r if r is None else r
    if d is None:
        d = np.concatenate([qp.x_s[:, None], qp.C], axis=1)
    Qi, Ri = _inv_diag(qp.Q), _inv_diag(qp.R)
    g = np.empty_like(d)
    g[:, 0] = Qi[:, 0] * q[:, 0]
    g[:, 1:] = (np.einsum("btij,btj->bti", qp.A, Qi[:, :-1] * q[:, :-1])
                + np.einsum("btij,btj->bti", qp.Bm, Ri * r)
                + np.einsum("btij,btj->bti", qp.Ap, Qi[:, 1:] * q[:, 1:]))
    return -(d + g)


def preconditioner_blocks(D, O):
    """Phi^-1 blocks: diagonal D_i^-1 and sub-diagonal -D_i^-1 O_{i,i-1} D_{i-1}^-1 (Eq. 10)."""
    Dinv = np.linalg.inv(D)
    P = np.zeros_like(O)
    P[:, 1:] = -np.einsum("btij,btjk,btkl->btil", Dinv[:, 1:], O[:, 1:], Dinv[:, :-1])
    return Dinv, P


def block_tridiag_matvec(Md, Mo, v):
    """(M v)_i = Md_i v_i + Mo_i v_{i-1} + Mo_{i+1}^T v_{i+1} for symmetric block-tridiagonal M."""
    y = np.einsum("btij,btj->bti", Md, v)
    y[:, 1:] += np.einsum("btij,btj->bti", Mo[:, 1:], v[:, :-1])
    y[:, :-1] += np.einsum("btji,btj->bti", Mo[:, 1:], v[:, 1:])
    return y


def dense_block_tridiag(Md, Mo, b):
    K, nx = Md.shape[1], Md.shape[2]
    M = np.zeros((K * nx, K * nx))
    for i in range(K):
        M[i * nx:(i + 1) * nx, i * nx:(i + 1) * nx] = Md[b, i]
        if i > 0:
            M[i * nx:(i + 1) * nx, (i - 1) * nx:i * nx] = Mo[b, i]
            M[(i - 1) * nx:i * nx, i * nx:(i + 1) * nx] = Mo[b, i].T
    return M


def pcg(D, O, Pd, Po, gamma, lam0, rel_tol, max_iter):
    """Algorithm 4 on S_spd lambda = gamma_spd, batched; each OCP stops on its own when
    eta <= rel_tol * eta_0 with eta_0 = gamma^T Phi^-1 gamma, or after max_iter iterations.
    Returns (lambda, iterations, final eta, eta_0)."""
    lam = lam0.copy()
    r = gamma - block_tridiag_matvec(D, O, lam)
    rt = block_tridiag_matvec(Pd, Po, r)
    p = rt.copy()
    eta = np.einsum("bti,bti->b", r, rt)
    eta0 = np.einsum("bti,bti->b", gamma, block_tridiag_matvec(Pd, Po, gamma))
    iters = np.zeros(lam.shape[0], dtype=np.int64)
    active = eta > rel_tol * eta0
    for _ in range(max_iter):
        if not active.any():
            break
        y = block_tridiag_matvec(D, O, p)
        v = np.einsum("bti,bti->b", p, y)
        alpha = np.where(active, eta / np.where(active, v, 1.0), 0.0)
        lam += alpha[:, None, None] * p
        r -= alpha[:, None, None] * y
        rt = block_tridiag_matvec(Pd, Po, r)
        eta_new = np.einsum("bti,bti->b", r, rt)
        beta = np.where(active, eta_new / np.where(active, eta, 1.0), 0.0)
        p = np.where(active[:, None, None], rt + beta[:, None, None] * p, p)
        eta = np.where(active, eta_new, eta)
        iters += active
        active = active & (eta > rel_tol * eta0)
    return lam, iters, eta, eta0


def recover_primal(qp, lam, q=None, r=None):
    """Eq. 11: x_t = -Q_t^-1 (q_t + A_{t-1}^+T lam_t + A_t^T lam_{t+1}),
    u_t = -R_t^-1 (r_t + B_t^T lam_{t+1}),  x_T = -Q_T^-1 (q_T + A_{T-1}^+T lam_T)."""
    q = qp.q if q is None else q
    r = qp.r if r is None else r
    T = qp.A.shape[1]
    ax = q.copy()
    ax[:, 0] += lam[:, 0]
    ax[:, 1:] += np.einsum("btji,btj->bti", qp.Ap, lam[:, 1:])
    ax[:, :T] += np.einsum("btji,btj->bti", qp.A, lam[:, 1:])
    au = r + np.einsum("btji,btj->bti", qp.Bm, lam[:, 1:])
    return -ax / qp.Q, -au / qp.R
