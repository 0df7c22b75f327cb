"""Finite-horizon discrete-time Riccati recursion with affine terms (textbook LQR):
an independent closed form for LQ OCPs, used to pin the KKT solve of Eq. 6.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Dynamics x_{t+1} = Abar_t x_t + Bbar_t u_t + c_t, cost sum_t 1/2 x^T Q_t x + q_t^T x
+ 1/2 u^T R_t u + r_t^T u (terminal Q_T, q_T).  Value function V_t(x) = 1/2 x^T P_t x + p_t^T x:
  P_T = Q_T, p_T = q_T;  for t = T-1 .. 0 with s = P_{t+1} c_t + p_{t+1}:
    Hxx = Q_t + Abar^T P Abar,  Huu = R_t + Bbar^T P Bbar,  Hux = Bbar^T P Abar
    hx = q_t + Abar^T s,        hu = r_t + Bbar^T s
    K_t = -Huu^-1 Hux,  k_t = -Huu^-1 hu
    P_t = Hxx + Hux^T K_t,  p_t = hx + Hux^T k_t
Rollout from x_0 = x_s with u_t = K_t x_t + k_t.  The multiplier of the constraint that
defines x_t (x_0 = x_s for t = 0) is the negative value gradient: lambda_t = -(P_t x_t + p_t).
"""
import numpy as np


def riccati_solve(Abar, Bbar, c, Qd, q, Rd, r, x_s):
    """Single OCP.  Abar (T,nx,nx), Bbar (T,nx,nu), c (T,nx), Qd (T+1,nx) diag, q (T+1,nx),
    Rd (T,nu) diag, r (T,nu), x_s (nx,).  Returns x (T+1,nx), u (T,nu), lam (T+1,nx)."""
    T, nx = Abar.shape[0], Abar.shape[1]
    nu = Bbar.shape[2]
    P = np.diag(Qd[T])
    p = q[T].copy()
    Ps, ps, Ks, ks = [None] * (T + 1), [None] * (T + 1), [None] * T, [None] * T
    Ps[T], ps[T] = P, p
    for t in range(T - 1, -1, -1):
        A, Bm = Abar[t], Bbar[t]
        s = P @ c[t] + p
        Hxx = np.diag(Qd[t]) + A.T @ P @ A
        Huu = np.diag(Rd[t]) + Bm.T @ P @ Bm
        Hux = Bm.T @ P @ A
        hx = q[t] + A.T @ s
        hu = r[t] + Bm.T @ s
        Kt = -np.linalg.solve(Huu, Hux)
        kt = -np.linalg.solve(Huu, hu)
        P = Hxx + Hux.T @ Kt
        P = 0.5 * (P + P.T)
        p = hx + Hux.T @ kt
        Ps[t], ps[t], Ks[t], ks[t] = P, p, Kt, kt
    x = np.zeros((T + 1, nx))
    u = np.zeros((T, nu))
    x[0] = x_s
    for t in range(T):
        u[t] = Ks[t] @ x[t] + ks[t]
        x[t + 1] = Abar[t] @ x[t] + Bbar[t] @ u[t] + c[t]
    lam = np.stack([-(Ps[t] @ x[t] + ps[t]) for t in range(T + 1)])
    return x, u, lam
