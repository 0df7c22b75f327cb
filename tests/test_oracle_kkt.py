"""Pins of the oracle's QP/KKT solve (Eq. 5-6), Schur complement and preconditioner
(Eq. 8-10, App. A.2), PCG (Algorithm 4) and recovery (Eq. 11) against the Riccati closed
form, brute-force dense LU, dense H G^-1 H^T and the structure the paper displays."""
import numpy as np
import pytest

from paper_2510_06179_gb300 import workloads
from oracle import ocp as O
from oracle import schur as S
from oracle.riccati import riccati_solve
from oracle.sqp import cold_start, sqp
from tests.oracle_helpers import to_ocp


def _lq(B=4, T=5, nx=4, nu=1, seed=3, c_var=0.0):
    w = workloads.lq_config(B=B, T=T, nx=nx, nu=nu, seed=seed, c_var=c_var)
    return w, to_ocp(w)


def _riccati_for(ocp, b, qp):
    nx, nu, T = ocp.nx, ocp.nu, ocp.T
    ths, thk, qd, rd, qtd = O.split_theta(ocp)
    Abar = thk[b, :, :nx * nx].reshape(T, nx, nx)
    Bbar = thk[b, :, nx * nx:nx * nx + nx * nu].reshape(T, nx, nu)
    c = thk[b, :, nx * nx + nx * nu:]
    return riccati_solve(Abar, Bbar, c, qp.Q[b], qp.q[b], qp.R[b], qp.r[b], ocp.x_s[b])


@pytest.mark.parametrize("c_var", [0.0, 0.01])
def test_lq_kkt_matches_riccati(c_var):
    """One QP of an LQ OCP = the finite-horizon LQR solution (states, inputs, multipliers)."""
    w, ocp = _lq(B=3, T=20, c_var=c_var)
    z0, _ = cold_start(ocp)
    qp = O.linearise(ocp, z0)
    for b in range(ocp.B):
        z, lam = O.solve_qp(qp, b)
        x, u = O.split_z(ocp, z[None])
        xr, ur, lr = _riccati_for(ocp, b, qp)
        np.testing.assert_allclose(x[0], xr, rtol=1e-10, atol=1e-11)
        np.testing.assert_allclose(u[0], ur, rtol=1e-10, atol=1e-11)
        np.testing.assert_allclose(lam.reshape(-1, ocp.nx), lr, rtol=1e-9, atol=1e-10)


def test_lq_one_sqp_step_is_lqr_from_any_start():
    """The Delta-form QP in absolute z makes one full SQP step exact for LQ from any z."""
    w, ocp = _lq(B=2, T=12, c_var=0.01)
    rng = np.random.default_rng(0)
    z0 = rng.standard_normal((ocp.B, ocp.n))
    out = sqp(ocp, 1, line_search_on=False, z0=z0)
    qp = O.linearise(ocp, z0)
    for b in range(ocp.B):
        xr, ur, _ = _riccati_for(ocp, b, qp)
        np.testing.assert_allclose(out["z"][b], O.join_z(xr[None], ur[None])[0], rtol=1e-10, atol=1e-11)


@pytest.mark.parametrize("name", ["lq", "cartpole"])
def test_banded_solve_matches_dense_lu(name):
    """Banded LU on the time-ordered KKT system vs brute-force dense LU (T <= 5)."""
    if name == "lq":
        w, ocp = _lq(B=2, T=5)
    else:
        w = workloads.cartpole_config(B=2, T=5, seed=1)
        ocp = to_ocp(w)
    rng = np.random.default_rng(5)
    z = rng.standard_normal((ocp.B, ocp.n))
    qp = O.linearise(ocp, z)
    for b in range(ocp.B):
        zb, lb = O.solve_qp(qp, b)
        zd, ld = O.solve_qp(qp, b, dense=True)
        np.testing.assert_allclose(zb, zd, rtol=1e-11, atol=1e-12)
        np.testing.assert_allclose(lb, ld, rtol=1e-11, atol=1e-12)
        # and the KKT equations of Eq. 6 hold
        Kd = O.kkt_dense(qp, b)
        mb, d = O.kkt_rhs(qp, b)
        np.testing.assert_allclose(Kd @ np.concatenate([zb, lb]), np.concatenate([mb, d]), atol=1e-10)


def test_kkt_matrix_structure_eq5():
    """G block diagonal (Q_0, R_0, ..., Q_T); H first block row [I 0 ...], then [A_t B_t A_t^+]."""
    w, ocp = _lq(B=1, T=3, nx=2, nu=1)
    qp = O.linearise(ocp, cold_start(ocp)[0])
    K = O.kkt_dense(qp, 0)
    n = ocp.n
    G, H = K[:n, :n], K[n:, :n]
    assert np.allclose(K[:n, n:], H.T) and np.allclose(K[n:, n:], 0)
    assert np.allclose(G, np.diag(np.diag(G)))
    assert np.allclose(H[:2, :2], np.eye(2)) and np.allclose(H[:2, 2:], 0)
    # second block row: A_0 at x_0, B_0 at u_0, A_0^+ = I at x_1
    np.testing.assert_allclose(H[2:4, 0:2], qp.A[0, 0])
    np.testing.assert_allclose(H[2:4, 2:3], qp.Bm[0, 0])
    np.testing.assert_allclose(H[2:4, 3:5], np.eye(2))


def _dense_GH(qp, b):
    K = O.kkt_dense(qp, b)
    n = qp.Q.shape[1] * qp.Q.shape[2] + qp.R.shape[1] * qp.R.shape[2]
    return K[:n, :n], K[n:, :n]


@pytest.mark.parametrize("name", ["lq", "cartpole", "kin_bicycle"])
def test_schur_blocks_match_dense(name):
    """chi_t, phi_t (Eq. 10) and gamma (App. A.2) vs dense H G^-1 H^T and d + H G^-1 b."""
    mk = {"lq": lambda: _lq(B=2, T=4, c_var=0.01)[0],
          "cartpole": lambda: workloads.cartpole_config(B=2, T=4, seed=2),
          "kin_bicycle": lambda: workloads.bicycle_config(B=2, T=4, seed=2)}[name]
    w = mk()
    ocp = to_ocp(w)
    rng = np.random.default_rng(9)
    z = rng.standard_normal((ocp.B, ocp.n))
    qp = O.linearise(ocp, z)
    D, Off = S.schur_blocks(qp)
    gam = S.gamma_spd(qp)
    for b in range(ocp.B):
        G, H = _dense_GH(qp, b)
        Sd = H @ np.linalg.solve(G, H.T)
        np.testing.assert_allclose(S.dense_block_tridiag(D, Off, b), Sd, rtol=1e-11, atol=1e-12)
        mb, d = O.kkt_rhs(qp, b)
        gd = d + H @ np.linalg.solve(G, -mb)
        np.testing.assert_allclose(gam[b].reshape(-1), -gd, rtol=1e-11, atol=1e-12)


def test_preconditioner_matches_displayed_blocks():
    """The first block rows of Phi^-1 as displayed in Eq. 10 (negative-definite convention
    there, so in terms of Q_0^-1, chi_t, phi_t): Q_0, -Q_0 phi_0^T chi_0^-1, chi_0^-1,
    -chi_0^-1 phi_1^T chi_1^-1, -chi_1^-1 phi_1 chi_0^-1, chi_1^-1."""
    w, ocp = _lq(B=1, T=4)
    qp = O.linearise(ocp, cold_start(ocp)[0])
    D, Off = S.schur_blocks(qp)
    Pd, Po = S.preconditioner_blocks(D, Off)
    P = S.dense_block_tridiag(Pd, Po, 0)
    nx = ocp.nx
    Q0 = np.diag(qp.Q[0, 0])
    chi0, chi1 = D[0, 1], D[0, 2]
    phi0, phi1 = Off[0, 1], Off[0, 2]
    blk = lambda i, j: P[i * nx:(i + 1) * nx, j * nx:(j + 1) * nx]
    inv = np.linalg.inv
    np.testing.assert_allclose(blk(0, 0), Q0, rtol=1e-12)
    np.testing.assert_allclose(blk(0, 1), -Q0 @ phi0.T @ inv(chi0), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(blk(1, 1), inv(chi0), rtol=1e-10)
    np.testing.assert_allclose(blk(1, 2), -inv(chi0) @ phi1.T @ inv(chi1), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(blk(2, 1), -inv(chi1) @ phi1 @ inv(chi0), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(blk(2, 2), inv(chi1), rtol=1e-10)
    assert np.allclose(blk(0, 2), 0)


def test_preconditioner_spd_and_exact_without_coupling():
    """Phi^-1 is SPD whenever S_spd is (block-tridiagonal => spectrum of D^-1/2 O D^-1/2 is
    symmetric about 0); with all off-diagonal blocks zero, Phi^-1 = S^-1 and PCG stops after
    one iteration."""
    for seed in range(5):
        w, ocp = _lq(B=2, T=8, seed=seed)
        rng = np.random.default_rng(seed)
        qp = O.linearise(ocp, rng.standard_normal((ocp.B, ocp.n)))
        D, Off = S.schur_blocks(qp)
        Pd, Po = S.preconditioner_blocks(D, Off)
        for b in range(ocp.B):
            assert np.linalg.eigvalsh(S.dense_block_tridiag(D, Off, b)).min() > 0
            assert np.linalg.eigvalsh(S.dense_block_tridiag(Pd, Po, b)).min() > 0
        Z = np.zeros_like(Off)
        Pd0, Po0 = S.preconditioner_blocks(D, Z)
        gam = S.gamma_spd(qp)
        lam, it, _, _ = S.pcg(D, Z, Pd0, Po0, gam, np.zeros_like(gam), 1e-24, 50)
        assert (it == 1).all()
        exact = np.linalg.solve(D, gam[..., None])[..., 0]
        np.testing.assert_allclose(lam, exact, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("name", ["lq", "cartpole"])
def test_pcg_and_recovery_match_direct_kkt(name):
    """Algorithm 4 (FP64, tight tolerance) + Eq. 11 recover the direct KKT solution."""
    if name == "lq":
        w, ocp = _lq(B=3, T=20, c_var=0.01)
    else:
        w = workloads.cartpole_config(B=3, T=30, seed=4)
        ocp = to_ocp(w)
    rng = np.random.default_rng(1)
    z = 0.3 * rng.standard_normal((ocp.B, ocp.n))
    qp = O.linearise(ocp, z)
    D, Off = S.schur_blocks(qp)
    Pd, Po = S.preconditioner_blocks(D, Off)
    gam = S.gamma_spd(qp)
    lam, it, eta, eta0 = S.pcg(D, Off, Pd, Po, gam, np.zeros_like(gam), 1e-26, 2000)
    assert (eta <= 1e-26 * eta0).all()
    xr, ur = S.recover_primal(qp, lam)
    for b in range(ocp.B):
        zd, ld = O.solve_qp(qp, b)
        np.testing.assert_allclose(lam[b].reshape(-1), ld, rtol=1e-8, atol=1e-9)
        np.testing.assert_allclose(O.join_z(xr[b:b + 1], ur[b:b + 1])[0], zd, rtol=1e-8, atol=1e-9)


def test_pcg_warm_start_from_solution_takes_no_iteration():
    w, ocp = _lq(B=2, T=10)
    qp = O.linearise(ocp, cold_start(ocp)[0])
    D, Off = S.schur_blocks(qp)
    Pd, Po = S.preconditioner_blocks(D, Off)
    gam = S.gamma_spd(qp)
    lam_star = np.linalg.solve(np.stack([S.dense_block_tridiag(D, Off, b) for b in range(2)]),
                               gam.reshape(2, -1, 1))[..., 0].reshape(gam.shape)
    _, it, _, _ = S.pcg(D, Off, Pd, Po, gam, lam_star, 1e-16, 10)
    assert (it == 0).all()


def test_adjoint_symmetry_of_kkt():
    """The KKT matrix of Eq. 5 is symmetric: <K^-1 a, b> = <a, K^-1 b> (used by Eq. 3)."""
    w = workloads.cartpole_config(B=1, T=6, seed=7)
    ocp = to_ocp(w)
    rng = np.random.default_rng(2)
    qp = O.linearise(ocp, 0.5 * rng.standard_normal((1, ocp.n)))
    N = ocp.n + ocp.m
    a, c = rng.standard_normal(N), rng.standard_normal(N)
    za, la = O.solve_qp(qp, 0, rhs=a)
    zc, lc = O.solve_qp(qp, 0, rhs=c)
    lhs = np.dot(np.concatenate([za, la]), c)
    rhs = np.dot(a, np.concatenate([zc, lc]))
    assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(lhs))
