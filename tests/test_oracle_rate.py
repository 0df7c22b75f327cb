"""Pins of the oracle's control-rate augmentation (App. B.3: state (x, u), input u_dot) against
the base model it wraps, the cost it is meant to express, and the KKT and gradient machinery."""
import numpy as np
import pytest

from paper_2510_06179_gb300 import workloads
from oracle import ocp as O
from oracle.backward import vjp
from oracle.fd import fd_gradient
from oracle.models import make_model
from oracle.sqp import sqp, newton_kkt
from tests.oracle_helpers import to_ocp


def _base_rollout(T=12, seed=0):
    """A trajectory of the base vehicle under smooth inputs, and the matching augmented one."""
    rng = np.random.default_rng(seed)
    base = make_model("single_track", dt=0.02)
    aug = make_model("single_track_rate", dt=0.02)
    ths = [0.8, 9e4]
    x = [np.array([0.0, 0.0, 0.05, 0.1, 0.2, 12.0])]
    u = np.stack([0.02 * np.sin(0.3 * np.arange(T + 1) + rng.uniform()), 300.0 * np.cos(0.2 * np.arange(T + 1))], 1)
    for t in range(T):
        x.append(np.array(base.step(list(x[t]), list(u[t]), ths, [])))
    return base, aug, ths, np.array(x), u


def test_augmented_step_reproduces_the_base_trajectory():
    """With v_t = (u_{t+1} - u_t) / dt the augmented model carries (x_t, u_t) exactly along the
    base model's trajectory."""
    base, aug, ths, x, u = _base_rollout()
    xa = np.concatenate([x[0], u[0]])
    for t in range(len(x) - 1):
        v = (u[t + 1] - u[t]) / aug.dt
        xa = np.array(aug.step(list(xa), list(v), ths, []))
        np.testing.assert_allclose(xa[:6], x[t + 1], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(xa[6:], u[t + 1], rtol=1e-12, atol=1e-9)


def test_input_cost_is_the_control_rate_cost():
    """On the augmented OCP the input cost 1/2 v^T diag(R) v equals the rate penalty
    1/2 sum_t ((u_{t+1} - u_t)/dt)^T diag(R) ((u_{t+1} - u_t)/dt) of the base inputs."""
    base, aug, ths, x, u = _base_rollout(T=10)
    T = 10
    q = np.array([1.0, 2.0, 3.0, 0.5, 0.25, 0.1, 0.7, 1e-3])
    r = np.array([0.3, 1e-6])
    w = workloads.vehicle_rate_config(B=1, T=T, seed=0)
    lay = workloads.theta_layout("single_track_rate", 8, 2, T)
    th = np.zeros((1, lay["size"]))
    th[0, :2] = ths
    th[0, lay["q"]:lay["r"]] = q
    th[0, lay["r"]:lay["qt"]] = r
    th[0, lay["qt"]:] = 10 * q
    xa = np.concatenate([x, u[:T + 1]], 1)                # (T+1, 8)
    v = (u[1:T + 1] - u[:T]) / aug.dt                      # (T, 2)
    ocp = O.OCPBatch(aug, T, xa[:1, :], th, np.zeros((1, T + 1, 8)))
    z = O.join_z(xa[None], v[None])
    rate_cost = 0.5 * np.sum(r * v * v)
    state_cost = 0.5 * np.sum(q * xa[:T] ** 2) + 0.5 * np.sum(10 * q * xa[T] ** 2)
    np.testing.assert_allclose(O.cost_value(ocp, z)[0], rate_cost + state_cost, rtol=1e-12)
    assert w.nx == 8 and w.nu == 2


def test_augmented_linearisation_has_the_block_structure():
    """Eq. 4 for the augmented model: A = [[A_b, B_b], [0, -I]], B = [0; -dt I] against the base
    model's own linearisation at the same point."""
    base, aug, ths, x, u = _base_rollout(T=6)
    T = 6
    wb = workloads.vehicle_config(B=1, T=T, seed=0)
    wa = workloads.vehicle_rate_config(B=1, T=T, seed=0)
    ob = to_ocp(wb)
    oa = to_ocp(wa)
    rng = np.random.default_rng(3)
    v = rng.standard_normal((T, 2)) * np.array([0.1, 100.0])
    za = O.join_z(np.concatenate([x, u[:T + 1]], 1)[None], v[None])
    zb = O.join_z(x[None], u[:T][None])
    qa = O.linearise(oa, za)
    qb = O.linearise(ob, zb)
    np.testing.assert_allclose(qa.A[0][:, :6, :6], qb.A[0], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(qa.A[0][:, :6, 6:], qb.Bm[0], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(qa.A[0][:, 6:, :6], 0.0)
    np.testing.assert_allclose(qa.A[0][:, 6:, 6:], np.broadcast_to(-np.eye(2), (T, 2, 2)))
    np.testing.assert_allclose(qa.Bm[0][:, :6], 0.0)
    np.testing.assert_allclose(qa.Bm[0][:, 6:], np.broadcast_to(-0.02 * np.eye(2), (T, 2, 2)))


def test_augmented_vehicle_exact_hessian_vjp_matches_fd():
    """At a Newton-polished KKT point of an augmented vehicle OCP the exact-Hessian IFT gradient
    equals central differences (steps relative to each entry, Newton-KKT re-solves)."""
    w = workloads.vehicle_rate_config(B=1, T=15, seed=2)
    ocp = to_ocp(w)
    out = sqp(ocp, 60)
    z, lam, _, _ = newton_kkt(ocp, out["z"], out["lam"])
    Fz, Fl = O.kkt_residual(ocp, z, lam)
    assert max(np.abs(Fz).max(), np.abs(Fl).max()) <= 1e-9
    rng = np.random.default_rng(5)
    wz = rng.standard_normal(ocp.n)

    def loss(zz):
        return 0.5 * np.sum(wz * zz * zz)
    g = wz * z[0]
    ex = vjp(ocp, z, lam, g[None], hessian="exact")
    fd = fd_gradient(ocp, loss, z, lam, rel_step=1e-5, step="relative", solver="newton")
    scale = np.maximum(np.abs(fd), 1e-3 * np.abs(fd).max())
    assert (np.abs(ex["dtheta"][0] - fd) / scale).max() <= 1e-5
