"""Pins of the oracle's stage costs (Sec. 3.1 OCP statement): c_t^x(x) = 1/2 (x - x_ref,t)^T
diag(Q) (x - x_ref,t) with diag(Q_T) at t = T and c_t^u(u) = 1/2 u^T diag(R) u, checked on a
hand-computed one-step example, and their gradient against central differences of the value
on OCPs that track a nonzero reference."""
import numpy as np

from paper_2510_06179_gb300 import workloads
from oracle import ocp as O
from oracle.models import make_model
from tests.oracle_helpers import to_ocp


def _one_step_pendulum():
    # theta = (m, L | diag Q | diag R | diag Q_T)
    theta = np.array([[1.0, 0.7, 2.0, 3.0, 5.0, 7.0, 11.0]])
    x_ref = np.array([[[1.0, -1.0], [0.5, 2.0]]])
    ocp = O.OCPBatch(make_model("pendulum", dt=0.05), 1, np.zeros((1, 2)), theta, x_ref)
    x = np.array([[[2.0, 1.0], [-1.0, 4.0]]])
    u = np.array([[[0.3]]])
    return ocp, O.join_z(x, u)


def test_cost_value_hand_computed():
    """1/2 (2*1^2 + 3*2^2) + 1/2 * 5 * 0.3^2 + 1/2 (7*1.5^2 + 11*2^2) = 7 + 0.225 + 29.875."""
    ocp, z = _one_step_pendulum()
    assert O.theta_size(ocp.model, ocp.T) == ocp.theta.shape[1]
    np.testing.assert_allclose(O.cost_value(ocp, z), [37.1], rtol=1e-14)


def test_cost_gradient_hand_computed():
    """(Q (x_0 - x_ref,0), R u_0, Q_T (x_1 - x_ref,1)) in the knot-interleaved z layout."""
    ocp, z = _one_step_pendulum()
    np.testing.assert_allclose(O.cost_gradient(ocp, z), [[2.0, 6.0, 1.5, -10.5, 22.0]], rtol=1e-14)


def test_cost_gradient_matches_differences_with_reference():
    w = workloads.bicycle_config(B=2, T=6, seed=5)
    ocp = to_ocp(w)
    assert np.abs(ocp.x_ref).max() > 1.0
    rng = np.random.default_rng(3)
    z = rng.standard_normal((ocp.B, ocp.n)) + np.concatenate(
        [np.concatenate([ocp.x_ref[:, t], np.zeros((ocp.B, ocp.nu))], 1) for t in range(ocp.T)]
        + [ocp.x_ref[:, ocp.T]], 1)
    g = O.cost_gradient(ocp, z)
    fd = np.zeros_like(z)
    for i in range(ocp.n):
        h = 1e-6 * max(1.0, np.abs(z[:, i]).max())
        zp, zm = z.copy(), z.copy()
        zp[:, i] += h
        zm[:, i] -= h
        fd[:, i] = (O.cost_value(ocp, zp) - O.cost_value(ocp, zm)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-6 * np.abs(fd).max())


def test_pd_projection_reading():
    """Reading of the PD projection (Sec. 3.1): each diagonal entry is clamped below at
    1e-6 max(1, largest entry); positive entries above the floor are left alone."""
    d = np.array([[-1.0, 0.0, 2e-7, 5.0], [0.5, -2.0, 0.25, 1e-3]])
    out = O.pd_project_diag(d)
    np.testing.assert_allclose(out[0], [5e-6, 5e-6, 5e-6, 5.0], rtol=1e-14)
    np.testing.assert_allclose(out[1], [0.5, 1e-6, 0.25, 1e-3], rtol=1e-14)
