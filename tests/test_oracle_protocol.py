"""Pins of the parity protocol for branching line searches (oracle/protocol.py): the replay of
a path reproduces the run it came from, the consistency test accepts exactly the choices
Algorithm 5 allows, and a step the oracle's tests rule out is caught."""
import numpy as np

from paper_2510_06179_gb300 import workloads
from oracle.protocol import alpha_index, path_consistency, step_consistent
from oracle.sqp import sqp, LS_ALPHAS
from tests.oracle_helpers import to_ocp


def test_step_consistency_follows_algorithm_5():
    phi = 100.0
    n = len(LS_ALPHAS)
    # first passing test (negative) is the choice; earlier tests fail (positive)
    d = np.array([3.0, 1.0, -2.0, -5.0, -9.0])
    assert step_consistent(2, d, phi, 0.0, n)
    assert not step_consistent(1, d, phi, 0.0, n)      # its test failed clearly
    assert not step_consistent(3, d, phi, 0.0, n)      # an earlier test passed clearly
    # no test passes: the smallest step is taken whatever its own test says
    d = np.array([3.0, 2.0, 1.0, 0.5, 0.2])
    assert step_consistent(n - 1, d, phi, 0.0, n)
    assert not step_consistent(2, d, phi, 0.0, n)
    # a test within tie * |phi| of zero may go either way
    d = np.array([3.0, 1e-5, -2.0, -5.0, -9.0])        # alpha_1 fails by 1e-7 |phi|
    assert step_consistent(1, d, phi, 1e-6, n) and step_consistent(2, d, phi, 1e-6, n)
    assert not step_consistent(1, d, phi, 1e-8, n)


def test_alpha_index_rejects_unknown_step():
    assert alpha_index(np.array([[1.0, 0.3, 0.01]])).tolist() == [[0, 2, 4]]
    try:
        alpha_index(np.array([0.5]))
    except ValueError:
        return
    raise AssertionError("step size outside the set accepted")


def test_replaying_a_path_reproduces_the_run_and_is_consistent():
    w = workloads.cartpole_config(B=12, T=30, seed=4, sqp_iters=8)
    ocp = to_ocp(w)
    run = sqp(ocp, 8)
    rep = sqp(ocp, 8, alpha_seq=run["alpha"])
    assert np.array_equal(rep["z"], run["z"]) and np.array_equal(rep["lam"], run["lam"])
    assert np.array_equal(rep["alpha_own"], run["alpha"])
    ok, first = path_consistency(run["alpha"], rep, tie=0.0)
    assert ok.all() and (first == -1).all()


def test_a_step_the_tests_rule_out_is_flagged():
    """Planted: one OCP takes the full step at an iteration where the oracle's test for it fails
    by far more than the tie, and the smallest step elsewhere where a larger one passed."""
    w = workloads.cartpole_config(B=12, T=30, seed=4, sqp_iters=8)
    ocp = to_ocp(w)
    run = sqp(ocp, 8)
    rel = run["delta"] / np.abs(run["phi0"])[..., None]
    # an (OCP, iteration) whose full-step test fails clearly
    cand = np.argwhere(rel[:, :, 0] > 1e-3)
    assert len(cand) > 0
    b, k = cand[0]
    path = run["alpha"].copy()
    path[b, k] = 1.0
    rep = sqp(ocp, 8, alpha_seq=path)
    ok, first = path_consistency(path, rep, tie=1e-5)
    assert not ok[b] and first[b] == k
    assert ok[np.arange(12) != b].all()
    # an (OCP, iteration) whose chosen step passed clearly: forcing the smallest step is ruled out
    idx = alpha_index(run["alpha"])
    cand = [(bb, kk) for bb, kk in np.argwhere(idx < 4) if rel[bb, kk, idx[bb, kk]] < -1e-3]
    assert cand
    b2, k2 = cand[0]
    path = run["alpha"].copy()
    path[b2, k2] = 0.01
    rep = sqp(ocp, 8, alpha_seq=path)
    ok, first = path_consistency(path, rep, tie=1e-5)
    assert not ok[b2] and first[b2] == k2
