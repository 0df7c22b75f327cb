"""Parity protocol for SQP runs whose line search can branch (the paper's Algorithm 5 on
nonconvex OCPs).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The line search takes the first step size alpha_j (in decreasing order) whose decrease test
Delta phi_j < 0 holds (Eq. 14), else the smallest one.  When a test value lies within the
rounding of the arithmetic of zero, an FP32 run and the FP64 oracle can decide it differently
and continue along different, equally valid paths of the method.  So a run is compared with the
oracle in two parts:

  * path: every step size the run took must be a choice the oracle's own test values allow up
    to a tie tolerance: the tests before the chosen one fail (Delta phi_i >= -tie |phi|), and
    the chosen one passes (Delta phi_j < tie |phi|) unless it is the smallest step, which the
    line search takes regardless of its test;
  * values: the oracle replays that path (oracle.sqp.sqp with alpha_seq), logging its test
    values at every iterate of the path, and the run's solution is gated against the replay.

An OCP whose path is consistent and whose solution is within the gate of the FP64 replay is a
result of the method within the solution tolerance; one whose path is inconsistent took a step
the oracle's tests rule out by more than rounding, which is a failure.
"""
import numpy as np

from .sqp import LS_ALPHAS


def alpha_index(alpha, alphas=LS_ALPHAS):
    """Index of each taken step size in the candidate set (compared in float32)."""
    a = np.asarray(alpha, np.float32)
    cand = np.asarray(alphas, np.float32)
    idx = np.argmin(np.abs(a[..., None] - cand), axis=-1)
    if not np.all(cand[idx] == a):
        raise ValueError("a step size outside the candidate set")
    return idx


def step_consistent(j, delta, phi0, tie, n_alpha):
    """Whether taking candidate j agrees with the test values delta (one per candidate) of the
    iterate whose merit is phi0, up to tie * |phi0|."""
    t = tie * max(abs(phi0), 1e-300)
    if np.any(delta[:j] < -t):
        return False
    return j == n_alpha - 1 or delta[j] < t


def path_consistency(alpha, replay, tie=1e-5, alphas=LS_ALPHAS):
    """Per OCP: whether every step of the path `alpha` (B, iters) agrees with the test values
    the oracle logged while replaying it (replay = oracle.sqp.sqp(..., alpha_seq=alpha)), and
    the first iteration that does not (-1 if none)."""
    idx = alpha_index(alpha, alphas)
    B, iters = idx.shape
    ok = np.ones(B, bool)
    first_bad = np.full(B, -1)
    for b in range(B):
        for k in range(iters):
            if not step_consistent(idx[b, k], replay["delta"][b, k], replay["phi0"][b, k], tie, len(alphas)):
                ok[b] = False
                first_bad[b] = k
                break
    return ok, first_bad
