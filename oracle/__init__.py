"""FP64 CPU oracle for one SQP iteration + backward of DiffMPC (arXiv 2510.06179).

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and the CPU-baseline /
reference legs of bench.py may import this package.  It shares no code with the CUDA
path (paper_2510_06179_gb300/), and the product path never calls it.

What it computes, and where in the paper each part comes from:
  models.py    dynamics f_t (OCP statement, Sec. 3; cart-pole App. B.2; LQ App. B.1;
               attitude App. B.1; vehicle App. B.3 as re-specified for the workloads)
  jet.py       second-order forward-mode derivatives (for Eq. 4 and dF/dtheta in Eq. 3)
  ocp.py       QP matrices (Eq. 4), KKT system (Eq. 5-6) solved directly (banded LU,
               dense LU for small T), KKT residual F (Eq. 1)
  schur.py     S, gamma, Phi^-1 (Eq. 8-10, App. A.2), PCG (Algorithm 4), recovery (Eq. 11)
  sqp.py       SQP (Algorithm 2) with the line search (Algorithm 5, Eq. 12-15)
  backward.py  VJP (Eq. 3, Eq. 7, Algorithm 3), Gauss-Newton and exact-Hessian variants
  riccati.py   textbook finite-horizon Riccati recursion (independent LQ closed form)
  fd.py        central finite differences of the loss

Pins (tests/test_oracle_*.py) tie these to things other than the oracle itself: the
Riccati closed form, brute-force dense LU, dense H G^-1 H^T, complex-step and finite
differences of the dynamics, the textbook linearisation of the cart-pole, finite
differences of the loss, and the KKT conditions (Eq. 1).
"""
