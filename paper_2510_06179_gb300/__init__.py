"""DiffMPC hot path on GB300: batched SQP solves of optimal control problems and their
implicit-function gradients (arXiv 2510.06179), as CUDA kernels behind the C-ABI declared in
include/dmpc.h.

Modules (imported on demand, so importing the package needs no GPU):
  solver     OCPBatch (create / solve / vjp / inspect / tiling / set_solution on one C-ABI handle),
             DiffMPCFunction and diffmpc (torch.autograd entry points)
  _lib       ctypes binding of libdmpc.so (argument marshalling only; fails loudly when missing)
  build      compiles the library for sm_103a
  workloads  seeded synthetic inputs (LQ, pendulum, cart-pole, bicycle, vehicle, rigid body,
             attitude, uneven mixes, serving traces, RL problems)
  autotune   tiling search and CUDA-graph replay of a solve + vjp step
  serving    continuous-batching request loop over slot arenas
  rollout    closed-loop MPC rollouts with gradients through every solve
  cost_mlp   learned cost weights for the vehicle OCPs
"""
