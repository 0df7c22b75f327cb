// Fused and plain kernels for LQ OCPs with nx = 16, nu = 8 (the RL benchmark's problems 5 and 6,
// App. B.1) on 32-thread teams; the 256-thread ones are compiled with the cluster kernel
// (cl_lq16.cu), and the other team sizes register nothing (an instantiation of this size takes
// about two minutes of nvcc).
#include "launch_impl.cuh"

#ifndef DMPC_TEAM
#error "compile with -DDMPC_TEAM=<team size>"
#endif

namespace dmpc {
int DMPC_REGISTER_NAME(lq16, DMPC_TEAM)(KernelEntry* out) {
#if DMPC_TEAM == 32
  return register_team<LQ<16, 8>, 32>(out, M_LQ);
#else
  (void)out;
  return 0;
#endif
}
}  // namespace dmpc
