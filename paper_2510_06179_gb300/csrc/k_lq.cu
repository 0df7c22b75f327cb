// Fused and plain kernels instantiated for LQ OCPs of the supported sizes, one team size per
// compilation (the build compiles this file once per DMPC_TEAM in 32, 64, 128, 256).
#include "launch_impl.cuh"

#ifndef DMPC_TEAM
#error "compile with -DDMPC_TEAM=<team size>"
#endif

namespace dmpc {
int DMPC_REGISTER_NAME(lq, DMPC_TEAM)(KernelEntry* out) {
  int n = 0;
  n += register_team<LQ<2, 1>, DMPC_TEAM>(out + n, M_LQ);
  n += register_team<LQ<3, 2>, DMPC_TEAM>(out + n, M_LQ);
  n += register_team<LQ<4, 1>, DMPC_TEAM>(out + n, M_LQ);
  n += register_team<LQ<8, 4>, DMPC_TEAM>(out + n, M_LQ);
  return n;
}
}  // namespace dmpc
