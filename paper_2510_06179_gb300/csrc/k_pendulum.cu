// Fused and plain kernels instantiated for the Pendulum model, one team size per compilation
// (the build compiles this file once per DMPC_TEAM in 32, 64, 128, 256).
#include "launch_impl.cuh"

#ifndef DMPC_TEAM
#error "compile with -DDMPC_TEAM=<team size>"
#endif

namespace dmpc {
int DMPC_REGISTER_NAME(pendulum, DMPC_TEAM)(KernelEntry* out) {
  int n = register_team<Pendulum, DMPC_TEAM>(out, M_PENDULUM);
  n += register_team<Trap<Pendulum>, DMPC_TEAM>(out + n, M_PENDULUM_TRAP);
  return n;
}
}  // namespace dmpc
