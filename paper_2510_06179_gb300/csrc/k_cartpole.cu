// Fused and plain kernels instantiated for the CartPole model, one team size per compilation
// (the build compiles this file once per DMPC_TEAM in 32, 64, 128, 256).
#include "launch_impl.cuh"

#ifndef DMPC_TEAM
#error "compile with -DDMPC_TEAM=<team size>"
#endif

namespace dmpc {
int DMPC_REGISTER_NAME(cartpole, DMPC_TEAM)(KernelEntry* out) {
  int n = register_team<CartPole, DMPC_TEAM>(out, M_CARTPOLE);
  n += register_team<Trap<CartPole>, DMPC_TEAM>(out + n, M_CARTPOLE_TRAP);
  return n;
}
}  // namespace dmpc
