// Fused and plain kernels instantiated for the KinBicycle model, one team size per compilation
// (the build compiles this file once per DMPC_TEAM in 32, 64, 128, 256).
#include "launch_impl.cuh"

#ifndef DMPC_TEAM
#error "compile with -DDMPC_TEAM=<team size>"
#endif

namespace dmpc {
int DMPC_REGISTER_NAME(bicycle, DMPC_TEAM)(KernelEntry* out) { return register_team<KinBicycle, DMPC_TEAM>(out, M_KIN_BICYCLE); }
}  // namespace dmpc
