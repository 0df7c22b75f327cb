// Fused and plain kernels instantiated for the SingleTrack model, one team size per compilation
// (the build compiles this file once per DMPC_TEAM in 32, 64, 128, 256).
#include "launch_impl.cuh"

#ifndef DMPC_TEAM
#error "compile with -DDMPC_TEAM=<team size>"
#endif

namespace dmpc {
int DMPC_REGISTER_NAME(single_track, DMPC_TEAM)(KernelEntry* out) { return register_team<SingleTrack, DMPC_TEAM>(out, M_SINGLE_TRACK); }
}  // namespace dmpc
