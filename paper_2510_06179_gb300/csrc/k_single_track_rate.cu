// Fused and plain kernels instantiated for the SingleTrack model with control-rate augmentation
// (state (x, u), input u_dot), one team size per compilation (the build compiles this file once
// per DMPC_TEAM in 32, 64, 128, 256).
#include "launch_impl.cuh"

#ifndef DMPC_TEAM
#error "compile with -DDMPC_TEAM=<team size>"
#endif

namespace dmpc {
int DMPC_REGISTER_NAME(single_track_rate, DMPC_TEAM)(KernelEntry* out) {
  return register_team<Rate<SingleTrack, M_SINGLE_TRACK_RATE>, DMPC_TEAM>(out, M_SINGLE_TRACK_RATE);
}
}  // namespace dmpc
