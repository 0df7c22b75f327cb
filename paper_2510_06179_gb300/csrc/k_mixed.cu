// Fused and plain kernels for batches that mix the nonlinear models: each team dispatches on
// the model of the OCP it takes from the work list.  One team size per compilation.
#include "launch_impl.cuh"

#ifndef DMPC_TEAM
#error "compile with -DDMPC_TEAM=<team size>"
#endif

namespace dmpc {
int DMPC_REGISTER_NAME(mixed, DMPC_TEAM)(KernelEntry* out) {
  out[0] = {-1, 0, 0, DMPC_TEAM,
            &launch_fused<DMPC_TEAM, Pendulum, CartPole, KinBicycle, SingleTrack, RigidBody12, Attitude>,
            &launch_plain<DMPC_TEAM, Pendulum, CartPole, KinBicycle, SingleTrack, RigidBody12, Attitude>};
  return 1;
}
}  // namespace dmpc
