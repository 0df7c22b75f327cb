// Fused kernel for batches that mix the nonlinear models (team of 64 threads): each team
// dispatches on the model of the OCP it takes from the work list.
#include "launch_impl.cuh"

namespace dmpc {
LaunchFn mixed_launcher_64() {
  return &launch_fused<64, Pendulum, CartPole, KinBicycle, SingleTrack, RigidBody12, Attitude>;
}
}  // namespace dmpc
