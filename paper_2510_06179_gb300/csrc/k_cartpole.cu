// Fused SQP / backward kernels instantiated for the CartPole model.
#include "launch_impl.cuh"

namespace dmpc {
int register_cartpole(KernelEntry* out) { return register_teams<CartPole>(out, M_CARTPOLE); }
}  // namespace dmpc
