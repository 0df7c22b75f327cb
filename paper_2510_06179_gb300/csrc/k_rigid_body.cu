// Fused SQP / backward kernels instantiated for the RigidBody12 model.
#include "launch_impl.cuh"

namespace dmpc {
int register_rigid_body(KernelEntry* out) { return register_teams<RigidBody12>(out, M_RIGID_BODY12); }
}  // namespace dmpc
