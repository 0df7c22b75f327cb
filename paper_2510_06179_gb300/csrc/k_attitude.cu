// Fused SQP / backward kernels instantiated for the Attitude model.
#include "launch_impl.cuh"

namespace dmpc {
int register_attitude(KernelEntry* out) { return register_teams<Attitude>(out, M_ATTITUDE); }
}  // namespace dmpc
