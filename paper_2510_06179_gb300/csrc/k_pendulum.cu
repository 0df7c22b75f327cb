// Fused SQP / backward kernels instantiated for the Pendulum model.
#include "launch_impl.cuh"

namespace dmpc {
int register_pendulum(KernelEntry* out) { return register_teams<Pendulum>(out, M_PENDULUM); }
}  // namespace dmpc
