// Fused SQP / backward kernels instantiated for the KinBicycle model.
#include "launch_impl.cuh"

namespace dmpc {
int register_bicycle(KernelEntry* out) { return register_teams<KinBicycle>(out, M_KIN_BICYCLE); }
}  // namespace dmpc
