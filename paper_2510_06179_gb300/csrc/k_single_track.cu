// Fused SQP / backward kernels instantiated for the SingleTrack model.
#include "launch_impl.cuh"

namespace dmpc {
int register_single_track(KernelEntry* out) { return register_teams<SingleTrack>(out, M_SINGLE_TRACK); }
}  // namespace dmpc
