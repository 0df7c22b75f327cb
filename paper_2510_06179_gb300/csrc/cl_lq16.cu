// Cluster kernel and 256-thread fused and plain kernels for LQ OCPs with nx = 16, nu = 8 (the RL
// benchmark's problems 5 and 6, App. B.1): their workspace (~7 KB per knot) does not fit one CTA's
// shared memory at T = 30, so each OCP runs on a thread-block cluster whose CTA 0 is a 256-thread
// team.
#define DMPC_CLUSTER_PCG 1
#include "launch_impl.cuh"

namespace dmpc {
int register_cluster_lq16(ClusterEntry* out) { return register_cluster<LQ<16, 8>>(out, M_LQ); }
int register_lq16_team256(KernelEntry* out) { return register_team<LQ<16, 8>, 256>(out, M_LQ); }
}  // namespace dmpc
