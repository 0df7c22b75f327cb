// Cluster kernel for the RigidBody12 model: each OCP runs on a cluster of CTAs whose shared
// memory holds its S and Phi^-1 blocks during the PCG solves (the workspace of a 12-state OCP
// with more than a few dozen knots does not fit in one CTA).
#define DMPC_CLUSTER_PCG 1
#include "launch_impl.cuh"

namespace dmpc {
int register_cluster_rigid_body(ClusterEntry* out) { return register_cluster<RigidBody12>(out, M_RIGID_BODY12); }
}  // namespace dmpc
