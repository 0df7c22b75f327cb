// Fused SQP / backward kernels instantiated for LQ OCPs of the supported sizes.
#include "launch_impl.cuh"

namespace dmpc {
int register_lq(KernelEntry* out) {
  int n = 0;
  n += register_teams<LQ<2, 1>>(out + n, M_LQ);
  n += register_teams<LQ<3, 2>>(out + n, M_LQ);
  n += register_teams<LQ<4, 1>>(out + n, M_LQ);
  n += register_teams<LQ<8, 4>>(out + n, M_LQ);
  return n;
}
}  // namespace dmpc
