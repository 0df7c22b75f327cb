// Collects the kernel entries of every per-team kernel translation unit.
#include "launch.h"

namespace dmpc {
int collect_kernel_entries(KernelEntry* out) {
  int n = 0;
#define DMPC_COLLECT(model)                          \
  n += DMPC_REGISTER_NAME(model, 32)(out + n);       \
  n += DMPC_REGISTER_NAME(model, 64)(out + n);       \
  n += DMPC_REGISTER_NAME(model, 128)(out + n);      \
  n += DMPC_REGISTER_NAME(model, 256)(out + n);
  DMPC_COLLECT(lq)
  DMPC_COLLECT(pendulum)
  DMPC_COLLECT(cartpole)
  DMPC_COLLECT(bicycle)
  DMPC_COLLECT(single_track)
  DMPC_COLLECT(rigid_body)
  DMPC_COLLECT(attitude)
  DMPC_COLLECT(mixed)
#undef DMPC_COLLECT
  return n;
}
}  // namespace dmpc
