// Registry entries of the mixed-model kernels (instantiated in k_mixed_<team>.cu).
#include "launch.h"

namespace dmpc {
LaunchFn mixed_launcher_32();
LaunchFn mixed_launcher_64();
LaunchFn mixed_launcher_128();
LaunchFn mixed_launcher_256();
int register_mixed(KernelEntry* out) {
  out[0] = {-1, 0, 0, 32, mixed_launcher_32()};
  out[1] = {-1, 0, 0, 64, mixed_launcher_64()};
  out[2] = {-1, 0, 0, 128, mixed_launcher_128()};
  out[3] = {-1, 0, 0, 256, mixed_launcher_256()};
  return 4;
}
}  // namespace dmpc
