// Collects the kernel entries of every per-team kernel translation unit, and keeps the
// per-device dynamic shared-memory limits of the kernels.
#include <map>
#include <mutex>
#include <utility>

#include "launch.h"

namespace dmpc {
cudaError_t raise_smem_limit(const void* kernel, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> configured;  // (kernel, device) -> bytes
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = configured[{kernel, dev}];
  if (smem <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) cur = smem;
  return e;
}

int collect_kernel_entries(KernelEntry* out) {
  int n = 0;
#define DMPC_COLLECT(model)                          \
  n += DMPC_REGISTER_NAME(model, 32)(out + n);       \
  n += DMPC_REGISTER_NAME(model, 64)(out + n);       \
  n += DMPC_REGISTER_NAME(model, 128)(out + n);      \
  n += DMPC_REGISTER_NAME(model, 256)(out + n);
  DMPC_COLLECT(lq)
  DMPC_COLLECT(lq16)
  DMPC_COLLECT(pendulum)
  DMPC_COLLECT(cartpole)
  DMPC_COLLECT(bicycle)
  DMPC_COLLECT(single_track)
  DMPC_COLLECT(single_track_rate)
  DMPC_COLLECT(rigid_body)
  DMPC_COLLECT(attitude)
  DMPC_COLLECT(mixed)
#undef DMPC_COLLECT
  n += register_lq16_team256(out + n);
  return n;
}

int collect_cluster_entries(ClusterEntry* out) {
  int n = 0;
  n += register_cluster_rigid_body(out + n);
  n += register_cluster_lq16(out + n);
  return n;
}
}  // namespace dmpc
