// Launch helper shared by the kernel translation units.
#pragma once
#include "fused.cuh"
#include "launch.h"

namespace dmpc {

template <int TEAM, class... Ms>
cudaError_t launch_fused(const KParams& P, int grid, int threads, size_t smem, cudaStream_t s) {
  static size_t configured = 0;  // largest dynamic smem size set so far for this kernel
  auto fn = fused_kernel<TEAM, Ms...>;
  if (smem > 48 * 1024 && smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  fn<<<grid, threads, smem, s>>>(P);
  return cudaGetLastError();
}

template <class M>
int register_teams(KernelEntry* out, int model_id) {
  out[0] = {model_id, M::NX, M::NU, 32, &launch_fused<32, M>};
  out[1] = {model_id, M::NX, M::NU, 64, &launch_fused<64, M>};
  out[2] = {model_id, M::NX, M::NU, 128, &launch_fused<128, M>};
  out[3] = {model_id, M::NX, M::NU, 256, &launch_fused<256, M>};
  return 4;
}

}  // namespace dmpc
