// Launch helper shared by the kernel translation units.
#pragma once
#include "fused.cuh"
#include "plain.cuh"
#include "launch.h"

namespace dmpc {

template <int TEAM, class... Ms>
cudaError_t launch_fused(const KParams& P, int grid, int threads, size_t smem, cudaStream_t s) {
  auto fn = fused_kernel<TEAM, Ms...>;
  if (smem > 48 * 1024) {
    cudaError_t e = raise_smem_limit(reinterpret_cast<const void*>(fn), smem);
    if (e != cudaSuccess) return e;
  }
  fn<<<grid, threads, smem, s>>>(P);
  return cudaGetLastError();
}

template <int TEAM, class... Ms>
cudaError_t launch_plain(const KParams* P, PlainState* st, int step, int s_iter, int grid, int threads, cudaStream_t s) {
  plain_kernel<TEAM, Ms...><<<grid, threads, 0, s>>>(P, st, step, s_iter);
  return cudaGetLastError();
}

template <class M, int TEAM>
int register_team(KernelEntry* out, int model_id) {
  out[0] = {model_id, M::NX, M::NU, TEAM, &launch_fused<TEAM, M>, &launch_plain<TEAM, M>};
  return 1;
}

}  // namespace dmpc
