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

#ifdef DMPC_CLUSTER_PCG
template <class M>
cudaError_t launch_fused_cluster(const KParams& P, int grid, int ncta, size_t smem, cudaStream_t s) {
  auto fn = fused_cluster_kernel<M>;
  if (smem > 48 * 1024) {
    cudaError_t e = raise_smem_limit(reinterpret_cast<const void*>(fn), smem);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(kClThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = ncta;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fn, P);
}

template <class M>
int cluster_occupancy(int ncta, size_t smem) {
  auto fn = fused_cluster_kernel<M>;
  if (smem > 48 * 1024 && raise_smem_limit(reinterpret_cast<const void*>(fn), smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ncta * 64, 1, 1);
  cfg.blockDim = dim3(kClThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = ncta;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <class M>
int register_cluster(ClusterEntry* out, int model_id) {
  out[0] = {model_id, M::NX, M::NU, &launch_fused_cluster<M>, &cluster_occupancy<M>};
  return 1;
}
#endif

}  // namespace dmpc
