// Kernel registry of the fused SQP/backward kernels: one entry per (model set, team size).
#pragma once
#include <cuda_runtime.h>
#include "params.h"

namespace dmpc {

typedef cudaError_t (*LaunchFn)(const KParams& P, int grid, int threads, size_t smem, cudaStream_t s);

struct PlainState;
// plain one-launch-per-step form: one launch = one step for the batch (grid = batch, block = team);
// P is a device pointer
typedef cudaError_t (*PlainFn)(const KParams* P, PlainState* st, int step, int s_iter, int grid, int threads,
                               cudaStream_t s);

struct KernelEntry {
  int model;   // model id, or -1 for the mixed kernel (all nonlinear models)
  int nx, nu;
  int team;
  LaunchFn fn;
  PlainFn plain;
};

// Each kernel translation unit is compiled once per team size and appends its entries;
// the functions return the number of entries written.
#define DMPC_REGISTER_NAME2(model, team) register_##model##_##team
#define DMPC_REGISTER_NAME(model, team) DMPC_REGISTER_NAME2(model, team)
#define DMPC_DECLARE_TEAMS(model)                 \
  int DMPC_REGISTER_NAME(model, 32)(KernelEntry*);  \
  int DMPC_REGISTER_NAME(model, 64)(KernelEntry*);  \
  int DMPC_REGISTER_NAME(model, 128)(KernelEntry*); \
  int DMPC_REGISTER_NAME(model, 256)(KernelEntry*);
DMPC_DECLARE_TEAMS(lq)
DMPC_DECLARE_TEAMS(lq16)
DMPC_DECLARE_TEAMS(pendulum)
DMPC_DECLARE_TEAMS(cartpole)
DMPC_DECLARE_TEAMS(bicycle)
DMPC_DECLARE_TEAMS(single_track)
DMPC_DECLARE_TEAMS(single_track_rate)
DMPC_DECLARE_TEAMS(rigid_body)
DMPC_DECLARE_TEAMS(attitude)
DMPC_DECLARE_TEAMS(mixed)

// Cluster kernel of one model (distributed PCG): launch with `ncta` CTAs per cluster and
// `grid` CTAs in total; `max_clusters` returns how many such clusters fit on the device at once.
typedef cudaError_t (*ClusterLaunchFn)(const KParams& P, int grid, int ncta, size_t smem, cudaStream_t s);
typedef int (*ClusterOccFn)(int ncta, size_t smem);
struct ClusterEntry {
  int model, nx, nu;
  ClusterLaunchFn fn;
  ClusterOccFn max_clusters;
};
int register_cluster_rigid_body(ClusterEntry*);
int register_cluster_lq16(ClusterEntry*);
int register_lq16_team256(KernelEntry*);   // the 256-thread LQ nx 16 kernels live in the cluster unit
constexpr int kMaxClusterEntries = 8;
int collect_cluster_entries(ClusterEntry* out);

// Raise a kernel's dynamic shared-memory limit to at least `smem` bytes on the current device.
// The attribute is per device, so the largest size set so far is kept per (kernel, device);
// a mutex makes concurrent callers (different host threads or devices) safe.
cudaError_t raise_smem_limit(const void* kernel, size_t smem);

// Fill `out` with every compiled kernel entry; returns the count (at most kMaxKernelEntries).
constexpr int kMaxKernelEntries = 160;
int collect_kernel_entries(KernelEntry* out);

}  // namespace dmpc
