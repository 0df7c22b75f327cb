// Kernel registry of the fused SQP/backward kernels: one entry per (model set, team size).
#pragma once
#include <cuda_runtime.h>
#include "params.h"

namespace dmpc {

typedef cudaError_t (*LaunchFn)(const KParams& P, int grid, int threads, size_t smem, cudaStream_t s);

struct KernelEntry {
  int model;   // model id, or -1 for the mixed kernel (all nonlinear models)
  int nx, nu;
  int team;
  LaunchFn fn;
};

// each translation unit appends its entries; returns the number written
int register_lq(KernelEntry* out);
int register_pendulum(KernelEntry* out);
int register_cartpole(KernelEntry* out);
int register_bicycle(KernelEntry* out);
int register_single_track(KernelEntry* out);
int register_rigid_body(KernelEntry* out);
int register_attitude(KernelEntry* out);
int register_mixed(KernelEntry* out);

}  // namespace dmpc
