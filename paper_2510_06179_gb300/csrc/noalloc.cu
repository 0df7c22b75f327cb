// Allocation-free forward solve (dmpc_solve_noalloc, declared in include/dmpc.h).
//
// Some callers cannot allocate device memory at the point where they need a solve: a
// controller running in a hard real-time loop that may only use memory reserved at start-up,
// a plug-in hosted by a framework whose allocator owns the whole device, or a process that
// has reached its memory limit.  The regular path (dmpc_create_problem_batch) allocates a
// handle's tables, resident state and, for very long horizons, a global workspace; this entry
// point allocates nothing.  Its scratch (the per-OCP record table, the work list and, when an
// OCP's workspace exceeds shared memory, the per-team workspace) lives in one file-scope
// device array of fixed size that every GPU loading the library holds until exit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/dmpc.h"
#include "fused.cuh"
#include "launch.h"

using namespace dmpc;

namespace {

constexpr size_t kScratchBytes = 4u << 20;  // DMPC_NOALLOC_SCRATCH_BYTES in include/dmpc.h
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Host view of the scratch array on the current device, looked up once per device.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// Fill the record table and the work list of a uniform batch (every OCP of one shape).
__global__ void noalloc_tables(OcpRec* recs, int* order, int batch, OcpRec proto) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < batch; b += gridDim.x * blockDim.x) {
    OcpRec r = proto;
    r.z_off = (long long)b * proto.n;
    r.lam_off = (long long)b * proto.m;
    r.th_off = (long long)b * proto.p;
    r.xs_off = (long long)b * proto.nx;
    r.xref_off = (long long)b * (proto.T + 1) * proto.nx;
    r.gws_off = 0;
    recs[b] = r;
    order[b] = b;
  }
}

bool shape_ok(const dmpc_ocp_desc& d, int* p_shared) {
  int nx = -1, nu = -1, ps = 0;
  switch (d.model) {
    case DMPC_MODEL_LQ:
      if (!((d.nx == 2 && d.nu == 1) || (d.nx == 3 && d.nu == 2) || (d.nx == 4 && d.nu == 1) || (d.nx == 8 && d.nu == 4) ||
            (d.nx == 16 && d.nu == 8)))
        return false;
      nx = d.nx; nu = d.nu; ps = 0;
      break;
    case DMPC_MODEL_PENDULUM: nx = 2; nu = 1; ps = 2; break;
    case DMPC_MODEL_CARTPOLE: nx = 4; nu = 1; ps = 2; break;
    case DMPC_MODEL_KIN_BICYCLE: nx = 4; nu = 2; ps = 1; break;
    case DMPC_MODEL_SINGLE_TRACK: nx = 6; nu = 2; ps = 2; break;
    case DMPC_MODEL_RIGID_BODY12: nx = 12; nu = 4; ps = 4; break;
    case DMPC_MODEL_ATTITUDE: nx = 3; nu = 3; ps = 3; break;
    case DMPC_MODEL_SINGLE_TRACK_RATE: nx = 8; nu = 2; ps = 2; break;
    default: return false;
  }
  *p_shared = ps;
  const bool integ_ok = d.integrator == DMPC_INTEGRATOR_DEFAULT ||
                        (d.integrator == DMPC_INTEGRATOR_TRAPEZOID &&
                         (d.model == DMPC_MODEL_PENDULUM || d.model == DMPC_MODEL_CARTPOLE));
  return d.nx == nx && d.nu == nu && d.T >= 1 && d.T <= 4096 && integ_ok &&
         (d.model == DMPC_MODEL_LQ || (d.dt > 0.f && std::isfinite(d.dt)));
}

}  // namespace

extern "C" dmpc_err dmpc_solve_noalloc(const dmpc_ocp_desc* desc, int batch, const dmpc_options* opt,
                                       void* cuda_stream, const float* x_s, const float* theta,
                                       const float* x_ref, const float* z_init, const float* lam_init,
                                       float* z_out, float* lam_out, int* status_out, int* pcg_iters_out,
                                       float* alpha_out) {
  if (!desc || batch < 1 || !x_s || !theta || !z_out) return DMPC_E_ARG;
  int ps = 0;
  if (!shape_ok(*desc, &ps)) return DMPC_E_UNSUPPORTED;
  dmpc_options o;
  if (opt) o = *opt; else dmpc_default_options(&o);
  if (o.sqp_iters < 1 || o.sqp_iters > 1000 || o.n_alpha < 1 || o.n_alpha > 8 || !(o.pcg_tol > 0.f) ||
      !(o.pcg_tol < 1.f) || o.pcg_max_iters < 1 || !(o.ru_delta > 0.f && o.ru_delta < 1.f) ||
      !(o.ls_eta > 0.f && o.ls_eta < 1.f) || !(o.feas_tol >= 0.f) || (o.pcg_precision != 0 && o.pcg_precision != 1) ||
      (o.exact_hessian != 0 && o.exact_hessian != 1) || (o.pcg_variant != 0 && o.pcg_variant != 1))
    return DMPC_E_ARG;
  for (int i = 0; i < o.n_alpha; ++i)
    if (!(o.alpha[i] > 0.f && o.alpha[i] <= 1.f)) return DMPC_E_ARG;

  const int nx = desc->nx, nu = desc->nu, T = desc->T, K = T + 1;
  OcpRec proto;
  std::memset(&proto, 0, sizeof(proto));
  const int implicit = desc->integrator == DMPC_INTEGRATOR_TRAPEZOID ? 1 : 0;
  const int kmodel = implicit ? desc->model + kTrapIdOffset : desc->model;  // kernel-side id
  proto.model = kmodel; proto.nx = nx; proto.nu = nu; proto.T = T; proto.dt = desc->dt;
  proto.n = K * nx + T * nu;
  proto.m = K * nx;
  proto.p = ps + T * (desc->model == DMPC_MODEL_LQ ? nx * nx + nx * nu + nx : 0) + 2 * nx + nu;

  int dev = 0, n_sm = 0, smem_optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DMPC_E_CUDA;
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);

  // tiling: the same rules as the regular path
  int team = o.team_threads;
  if (team == 0) {
    if (nx <= 6 && K <= 256) team = K <= 64 ? (nx <= 4 ? 32 : 64) : (K <= 128 ? 128 : 256);
    else team = K <= 32 ? 32 : (K <= 64 ? 64 : (K <= 128 ? 128 : 256));
  }
  if (team != 32 && team != 64 && team != 128 && team != 256) return DMPC_E_ARG;
  KernelEntry table[kMaxKernelEntries];
  const int n_entries = collect_kernel_entries(table);
  auto find = [&](int tm) -> LaunchFn {
    for (int i = 0; i < n_entries; ++i)
      if (table[i].team == tm && table[i].model == kmodel && table[i].nx == nx && table[i].nu == nu) return table[i].fn;
    return nullptr;
  };
  if (o.team_threads == 0 && !find(team)) {
    // a shape compiled for fewer team sizes (LQ with nx = 16: 32 threads) takes the one it has
    for (int alt : {32, 64, 128, 256})
      if (find(alt)) { team = alt; break; }
  }
  const int ws = make_layout(nx, nu, K, team, o.exact_hessian, implicit).total_floats;
  const size_t ws_bytes = (size_t)ws * sizeof(float);
  const bool use_gws = ws_bytes > (size_t)smem_optin;
  const int max_tpb = 256 / team;
  const int cap = use_gws ? max_tpb : std::min(max_tpb, (int)std::max<size_t>(1, (size_t)smem_optin / ws_bytes));
  int tpb = o.teams_per_block > 0 ? o.teams_per_block : std::max(1, std::min(cap, batch / std::max(1, n_sm)));
  tpb = std::max(1, std::min(tpb, cap));
  int grid = (batch + tpb - 1) / tpb;

  // scratch budget: records + work list (+ per-team workspace in global memory).  Teams walk
  // the work list (team g takes items g, g + G, ...), so any grid of at least one block
  // covers the batch: with a global workspace the grid is capped by what fits in the array.
  const size_t rec_bytes = ((size_t)batch * sizeof(OcpRec) + 255) & ~(size_t)255;
  const size_t ord_bytes = ((size_t)batch * sizeof(int) + 255) & ~(size_t)255;
  if (rec_bytes + ord_bytes > kScratchBytes) return DMPC_E_BUDGET;
  if (use_gws) {
    const size_t fit = (kScratchBytes - rec_bytes - ord_bytes) / ((size_t)tpb * ws_bytes);
    if (fit < 1) return DMPC_E_BUDGET;
    grid = (int)std::min<size_t>({(size_t)grid, (size_t)2 * n_sm, fit});
  }

  LaunchFn fn = find(team);
  if (!fn) return DMPC_E_UNSUPPORTED;

  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return DMPC_E_CUDA;
  unsigned char* sb = static_cast<unsigned char*>(base);
  OcpRec* recs = reinterpret_cast<OcpRec*>(sb);
  int* order = reinterpret_cast<int*>(sb + rec_bytes);
  float* gws = use_gws ? reinterpret_cast<float*>(sb + rec_bytes + ord_bytes) : nullptr;
  cudaStream_t s = (cudaStream_t)cuda_stream;

  noalloc_tables<<<std::min((batch + 255) / 256, 1024), 256, 0, s>>>(recs, order, batch, proto);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return DMPC_E_CUDA;

  KParams P;
  std::memset(&P, 0, sizeof(P));
  P.ocps = recs;
  P.order = order;
  P.n_work = batch;
  P.mode = MODE_SOLVE;
  P.opt.sqp_iters = o.sqp_iters;
  P.opt.line_search = o.line_search;
  P.opt.n_alpha = o.n_alpha;
  for (int i = 0; i < 8; ++i) P.opt.alpha[i] = o.alpha[i];
  P.opt.ls_eta = o.ls_eta;
  P.opt.feas_tol = o.feas_tol;
  P.opt.pcg_tol = o.pcg_tol;
  P.opt.pcg_max_iters = o.pcg_max_iters;
  P.opt.ru_delta = o.ru_delta;
  P.opt.pcg_precision = o.pcg_precision;
  P.opt.exact_hessian = o.exact_hessian;
  P.opt.pcg_variant = o.pcg_variant;
  P.x_s = x_s; P.theta = theta; P.x_ref = x_ref;
  P.z_init = z_init; P.lam_init_f = lam_init;
  P.z_out = z_out; P.lam_out = lam_out;
  P.status = status_out; P.pcg_iters = pcg_iters_out; P.alpha_hist = alpha_out;
  P.ws_floats = ws;
  P.gws = gws;
  P.use_gws = use_gws ? 1 : 0;
  P.teams_per_block = tpb;
  e = fn(P, grid, team * tpb, use_gws ? 0 : (size_t)tpb * ws_bytes, s);
  return e == cudaSuccess ? DMPC_OK : DMPC_E_CUDA;
}
