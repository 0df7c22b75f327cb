// C-ABI of the DiffMPC CUDA path (declared in include/dmpc.h): handle management, argument
// validation, layout, tiling choice and kernel launches.  No computation happens on the
// host; every step of solve / vjp / inspect runs in the fused kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/dmpc.h"
#include "fused.cuh"
#include "plain.cuh"
#include "launch.h"

using namespace dmpc;

namespace dmpc {
__global__ void plain_pcg_continue(const PlainState* st, const KParams* P, cudaGraphConditionalHandle cond) {
  const int n = P->n_work;
  const int* order = P->order;
  int any = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) any |= st[order ? order[i] : i].active;
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) cudaGraphSetConditional(cond, any ? 1u : 0u);
}
}  // namespace dmpc

namespace {

struct ModelInfo {
  int nx, nu, p_shared, integ;
};

bool model_info(int model, int nx, int nu, ModelInfo* mi) {
  switch (model) {
    case DMPC_MODEL_LQ:
      if (!((nx == 2 && nu == 1) || (nx == 3 && nu == 2) || (nx == 4 && nu == 1) || (nx == 8 && nu == 4) ||
            (nx == 16 && nu == 8)))
        return false;
      *mi = {nx, nu, 0, I_AFFINE};
      return true;
    case DMPC_MODEL_PENDULUM: *mi = {2, 1, 2, I_RK4}; break;
    case DMPC_MODEL_CARTPOLE: *mi = {4, 1, 2, I_RK4}; break;
    case DMPC_MODEL_KIN_BICYCLE: *mi = {4, 2, 1, I_RK4}; break;
    case DMPC_MODEL_SINGLE_TRACK: *mi = {6, 2, 2, I_RK4}; break;
    case DMPC_MODEL_RIGID_BODY12: *mi = {12, 4, 4, I_RK4}; break;
    case DMPC_MODEL_ATTITUDE: *mi = {3, 3, 3, I_EULER}; break;
    case DMPC_MODEL_SINGLE_TRACK_RATE: *mi = {8, 2, 2, I_RATE}; break;
    default: return false;
  }
  return mi->nx == nx && mi->nu == nu;
}

int p_knot(int model, int nx, int nu) { return model == DMPC_MODEL_LQ ? nx * nx + nx * nu + nx : 0; }

// Kernel-side model id: the trapezoidal (implicit) variants have their own instantiations.
// Returns -1 for an integrator the model does not support.
int kernel_model_id(const dmpc_ocp_desc& d) {
  if (d.integrator == DMPC_INTEGRATOR_DEFAULT) return d.model;
  if (d.integrator == DMPC_INTEGRATOR_TRAPEZOID &&
      (d.model == DMPC_MODEL_PENDULUM || d.model == DMPC_MODEL_CARTPOLE))
    return d.model + kTrapIdOffset;
  return -1;
}
int is_implicit_desc(const dmpc_ocp_desc& d) { return d.integrator == DMPC_INTEGRATOR_TRAPEZOID ? 1 : 0; }

std::mutex g_reg_mu;
std::vector<KernelEntry> g_registry;
std::string g_create_error;

std::vector<ClusterEntry> g_cl_registry;
std::once_flag g_cl_registry_once;
const std::vector<ClusterEntry>& cluster_registry() {
  std::call_once(g_cl_registry_once, [] {
    ClusterEntry buf[kMaxClusterEntries];
    const int n = collect_cluster_entries(buf);
    g_cl_registry.assign(buf, buf + n);
  });
  return g_cl_registry;
}

const std::vector<KernelEntry>& registry() {
  std::lock_guard<std::mutex> lk(g_reg_mu);
  if (g_registry.empty()) {
    KernelEntry buf[kMaxKernelEntries];
    int n = collect_kernel_entries(buf);
    g_registry.assign(buf, buf + n);
  }
  return g_registry;
}

}  // namespace

struct dmpc_handle {
  // pointers already found to be device memory (serving loops pass the same arena pointers
  // every tick; each cudaPointerGetAttributes costs microseconds of host time)
  const void* dev_ptr_seen[16] = {};
  unsigned dev_ptr_next = 0;
  int batch = 0;
  std::vector<dmpc_ocp_desc> descs;
  dmpc_options opt;
  cudaStream_t stream = nullptr;
  int device = 0;
  int n_sm = 0;
  int smem_optin = 0;
  std::vector<OcpRec> recs;
  std::vector<int> order;
  long long tot_z = 0, tot_lam = 0, tot_th = 0, tot_xs = 0, tot_xref = 0, tot_rec = 0, tot_store = 0;
  std::vector<long long> rec_off;
  OcpRec* d_recs = nullptr;
  int* d_order = nullptr;
  long long* d_rec_off = nullptr;
  float* res_z = nullptr;
  double* res_lam = nullptr;
  float* res_xs = nullptr;
  float* res_th = nullptr;
  float* res_xref = nullptr;
  bool last_had_xref = false;
  double* res_lamt = nullptr;
  float* store = nullptr;
  float* gws = nullptr;
  size_t gws_floats = 0;
  bool have_solution = false, have_lamt = false, have_store = false;
  // tiling
  bool uniform = true;
  int model0 = 0, nx0 = 0, nu0 = 0;
  int max_ws_floats = 0;  // per team, for team_threads
  int team = 32, tpb = 1, grid = 1;
  bool use_gws = false;
  size_t smem = 0;
  LaunchFn fn = nullptr;
  PlainFn plain_fn = nullptr;
  // cluster form (distributed PCG): CTAs per cluster, knot capacity per CTA, clusters resident
  bool use_cluster = false;
  int cl_ncta = 0, cl_kc = 0, cl_max = 0;
  ClusterLaunchFn cl_fn = nullptr;
  // plain one-launch-per-step form (allocated on first use)
  // serving: slot capacities (the shapes given at creation), cold-start flags, update staging
  std::vector<OcpRec> cap;
  unsigned char* d_cold = nullptr;
  OcpRec* d_upd = nullptr;
  int* d_upd_idx = nullptr;
  size_t bytes = 0;
  float* plain_ws = nullptr;
  PlainState* plain_st = nullptr;
  KParams* plain_params = nullptr;     // device copy of the plain form's launch parameters
  cudaStream_t plain_cap[2] = {nullptr, nullptr};  // capture streams (main sequence, PCG bodies)
  cudaGraphExec_t plain_graph[2] = {nullptr, nullptr};  // instantiated forward / backward graphs
  PlainFn plain_graph_fn[2] = {nullptr, nullptr};       // kernel set each graph was captured with
  int plain_graph_team[2] = {0, 0};
  int plain_ws_floats = 0;
  std::string err;
};

static dmpc_err fail(dmpc_handle* h, dmpc_err code, const std::string& msg) {
  if (h) h->err = msg; else g_create_error = msg;
  return code;
}

static dmpc_err cuda_fail(dmpc_handle* h, cudaError_t e, const char* what) {
  return fail(h, DMPC_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

extern "C" void dmpc_default_options(dmpc_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->sqp_iters = 1;
  o->line_search = 0;
  o->n_alpha = 5;
  const float a[5] = {1.0f, 0.7f, 0.3f, 0.1f, 0.01f};
  for (int i = 0; i < 5; ++i) o->alpha[i] = a[i];
  o->ls_eta = 0.4f;
  o->feas_tol = 1e-5f;
  o->pcg_tol = 1e-9f;
  o->pcg_max_iters = 1000;
  o->ru_delta = 0.1f;
  o->warm_start = 1;
  o->store_schur = 0;
  o->team_threads = 0;
  o->teams_per_block = 0;
  o->pcg_precision = 0;
  o->exact_hessian = 0;
  o->pcg_variant = 0;
  o->cluster_ctas = 0;
}

static Options to_kernel_options(const dmpc_options& o) {
  Options k;
  std::memset(&k, 0, sizeof(k));
  k.sqp_iters = o.sqp_iters;
  k.line_search = o.line_search;
  k.n_alpha = o.n_alpha;
  for (int i = 0; i < 8; ++i) k.alpha[i] = o.alpha[i];
  k.ls_eta = o.ls_eta;
  k.feas_tol = o.feas_tol;
  k.pcg_tol = o.pcg_tol;
  k.pcg_max_iters = o.pcg_max_iters;
  k.ru_delta = o.ru_delta;
  k.pcg_precision = o.pcg_precision;
  k.exact_hessian = o.exact_hessian;
  k.pcg_variant = o.pcg_variant;
  return k;
}

static dmpc_err validate_options(dmpc_handle* h, const dmpc_options& o) {
  if (o.sqp_iters < 1 || o.sqp_iters > 1000) return fail(h, DMPC_E_ARG, "sqp_iters must be in [1, 1000]");
  if (o.n_alpha < 1 || o.n_alpha > 8) return fail(h, DMPC_E_ARG, "n_alpha must be in [1, 8]");
  for (int i = 0; i < o.n_alpha; ++i)
    if (!(o.alpha[i] > 0.f && o.alpha[i] <= 1.f)) return fail(h, DMPC_E_ARG, "alpha values must be in (0, 1]");
  if (!(o.ls_eta > 0.f && o.ls_eta < 1.f)) return fail(h, DMPC_E_ARG, "ls_eta must be in (0, 1)");
  if (!(o.pcg_tol > 0.f && o.pcg_tol < 1.f)) return fail(h, DMPC_E_ARG, "pcg_tol must be in (0, 1)");
  if (o.pcg_max_iters < 1) return fail(h, DMPC_E_ARG, "pcg_max_iters must be >= 1");
  if (!(o.ru_delta > 0.f && o.ru_delta < 1.f)) return fail(h, DMPC_E_ARG, "ru_delta must be in (0, 1)");
  if (!(o.feas_tol >= 0.f)) return fail(h, DMPC_E_ARG, "feas_tol must be >= 0");
  if (o.team_threads != 0 && o.team_threads != 32 && o.team_threads != 64 && o.team_threads != 128 &&
      o.team_threads != 256)
    return fail(h, DMPC_E_ARG, "team_threads must be 0, 32, 64, 128 or 256");
  if (o.teams_per_block < 0) return fail(h, DMPC_E_ARG, "teams_per_block must be >= 0");
  if (o.pcg_precision != 0 && o.pcg_precision != 1) return fail(h, DMPC_E_ARG, "pcg_precision must be 0 or 1");
  if (o.exact_hessian != 0 && o.exact_hessian != 1) return fail(h, DMPC_E_ARG, "exact_hessian must be 0 or 1");
  if (o.pcg_variant != 0 && o.pcg_variant != 1) return fail(h, DMPC_E_ARG, "pcg_variant must be 0 or 1");
  if (o.cluster_ctas < 0 || o.cluster_ctas > kClMaxCtas)
    return fail(h, DMPC_E_ARG, "cluster_ctas must be in [0, 8]");
  return DMPC_OK;
}

static bool has_implicit_desc(const dmpc_handle* h) {
  for (auto& d : h->descs)
    if (is_implicit_desc(d)) return true;
  return false;
}

// Shape of the cluster form (Algorithm 4 distributed over a thread-block cluster) for OCPs of nx
// states, nu inputs and at most maxK knots: ncta CTAs per OCP, each holding kc = ceil(maxK / ncta)
// knots of the PCG's blocks in smem bytes of shared memory.  req = 0 chooses ncta from the longest
// horizon: about 40 knots per CTA, or as many as one CTA's shared memory holds where that is fewer
// (at most 8 CTAs): the fewest CTAs that hold the OCP, since an iteration's cost per CTA grows
// slowly with its knots (its chain is the two all-reduces) and fewer CTAs per OCP leave more SMs to
// the rest of a batch.  ncta = 0 when no shape fits the thread and shared-memory limits.
static void cluster_shape(int nx, int nu, int maxK, int req, size_t smem_limit, int* ncta_out, int* kc_out,
                          size_t* smem_out) {
  *ncta_out = 0;
  *kc_out = 0;
  *smem_out = 0;
  // (bounds far above any cluster shape keep the layout's int arithmetic from overflowing)
  if (nx < kClRows || nx % kClRows != 0 || nx > 512 || nu < 1 || nu > 512 || maxK < 1 || maxK > (1 << 20)) return;
  const int kc_max = cl_max_kc(nx);
  auto cl_bytes = [&](int kc) { return (size_t)cl_layout(nx, nu, kc).total * sizeof(float); };
  int ncta = req;
  if (ncta == 0) {
    // from ~40 knots per CTA up, the first count whose share fits the thread and shared-memory
    // limits (LQ with nx 16 holds at most 25 knots per CTA)
    ncta = std::min(kClMaxCtas, std::max(2, (maxK + 39) / 40));
    while (ncta < kClMaxCtas) {
      const int k = (maxK + ncta - 1) / ncta;
      if (k <= kc_max && cl_bytes(k) <= smem_limit) break;
      ++ncta;
    }
  }
  if (ncta < 2 || ncta > kClMaxCtas) return;
  const int kc = (maxK + ncta - 1) / ncta;
  if (kc > kc_max) return;
  const size_t smem = cl_bytes(kc);
  if (smem > smem_limit) return;
  *ncta_out = ncta;
  *kc_out = kc;
  *smem_out = smem;
}

// Cluster form for OCPs whose workspace does not fit in one CTA's shared memory: one cluster of
// ncta CTAs per OCP in the shape cluster_shape gives.  Leaves the single-team form in place when
// no cluster kernel fits.
static dmpc_err configure_cluster(dmpc_handle* h, int maxK) {
  const ClusterEntry* ce = nullptr;
  for (auto& e : cluster_registry())
    if (e.model == h->model0 && e.nx == h->nx0 && e.nu == h->nu0) ce = &e;
  if (!ce) return DMPC_OK;
  int ncta = 0, kc = 0;
  size_t smem = 0;
  cluster_shape(h->nx0, h->nu0, maxK, h->opt.cluster_ctas, (size_t)h->smem_optin, &ncta, &kc, &smem);
  if (ncta == 0) return DMPC_OK;
  const int fit = ce->max_clusters(ncta, smem);
  if (fit < 1) return DMPC_OK;
  // the leader runs the OCP as a 256-thread team: that team's kernels and workspace layout
  LaunchFn fn = h->fn;
  PlainFn pfn = h->plain_fn;
  if (h->team != kClThreads) {
    fn = nullptr;
    for (auto& e : registry())
      if (e.team == kClThreads && e.model == h->model0 && e.nx == h->nx0 && e.nu == h->nu0) { fn = e.fn; pfn = e.plain; }
    if (!fn) return DMPC_OK;
  }
  int ws = 0;
  for (auto& d : h->descs)
    ws = std::max(ws, make_layout(d.nx, d.nu, d.T + 1, kClThreads, h->opt.exact_hessian, 0).total_floats);
  const int ncl = std::min(h->batch, fit);
  const size_t need = (size_t)ncl * ws;
  if (need != h->gws_floats) {  // one slot per cluster (the single-team form may have sized it larger)
    if (h->gws) cudaFree(h->gws);
    h->gws = nullptr;
    cudaError_t e = cudaMalloc(&h->gws, need * sizeof(float));
    if (e != cudaSuccess) { h->gws_floats = 0; return fail(h, DMPC_E_OOM, "global workspace allocation failed"); }
    h->gws_floats = need;
  }
  h->team = kClThreads;
  h->fn = fn;
  h->plain_fn = pfn;
  h->max_ws_floats = ws;
  h->use_gws = true;   // the leader's workspace is a global slot per cluster
  h->use_cluster = true;
  h->cl_ncta = ncta;
  h->cl_kc = kc;
  h->cl_max = ncl;
  h->cl_fn = ce->fn;
  h->tpb = 1;
  h->grid = ncta * ncl;
  h->smem = smem;
  return DMPC_OK;
}

// Pick the kernel and launch shape for (team, tpb); tpb = 0 chooses automatically.
static dmpc_err configure_tiling(dmpc_handle* h, int team, int tpb) {
  int maxK = 0;
  for (auto& d : h->descs) maxK = std::max(maxK, d.T + 1);
  int maxnx = 0;
  for (auto& d : h->descs) maxnx = std::max(maxnx, d.nx);
  const bool team_is_default = team == 0;
  if (team == 0) {
    // one knot per lane (register-resident PCG) when it fits, else a few knots per lane:
    // nx <= 4: one warp with one or two knots per lane up to K = 64; nx <= 6: one knot per lane
    // (64 to 256 threads); larger nx: shared-memory PCG with one knot per thread up to 256
    if (maxnx <= 6 && maxK <= 256)
      team = maxK <= 64 ? (maxnx <= 4 ? 32 : 64) : (maxK <= 128 ? 128 : 256);
    else  // one knot per thread up to 256 threads (12-state rigid body, T 241: 107 ms on 256 against 195 on 128)
      team = maxK <= 32 ? 32 : (maxK <= 64 ? 64 : (maxK <= 128 ? 128 : 256));
  }
  if (h->uniform && team_is_default) {
    // a shape compiled for fewer team sizes (LQ with nx = 16: 32 threads) takes the one it has
    bool have = false;
    for (auto& e : registry()) have |= e.team == team && e.model == h->model0 && e.nx == h->nx0 && e.nu == h->nu0;
    for (int alt : {32, 64, 128, 256}) {
      if (have) break;
      for (auto& e : registry())
        if (e.team == alt && e.model == h->model0 && e.nx == h->nx0 && e.nu == h->nu0) { team = alt; have = true; break; }
    }
  }
  int ws = 0;
  for (auto& d : h->descs) ws = std::max(ws, make_layout(d.nx, d.nu, d.T + 1, team, h->opt.exact_hessian, is_implicit_desc(d)).total_floats);
  const size_t ws_bytes = (size_t)ws * sizeof(float);
  const int max_tpb_threads = 256 / team;
  h->use_gws = ws_bytes > (size_t)h->smem_optin;
  int smem_tpb = h->use_gws ? max_tpb_threads : (int)std::max<size_t>(1, (size_t)h->smem_optin / ws_bytes);
  int cap = std::min(max_tpb_threads, smem_tpb);
  if (tpb == 0) {
    tpb = std::max(1, std::min(cap, h->batch / std::max(1, h->n_sm)));
  }
  tpb = std::min(tpb, cap);
  if (tpb < 1) tpb = 1;
  // find the kernel
  LaunchFn fn = nullptr;
  PlainFn pfn = nullptr;
  for (auto& e : registry()) {
    if (e.team != team) continue;
    if (h->uniform && e.model == h->model0 && e.nx == h->nx0 && e.nu == h->nu0) { fn = e.fn; pfn = e.plain; break; }
  }
  if (!fn) {
    bool has_lq = false, has_implicit = false, has_rate = false;
    for (auto& d : h->descs) {
      has_lq |= d.model == DMPC_MODEL_LQ;
      has_implicit |= is_implicit_desc(d) != 0;
      has_rate |= d.model == DMPC_MODEL_SINGLE_TRACK_RATE;
    }
    if (has_lq) return fail(h, DMPC_E_UNSUPPORTED, "LQ OCPs cannot be mixed with other models in one batch");
    if (has_rate)
      return fail(h, DMPC_E_UNSUPPORTED, "control-rate OCPs cannot be mixed with other models in one batch");
    if (has_implicit)
      return fail(h, DMPC_E_UNSUPPORTED, "implicit-integrator OCPs cannot be mixed with other models in one batch");
    for (auto& e : registry())
      if (e.model == -1 && e.team == team) { fn = e.fn; pfn = e.plain; break; }
  }
  if (!fn) return fail(h, DMPC_E_UNSUPPORTED, "no kernel for this model / team size");
  int grid = (h->batch + tpb - 1) / tpb;
  if (h->use_gws) {
    grid = std::min(grid, 2 * h->n_sm);
    const size_t need = (size_t)grid * tpb * ws;
    if (need > h->gws_floats) {
      if (h->gws) cudaFree(h->gws);
      h->gws = nullptr;
      cudaError_t e = cudaMalloc(&h->gws, need * sizeof(float));
      if (e != cudaSuccess) { h->gws_floats = 0; return fail(h, DMPC_E_OOM, "global workspace allocation failed"); }
      h->gws_floats = need;
    }
  }
  h->team = team;
  h->tpb = tpb;
  h->grid = grid;
  h->max_ws_floats = ws;
  h->smem = h->use_gws ? 0 : (size_t)tpb * ws_bytes;
  h->fn = fn;
  h->plain_fn = pfn;
  h->use_cluster = false;
  // the cluster form where one CTA cannot hold the workspace, and for nx >= 16, whose one-warp team
  // would carry four 16 x 16 blocks per lane even when the workspace fits
  if ((h->use_gws || maxnx >= 16) && h->uniform && team_is_default && h->opt.cluster_ctas != 1 &&
      !has_implicit_desc(h)) {
    dmpc_err ce = configure_cluster(h, maxK);
    if (ce != DMPC_OK) return ce;
  }
  return DMPC_OK;
}

extern "C" dmpc_err dmpc_create_problem_batch(const dmpc_ocp_desc* descs, int batch, const dmpc_options* opt,
                                              void* cuda_stream, dmpc_handle** out) {
  if (!out) return fail(nullptr, DMPC_E_ARG, "out is NULL");
  *out = nullptr;
  if (!descs || batch < 1 || batch > (1 << 24)) return fail(nullptr, DMPC_E_ARG, "descs NULL or batch out of range");
  dmpc_handle* h = new dmpc_handle();
  if (opt) h->opt = *opt; else dmpc_default_options(&h->opt);
  dmpc_err er = validate_options(nullptr, h->opt);
  if (er != DMPC_OK) { delete h; return er; }
  h->batch = batch;
  h->descs.assign(descs, descs + batch);
  h->stream = (cudaStream_t)cuda_stream;
  cudaError_t ce = cudaGetDevice(&h->device);
  if (ce != cudaSuccess) { delete h; return cuda_fail(nullptr, ce, "cudaGetDevice"); }
  cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->device);
  cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  h->model0 = kernel_model_id(descs[0]); h->nx0 = descs[0].nx; h->nu0 = descs[0].nu;
  h->recs.resize(batch);
  h->rec_off.resize(batch + 1);
  std::vector<double> cost(batch);
  for (int b = 0; b < batch; ++b) {
    const dmpc_ocp_desc& d = descs[b];
    ModelInfo mi;
    if (!model_info(d.model, d.nx, d.nu, &mi)) {
      delete h;
      return fail(nullptr, DMPC_E_UNSUPPORTED, "OCP " + std::to_string(b) + ": unknown model or sizes not matching the model");
    }
    if (d.T < 1 || d.T > 4096) { delete h; return fail(nullptr, DMPC_E_ARG, "OCP " + std::to_string(b) + ": T must be in [1, 4096]"); }
    if (kernel_model_id(d) < 0) {
      delete h;
      return fail(nullptr, DMPC_E_UNSUPPORTED, "OCP " + std::to_string(b) + ": integrator not available for this model");
    }
    if (is_implicit_desc(d) && h->opt.exact_hessian) {
      delete h;
      return fail(nullptr, DMPC_E_UNSUPPORTED, "exact_hessian is not available with implicit integrators");
    }
    if (d.model != DMPC_MODEL_LQ && !(d.dt > 0.f && std::isfinite(d.dt))) {
      delete h;
      return fail(nullptr, DMPC_E_ARG, "OCP " + std::to_string(b) + ": dt must be positive");
    }
    h->uniform &= (kernel_model_id(d) == h->model0 && d.nx == h->nx0 && d.nu == h->nu0);
    const int K = d.T + 1;
    OcpRec& r = h->recs[b];
    r.model = kernel_model_id(d); r.nx = d.nx; r.nu = d.nu; r.T = d.T; r.dt = d.dt;
    r.n = K * d.nx + d.T * d.nu;
    r.m = K * d.nx;
    r.p = mi.p_shared + d.T * p_knot(d.model, d.nx, d.nu) + 2 * d.nx + d.nu;
    r.z_off = h->tot_z; h->tot_z += r.n;
    r.lam_off = h->tot_lam; h->tot_lam += r.m;
    r.th_off = h->tot_th; h->tot_th += r.p;
    r.xs_off = h->tot_xs; h->tot_xs += d.nx;
    r.xref_off = h->tot_xref; h->tot_xref += (long long)K * d.nx;
    r.gws_off = h->tot_store;
    h->tot_store += (long long)K * (5 * d.nx * d.nx + d.nx * d.nu);
    h->rec_off[b] = h->tot_rec;
    h->tot_rec += (long long)d.T * (d.nx * d.nx + d.nx * d.nu + d.nx) + (long long)K * d.nx +
                  4LL * K * d.nx * d.nx + 2LL * K * d.nx + r.n + 2;
    cost[b] = (double)K * d.nx * d.nx * (d.nx + 4);
  }
  h->rec_off[batch] = h->tot_rec;
  h->order.resize(batch);
  for (int b = 0; b < batch; ++b) h->order[b] = b;
  std::stable_sort(h->order.begin(), h->order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  // device tables and resident buffers
  auto dmal = [&](void** p, size_t bytes) { return cudaMalloc(p, std::max<size_t>(bytes, 16)); };
  if (dmal((void**)&h->d_recs, sizeof(OcpRec) * batch) != cudaSuccess ||
      dmal((void**)&h->d_order, sizeof(int) * batch) != cudaSuccess ||
      dmal((void**)&h->d_rec_off, sizeof(long long) * (batch + 1)) != cudaSuccess ||
      dmal((void**)&h->res_z, sizeof(float) * h->tot_z) != cudaSuccess ||
      dmal((void**)&h->res_lam, sizeof(double) * h->tot_lam) != cudaSuccess ||
      dmal((void**)&h->res_lamt, sizeof(double) * h->tot_lam) != cudaSuccess ||
      dmal((void**)&h->res_xs, sizeof(float) * h->tot_xs) != cudaSuccess ||
      dmal((void**)&h->res_th, sizeof(float) * h->tot_th) != cudaSuccess ||
      dmal((void**)&h->res_xref, sizeof(float) * h->tot_xref) != cudaSuccess) {
    dmpc_destroy(h);
    return fail(nullptr, DMPC_E_OOM, "device allocation failed");
  }
  if (h->opt.store_schur) {
    if (dmal((void**)&h->store, sizeof(float) * h->tot_store) != cudaSuccess) {
      dmpc_destroy(h);
      return fail(nullptr, DMPC_E_OOM, "stored-Schur buffer allocation failed");
    }
  }
  if (dmal((void**)&h->d_cold, batch) != cudaSuccess || dmal((void**)&h->d_upd, sizeof(OcpRec) * batch) != cudaSuccess ||
      dmal((void**)&h->d_upd_idx, sizeof(int) * 2 * batch) != cudaSuccess) {
    dmpc_destroy(h);
    return fail(nullptr, DMPC_E_OOM, "device allocation failed");
  }
  cudaMemset(h->d_cold, 0, batch);
  h->cap = h->recs;
  h->bytes = sizeof(OcpRec) * batch * 2 + sizeof(int) * batch * 3 + sizeof(long long) * (batch + 1) + batch +
             sizeof(float) * (h->tot_z + h->tot_xs + h->tot_th + h->tot_xref) + sizeof(double) * 2 * h->tot_lam +
             (h->store ? sizeof(float) * h->tot_store : 0);
  ce = cudaMemcpy(h->d_recs, h->recs.data(), sizeof(OcpRec) * batch, cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemcpy(h->d_order, h->order.data(), sizeof(int) * batch, cudaMemcpyHostToDevice);
  if (ce == cudaSuccess)
    ce = cudaMemcpy(h->d_rec_off, h->rec_off.data(), sizeof(long long) * (batch + 1), cudaMemcpyHostToDevice);
  if (ce != cudaSuccess) { dmpc_destroy(h); return cuda_fail(nullptr, ce, "table upload"); }
  er = configure_tiling(h, h->opt.team_threads, h->opt.teams_per_block);
  if (er != DMPC_OK) {
    g_create_error = h->err;
    dmpc_destroy(h);
    return er;
  }
  *out = h;
  return DMPC_OK;
}

extern "C" dmpc_err dmpc_layout(const dmpc_handle* h, long long* z_off, long long* lam_off, long long* theta_off,
                                long long* xs_off, long long* xref_off) {
  if (!h) return DMPC_E_ARG;
  for (int b = 0; b <= h->batch; ++b) {
    const bool last = b == h->batch;
    if (z_off) z_off[b] = last ? h->tot_z : h->recs[b].z_off;
    if (lam_off) lam_off[b] = last ? h->tot_lam : h->recs[b].lam_off;
    if (theta_off) theta_off[b] = last ? h->tot_th : h->recs[b].th_off;
    if (xs_off) xs_off[b] = last ? h->tot_xs : h->recs[b].xs_off;
    if (xref_off) xref_off[b] = last ? h->tot_xref : h->recs[b].xref_off;
  }
  return DMPC_OK;
}

extern "C" dmpc_err dmpc_inspect_offsets(const dmpc_handle* h, long long* rec_off) {
  if (!h || !rec_off) return DMPC_E_ARG;
  for (int b = 0; b <= h->batch; ++b) rec_off[b] = h->rec_off[b];
  return DMPC_OK;
}

static bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static KParams base_params(dmpc_handle* h) {
  KParams P;
  std::memset(&P, 0, sizeof(P));
  P.ocps = h->d_recs;
  P.order = h->d_order;
  P.n_work = h->batch;
  P.opt = to_kernel_options(h->opt);
  P.ws_floats = h->max_ws_floats;
  P.gws = h->gws;
  P.use_gws = h->use_gws ? 1 : 0;
  P.teams_per_block = h->tpb;
  return P;
}

// Launch the handle's kernel over n work items (the cluster form caps its clusters at n).
static cudaError_t launch_items(dmpc_handle* h, KParams P, int n) {
  if (h->use_cluster) {
    P.cl_kc = h->cl_kc;
    P.teams_per_block = 1;
    const int ncl = std::max(1, std::min(h->cl_max, n));
    return h->cl_fn(P, ncl * h->cl_ncta, h->cl_ncta, h->smem, h->stream);
  }
  const int grid = std::max(1, std::min(h->grid, (n + h->tpb - 1) / h->tpb));
  return h->fn(P, grid, h->team * h->tpb, h->smem, h->stream);
}

static dmpc_err launch(dmpc_handle* h, const KParams& P) {
  cudaError_t e = launch_items(h, P, P.n_work);
  if (e != cudaSuccess) return cuda_fail(h, e, "kernel launch");
  return DMPC_OK;
}

static bool is_device_ptr_seen(dmpc_handle* h, const void* p) {
  if (!p) return false;
  for (const void* q : h->dev_ptr_seen)
    if (q == p) return true;
  if (!is_device_ptr(p)) return false;
  h->dev_ptr_seen[h->dev_ptr_next++ % 16] = p;
  return true;
}

#define REQUIRE_DEV(ptr, name) \
  if (!is_device_ptr_seen(h, ptr)) return fail(h, DMPC_E_ARG, std::string(name) + " must be a device pointer")
#define OPTIONAL_DEV(ptr, name) \
  if ((ptr) && !is_device_ptr_seen(h, ptr)) return fail(h, DMPC_E_ARG, std::string(name) + " must be a device pointer")

extern "C" dmpc_err dmpc_solve(dmpc_handle* h, const float* x_s, const float* theta, const float* x_ref,
                               const float* z_init, const float* lam_init, float* z_out, float* lam_out,
                               int* status_out, int* pcg_iters_out, float* alpha_out) {
  if (!h) return DMPC_E_ARG;
  REQUIRE_DEV(x_s, "x_s");
  REQUIRE_DEV(theta, "theta");
  REQUIRE_DEV(z_out, "z_out");
  OPTIONAL_DEV(x_ref, "x_ref");
  OPTIONAL_DEV(z_init, "z_init");
  OPTIONAL_DEV(lam_init, "lam_init");
  OPTIONAL_DEV(lam_out, "lam_out");
  OPTIONAL_DEV(status_out, "status_out");
  OPTIONAL_DEV(pcg_iters_out, "pcg_iters_out");
  OPTIONAL_DEV(alpha_out, "alpha_out");
  KParams P = base_params(h);
  P.mode = MODE_SOLVE;
  P.x_s = x_s; P.theta = theta; P.x_ref = x_ref;
  const bool warm = h->opt.warm_start && h->have_solution;
  P.z_init = z_init ? z_init : (warm ? h->res_z : nullptr);
  P.lam_init_f = lam_init;
  P.lam_init_d = (!lam_init && warm) ? h->res_lam : nullptr;
  P.z_out = z_out; P.lam_out = lam_out;
  P.res_z = h->res_z; P.res_lam = h->res_lam;
  P.res_xs = h->res_xs; P.res_th = h->res_th; P.res_xref = h->res_xref;
  P.status = status_out; P.pcg_iters = pcg_iters_out; P.alpha_hist = alpha_out;
  P.store = h->store;
  P.store_mode = (h->opt.store_schur && h->store) ? 1 : 0;
  dmpc_err e = launch(h, P);
  if (e != DMPC_OK) return e;
  h->have_solution = true;
  h->have_store = P.store_mode != 0;
  h->last_had_xref = x_ref != nullptr;
  return DMPC_OK;
}

extern "C" dmpc_err dmpc_vjp(dmpc_handle* h, const float* dl_dz, float* dl_dtheta, float* dl_dxs, float* lamt_out,
                             int* status_out, int* pcg_iters_out) {
  if (!h) return DMPC_E_ARG;
  if (!h->have_solution) return fail(h, DMPC_E_STATE, "dmpc_vjp called before any dmpc_solve on this handle");
  REQUIRE_DEV(dl_dz, "dl_dz");
  REQUIRE_DEV(dl_dtheta, "dl_dtheta");
  REQUIRE_DEV(dl_dxs, "dl_dxs");
  OPTIONAL_DEV(lamt_out, "lamt_out");
  OPTIONAL_DEV(status_out, "status_out");
  OPTIONAL_DEV(pcg_iters_out, "pcg_iters_out");
  KParams P = base_params(h);
  P.mode = MODE_VJP;
  // the forward kernel kept copies of its inputs on the device
  P.x_s = h->res_xs; P.theta = h->res_th; P.x_ref = h->last_had_xref ? h->res_xref : nullptr;
  P.z_init = h->res_z;
  P.lam_init_d = h->res_lam;
  P.dl_dz = dl_dz;
  P.lamt_init = (h->opt.warm_start && h->have_lamt) ? h->res_lamt : nullptr;
  P.res_lamt = h->res_lamt;
  P.dl_dtheta = dl_dtheta; P.dl_dxs = dl_dxs; P.lamt_out = lamt_out;
  P.status = status_out; P.pcg_iters = pcg_iters_out;
  P.store = h->store;
  P.store_mode = h->have_store ? 1 : 0;
  dmpc_err e = launch(h, P);
  if (e != DMPC_OK) return e;
  h->have_lamt = true;
  return DMPC_OK;
}

extern "C" dmpc_err dmpc_qp_inspect(dmpc_handle* h, const float* x_s, const float* theta, const float* x_ref,
                                    const float* z, const float* lam, float* record) {
  if (!h) return DMPC_E_ARG;
  REQUIRE_DEV(x_s, "x_s");
  REQUIRE_DEV(theta, "theta");
  REQUIRE_DEV(z, "z");
  REQUIRE_DEV(record, "record");
  OPTIONAL_DEV(x_ref, "x_ref");
  OPTIONAL_DEV(lam, "lam");
  KParams P = base_params(h);
  P.mode = MODE_INSPECT;
  P.x_s = x_s; P.theta = theta; P.x_ref = x_ref;
  P.z_init = z;
  P.lam_init_f = lam;
  P.inspect = record;
  P.inspect_off = h->d_rec_off;
  return launch(h, P);
}

// ---------------------------------------------------------------------------------------
// Plain one-launch-per-step form (the comparator of the fused kernel): the same stages, one
// launch per step over the batch, per-OCP workspace in HBM.  All launches of a solve (or a vjp)
// form one CUDA graph, captured once per handle: each PCG solve is a conditional WHILE node
// whose body runs kPlainUnroll PCG iterations (four launches each) and plain_pcg_continue, which
// ends the loop on the device once no OCP is still iterating.  The launch parameters live in
// device memory (plain_params), written with one copy before each graph launch.
static const int kPlainUnroll = 8;

static dmpc_err plain_prepare(dmpc_handle* h, KParams* P) {
  const int team = h->team;
  int ws = 0;
  for (auto& d : h->descs) ws = std::max(ws, make_layout(d.nx, d.nu, d.T + 1, team, h->opt.exact_hessian, is_implicit_desc(d)).total_floats);
  if (!h->plain_ws || ws != h->plain_ws_floats) {
    cudaFree(h->plain_ws);
    h->plain_ws = nullptr;
    if (cudaMalloc(&h->plain_ws, (size_t)ws * h->batch * sizeof(float)) != cudaSuccess)
      return fail(h, DMPC_E_OOM, "plain-form workspace allocation failed");
    h->plain_ws_floats = ws;
  }
  if (!h->plain_st) {
    if (cudaMalloc(&h->plain_st, sizeof(PlainState) * h->batch) != cudaSuccess ||
        cudaMalloc(&h->plain_params, sizeof(KParams)) != cudaSuccess)
      return fail(h, DMPC_E_OOM, "plain-form state allocation failed");
    cudaMemsetAsync(h->plain_st, 0, sizeof(PlainState) * h->batch, h->stream);
  }
  if (!h->plain_cap[0]) {
    for (int i = 0; i < 2; ++i)
      if (cudaStreamCreateWithFlags(&h->plain_cap[i], cudaStreamNonBlocking) != cudaSuccess)
        return fail(h, DMPC_E_CUDA, "plain-form capture stream creation failed");
  }
  if (!h->plain_fn) return fail(h, DMPC_E_UNSUPPORTED, "no plain-form kernel for this batch");
  P->gws = h->plain_ws;
  P->use_gws = 1;
  P->ws_floats = ws;
  P->teams_per_block = 1;
  return DMPC_OK;
}

// Capture one PCG solve as a conditional WHILE node on the capture stream cs (its body captured
// on cb).  The condition starts at 1 on every launch; the body's last kernel sets it.
static cudaError_t capture_pcg_loop(dmpc_handle* h, cudaStream_t cs, cudaStream_t cb, int grid) {
  cudaStreamCaptureStatus status;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(cs, &status, nullptr, &g, &deps, nullptr, &ndeps);
  if (e != cudaSuccess) return e;
  if (status != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  cudaGraphConditionalHandle cond;
  e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
  np.conditional.handle = cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &np);
  if (e != cudaSuccess) return e;
  e = cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e != cudaSuccess) return e;
  cudaGraph_t body = np.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(cb, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  for (int u = 0; u < kPlainUnroll && e == cudaSuccess; ++u)
    for (int step : {PS_MATVEC, PS_AXPY, PS_PRECAPPLY, PS_BETA})
      if (e == cudaSuccess) e = h->plain_fn(h->plain_params, h->plain_st, step, 0, grid, h->team, cb);
  if (e == cudaSuccess) {
    plain_pcg_continue<<<1, 256, 0, cb>>>(h->plain_st, h->plain_params, cond);
    e = cudaGetLastError();
  }
  cudaGraph_t out = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cb, &out);
  return e != cudaSuccess ? e : e2;
}

// The graph of a forward solve (which = 0: load, per SQP iteration linearise / Schur /
// preconditioner / PCG setup / PCG loop / finish / recovery / line search, outputs) or of a vjp
// (which = 1), built on first use and rebuilt when the tiling changed.
static dmpc_err plain_graph(dmpc_handle* h, int which, cudaGraphExec_t* out) {
  if (h->plain_graph[which] && h->plain_graph_fn[which] == h->plain_fn && h->plain_graph_team[which] == h->team) {
    *out = h->plain_graph[which];
    return DMPC_OK;
  }
  if (h->plain_graph[which]) cudaGraphExecDestroy(h->plain_graph[which]);
  h->plain_graph[which] = nullptr;
  cudaStream_t cs = h->plain_cap[0], cb = h->plain_cap[1];
  const int grid = h->batch;  // blocks beyond the solve's work list return at once
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(h, e, "plain-form graph capture");
  auto L = [&](int step, int s_iter) {
    if (e == cudaSuccess) e = h->plain_fn(h->plain_params, h->plain_st, step, s_iter, grid, h->team, cs);
  };
  auto loop = [&]() {
    if (e == cudaSuccess) e = capture_pcg_loop(h, cs, cb, grid);
  };
  if (which == 0) {
    L(PS_LOAD, 0);
    for (int s_iter = 0; s_iter < h->opt.sqp_iters; ++s_iter) {
      L(PS_LIN, s_iter); L(PS_SCHUR, s_iter); L(PS_PREC, s_iter); L(PS_PCG_SETUP, s_iter);
      loop();
      L(PS_PCG_FINISH, s_iter); L(PS_RECOVER, s_iter); L(PS_LS, s_iter);
    }
    L(PS_FWD_OUT, 0);
  } else {
    L(PS_LOAD, 0); L(PS_LIN, 0); L(PS_SCHUR, 0); L(PS_PREC, 0); L(PS_PCG_SETUP, 0);
    loop();
    L(PS_PCG_FINISH, 0); L(PS_BWD_FINISH, 0);
  }
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cs, &g);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&h->plain_graph[which], g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    h->plain_graph[which] = nullptr;
    cudaGetLastError();
    return cuda_fail(h, e, "plain-form graph build");
  }
  h->plain_graph_fn[which] = h->plain_fn;
  h->plain_graph_team[which] = h->team;
  *out = h->plain_graph[which];
  return DMPC_OK;
}

// Write the launch parameters to the device and launch the forward (0) or vjp (1) graph on the
// handle's stream.  Asynchronous.
static dmpc_err plain_launch(dmpc_handle* h, const KParams& P, int which) {
  cudaGraphExec_t exec = nullptr;
  dmpc_err er = plain_graph(h, which, &exec);
  if (er != DMPC_OK) return er;
  cudaError_t e = cudaMemcpyAsync(h->plain_params, &P, sizeof(KParams), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "plain-form graph launch");
  return DMPC_OK;
}

extern "C" dmpc_err dmpc_solve_plain(dmpc_handle* h, const float* x_s, const float* theta, const float* x_ref,
                                     const float* z_init, const float* lam_init, float* z_out, float* lam_out,
                                     int* status_out, int* pcg_iters_out, float* alpha_out) {
  if (!h) return DMPC_E_ARG;
  REQUIRE_DEV(x_s, "x_s");
  REQUIRE_DEV(theta, "theta");
  REQUIRE_DEV(z_out, "z_out");
  OPTIONAL_DEV(x_ref, "x_ref");
  OPTIONAL_DEV(z_init, "z_init");
  OPTIONAL_DEV(lam_init, "lam_init");
  OPTIONAL_DEV(lam_out, "lam_out");
  OPTIONAL_DEV(status_out, "status_out");
  OPTIONAL_DEV(pcg_iters_out, "pcg_iters_out");
  OPTIONAL_DEV(alpha_out, "alpha_out");
  KParams P = base_params(h);
  dmpc_err er = plain_prepare(h, &P);
  if (er != DMPC_OK) return er;
  P.mode = MODE_SOLVE;
  P.x_s = x_s; P.theta = theta; P.x_ref = x_ref;
  const bool warm = h->opt.warm_start && h->have_solution;
  P.z_init = z_init ? z_init : (warm ? h->res_z : nullptr);
  P.lam_init_f = lam_init;
  P.lam_init_d = (!lam_init && warm) ? h->res_lam : nullptr;
  P.z_out = z_out; P.lam_out = lam_out;
  P.res_z = h->res_z; P.res_lam = h->res_lam;
  P.res_xs = h->res_xs; P.res_th = h->res_th; P.res_xref = h->res_xref;
  P.status = status_out; P.pcg_iters = pcg_iters_out; P.alpha_hist = alpha_out;
  er = plain_launch(h, P, 0);
  if (er != DMPC_OK) return er;
  h->have_solution = true;
  h->have_store = false;
  h->last_had_xref = x_ref != nullptr;
  return DMPC_OK;
}

extern "C" dmpc_err dmpc_vjp_plain(dmpc_handle* h, const float* dl_dz, float* dl_dtheta, float* dl_dxs,
                                   float* lamt_out, int* status_out, int* pcg_iters_out) {
  if (!h) return DMPC_E_ARG;
  if (!h->have_solution) return fail(h, DMPC_E_STATE, "dmpc_vjp_plain called before any solve on this handle");
  REQUIRE_DEV(dl_dz, "dl_dz");
  REQUIRE_DEV(dl_dtheta, "dl_dtheta");
  REQUIRE_DEV(dl_dxs, "dl_dxs");
  OPTIONAL_DEV(lamt_out, "lamt_out");
  OPTIONAL_DEV(status_out, "status_out");
  OPTIONAL_DEV(pcg_iters_out, "pcg_iters_out");
  KParams P = base_params(h);
  dmpc_err er = plain_prepare(h, &P);
  if (er != DMPC_OK) return er;
  P.mode = MODE_VJP;
  P.x_s = h->res_xs; P.theta = h->res_th; P.x_ref = h->last_had_xref ? h->res_xref : nullptr;
  P.z_init = h->res_z;
  P.lam_init_d = h->res_lam;
  P.dl_dz = dl_dz;
  P.lamt_init = (h->opt.warm_start && h->have_lamt) ? h->res_lamt : nullptr;
  P.res_lamt = h->res_lamt;
  P.dl_dtheta = dl_dtheta; P.dl_dxs = dl_dxs; P.lamt_out = lamt_out;
  P.status = status_out; P.pcg_iters = pcg_iters_out;   // written by the backward's last step only
  er = plain_launch(h, P, 1);
  if (er != DMPC_OK) return er;
  h->have_lamt = true;
  return DMPC_OK;
}

// ---------------------------------------------------------------------------------------
// Serving: re-describe slots within their capacity and solve a subset of them.
namespace dmpc {
__global__ void apply_slot_updates(OcpRec* recs, unsigned char* cold, const OcpRec* upd, const int* idx_reset,
                                   int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int b = idx_reset[2 * i];
    recs[b] = upd[i];
    if (idx_reset[2 * i + 1]) cold[b] = 1;
  }
}
}  // namespace dmpc

extern "C" dmpc_err dmpc_set_ocps(dmpc_handle* h, int n, const int* index, const dmpc_ocp_desc* descs,
                                  const int* reset) {
  if (!h || n < 0 || (n > 0 && (!index || !descs))) return DMPC_E_ARG;
  if (n == 0) return DMPC_OK;
  if (n > h->batch) return fail(h, DMPC_E_ARG, "more updates than slots");
  std::vector<OcpRec> upd(n);
  std::vector<int> idx_reset(2 * n);
  for (int i = 0; i < n; ++i) {
    const int b = index[i];
    if (b < 0 || b >= h->batch) return fail(h, DMPC_E_ARG, "slot index out of range");
    const dmpc_ocp_desc& d = descs[i];
    ModelInfo mi;
    if (!model_info(d.model, d.nx, d.nu, &mi) || d.T < 1 || kernel_model_id(d) < 0)
      return fail(h, DMPC_E_UNSUPPORTED, "bad slot shape");
    if (h->uniform && (kernel_model_id(d) != h->model0 || d.nx != h->nx0 || d.nu != h->nu0))
      return fail(h, DMPC_E_UNSUPPORTED, "a single-model handle cannot take another model");
    if (is_implicit_desc(d) && h->opt.exact_hessian)
      return fail(h, DMPC_E_UNSUPPORTED, "exact_hessian is not available with implicit integrators");
    if (d.model != DMPC_MODEL_LQ && !(d.dt > 0.f)) return fail(h, DMPC_E_ARG, "dt must be positive");
    const OcpRec& c = h->cap[b];
    OcpRec r = c;
    const int K = d.T + 1;
    r.model = kernel_model_id(d); r.nx = d.nx; r.nu = d.nu; r.T = d.T; r.dt = d.dt;
    r.n = K * d.nx + d.T * d.nu;
    r.m = K * d.nx;
    r.p = mi.p_shared + d.T * p_knot(d.model, d.nx, d.nu) + 2 * d.nx + d.nu;
    if (r.n > c.n || r.m > c.m || r.p > c.p || d.nx > c.nx || (long long)K * d.nx > (long long)(c.T + 1) * c.nx ||
        (long long)K * (5 * d.nx * d.nx + d.nx * d.nu) > (long long)(c.T + 1) * (5 * c.nx * c.nx + c.nx * c.nu) ||
        make_layout(d.nx, d.nu, K, h->team, h->opt.exact_hessian, is_implicit_desc(d)).total_floats > h->max_ws_floats)
      return fail(h, DMPC_E_BUDGET, "shape exceeds the slot's capacity");
    h->recs[b] = r;
    upd[i] = r;
    idx_reset[2 * i] = b;
    idx_reset[2 * i + 1] = reset ? reset[i] : 0;
  }
  // pageable sources: the copies are staged before these calls return
  cudaError_t e = cudaMemcpyAsync(h->d_upd, upd.data(), sizeof(OcpRec) * n, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d_upd_idx, idx_reset.data(), sizeof(int) * 2 * n, cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "slot update upload");
  apply_slot_updates<<<(n + 255) / 256, 256, 0, h->stream>>>(h->d_recs, h->d_cold, h->d_upd, h->d_upd_idx, n);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "slot update");
  return DMPC_OK;
}

static dmpc_err subset_common(dmpc_handle* h, const int* index, int n, const float* x_s, const float* theta,
                              const float* x_ref, float* z_out, KParams* P) {
  if (!h) return DMPC_E_ARG;
  if (n < 0 || n > h->batch) return fail(h, DMPC_E_ARG, "subset size out of range");
  REQUIRE_DEV(index, "index");
  REQUIRE_DEV(x_s, "x_s");
  REQUIRE_DEV(theta, "theta");
  REQUIRE_DEV(z_out, "z_out");
  OPTIONAL_DEV(x_ref, "x_ref");
  *P = base_params(h);
  P->order = index;
  P->n_work = n;
  P->cold = h->d_cold;
  P->mode = MODE_SOLVE;
  P->x_s = x_s; P->theta = theta; P->x_ref = x_ref;
  // every slot continues from its resident iterate unless it was reset
  P->z_init = h->res_z;
  P->lam_init_d = h->res_lam;
  P->z_out = z_out;
  P->res_z = h->res_z; P->res_lam = h->res_lam;
  P->res_xs = h->res_xs; P->res_th = h->res_th; P->res_xref = h->res_xref;
  return DMPC_OK;
}

extern "C" dmpc_err dmpc_solve_subset(dmpc_handle* h, const int* index, int n, const float* x_s, const float* theta,
                                      const float* x_ref, float* z_out, float* lam_out, int* status_out,
                                      int* pcg_iters_out, float* alpha_out) {
  KParams P;
  dmpc_err er = subset_common(h, index, n, x_s, theta, x_ref, z_out, &P);
  if (er != DMPC_OK || n == 0) return er;
  OPTIONAL_DEV(lam_out, "lam_out");
  P.lam_out = lam_out; P.status = status_out; P.pcg_iters = pcg_iters_out; P.alpha_hist = alpha_out;
  cudaError_t e = launch_items(h, P, n);
  if (e != cudaSuccess) return cuda_fail(h, e, "kernel launch");
  h->have_solution = true;
  h->last_had_xref = x_ref != nullptr;
  return DMPC_OK;
}

extern "C" dmpc_err dmpc_solve_subset_plain(dmpc_handle* h, const int* index, int n, const float* x_s,
                                            const float* theta, const float* x_ref, float* z_out, float* lam_out,
                                            int* status_out, int* pcg_iters_out, float* alpha_out) {
  KParams P;
  dmpc_err er = subset_common(h, index, n, x_s, theta, x_ref, z_out, &P);
  if (er != DMPC_OK || n == 0) return er;
  OPTIONAL_DEV(lam_out, "lam_out");
  er = plain_prepare(h, &P);
  if (er != DMPC_OK) return er;
  P.lam_out = lam_out; P.status = status_out; P.pcg_iters = pcg_iters_out; P.alpha_hist = alpha_out;
  er = plain_launch(h, P, 0);
  if (er != DMPC_OK) return er;
  h->have_solution = true;
  h->last_had_xref = x_ref != nullptr;
  return DMPC_OK;
}

extern "C" long long dmpc_device_bytes(const dmpc_handle* h) {
  if (!h) return -1;
  long long b = (long long)h->bytes + (long long)h->gws_floats * (long long)sizeof(float);
  if (h->plain_ws) b += (long long)h->plain_ws_floats * h->batch * (long long)sizeof(float) +
                       (long long)sizeof(PlainState) * h->batch + (long long)sizeof(KParams);
  return b;
}

__global__ void widen_to_double(const float* src, double* dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (double)src[i];
}

extern "C" dmpc_err dmpc_set_solution(dmpc_handle* h, const float* z, const float* lam, const float* x_s,
                                      const float* theta, const float* x_ref) {
  if (!h) return DMPC_E_ARG;
  REQUIRE_DEV(z, "z");
  REQUIRE_DEV(lam, "lam");
  REQUIRE_DEV(x_s, "x_s");
  REQUIRE_DEV(theta, "theta");
  OPTIONAL_DEV(x_ref, "x_ref");
  const cudaStream_t s = h->stream;
  cudaError_t e = cudaMemcpyAsync(h->res_z, z, sizeof(float) * h->tot_z, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->res_xs, x_s, sizeof(float) * h->tot_xs, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->res_th, theta, sizeof(float) * h->tot_th, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && x_ref)
    e = cudaMemcpyAsync(h->res_xref, x_ref, sizeof(float) * h->tot_xref, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "set_solution copy");
  if (h->tot_lam > 0) {
    const int grid = (int)std::min<long long>(4 * (long long)h->n_sm, (h->tot_lam + 255) / 256);
    widen_to_double<<<grid, 256, 0, s>>>(lam, h->res_lam, h->tot_lam);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "set_solution kernel");
  }
  h->have_solution = true;
  h->have_store = false;
  h->last_had_xref = x_ref != nullptr;
  return DMPC_OK;
}

extern "C" dmpc_err dmpc_set_stream(dmpc_handle* h, void* s) {
  if (!h) return DMPC_E_ARG;
  h->stream = (cudaStream_t)s;
  return DMPC_OK;
}

extern "C" dmpc_err dmpc_set_tiling(dmpc_handle* h, int team_threads, int teams_per_block) {
  if (!h) return DMPC_E_ARG;
  if (team_threads == 0 && teams_per_block == 0) return configure_tiling(h, 0, 0);   // the automatic choice
  if (team_threads != 32 && team_threads != 64 && team_threads != 128 && team_threads != 256)
    return fail(h, DMPC_E_ARG, "team_threads must be 32, 64, 128 or 256");
  if (teams_per_block < 1 || team_threads * teams_per_block > 256)
    return fail(h, DMPC_E_ARG, "teams_per_block must be >= 1 with team_threads * teams_per_block <= 256");
  return configure_tiling(h, team_threads, teams_per_block);
}

extern "C" dmpc_err dmpc_get_tiling(const dmpc_handle* h, int* team_threads, int* teams_per_block, int* grid,
                                    long long* smem_bytes) {
  if (!h) return DMPC_E_ARG;
  if (team_threads) *team_threads = h->team;
  if (teams_per_block) *teams_per_block = h->tpb;
  if (grid) *grid = h->grid;
  if (smem_bytes) *smem_bytes = (long long)h->smem;
  return DMPC_OK;
}

extern "C" dmpc_err dmpc_cluster_shape(int nx, int nu, int knots, int cluster_ctas, long long smem_per_cta,
                                       int* ctas_per_cluster, int* knots_per_cta, long long* smem_bytes) {
  if (nx < 1 || nu < 1 || knots < 1 || cluster_ctas < 0 || cluster_ctas > kClMaxCtas || smem_per_cta < 0)
    return DMPC_E_ARG;
  int ncta = 0, kc = 0;
  size_t smem = 0;
  cluster_shape(nx, nu, knots, cluster_ctas, (size_t)smem_per_cta, &ncta, &kc, &smem);
  if (ctas_per_cluster) *ctas_per_cluster = ncta;
  if (knots_per_cta) *knots_per_cta = kc;
  if (smem_bytes) *smem_bytes = (long long)smem;
  return DMPC_OK;
}

extern "C" dmpc_err dmpc_get_cluster(const dmpc_handle* h, int* ctas_per_cluster, int* knots_per_cta,
                                     int* clusters) {
  if (!h) return DMPC_E_ARG;
  if (ctas_per_cluster) *ctas_per_cluster = h->use_cluster ? h->cl_ncta : 0;
  if (knots_per_cta) *knots_per_cta = h->use_cluster ? h->cl_kc : 0;
  if (clusters) *clusters = h->use_cluster ? h->cl_max : 0;
  return DMPC_OK;
}

extern "C" void dmpc_destroy(dmpc_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream); else cudaDeviceSynchronize();
  cudaFree(h->d_recs);
  cudaFree(h->d_order);
  cudaFree(h->d_rec_off);
  cudaFree(h->res_z);
  cudaFree(h->res_lam);
  cudaFree(h->res_lamt);
  cudaFree(h->res_xs);
  cudaFree(h->res_th);
  cudaFree(h->res_xref);
  cudaFree(h->store);
  cudaFree(h->gws);
  cudaFree(h->d_cold);
  cudaFree(h->d_upd);
  cudaFree(h->d_upd_idx);
  cudaFree(h->plain_ws);
  cudaFree(h->plain_st);
  cudaFree(h->plain_params);
  for (int i = 0; i < 2; ++i) {
    if (h->plain_graph[i]) cudaGraphExecDestroy(h->plain_graph[i]);
    if (h->plain_cap[i]) cudaStreamDestroy(h->plain_cap[i]);
  }
  delete h;
}

extern "C" const char* dmpc_last_error(const dmpc_handle* h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

extern "C" const char* dmpc_version(void) { return "dmpc-gb300 0.1 (sm_103a)"; }
