// Host/device shared plain-data structures of the DiffMPC CUDA path.
#pragma once
#include <stdint.h>

namespace dmpc {

// Per-OCP record (device table).  Offsets are element offsets into the caller's packed
// arrays: z (n floats per OCP), lambda (m), theta (p), x_s (nx), x_ref ((T+1) nx).
struct OcpRec {
  int model, nx, nu, T;
  float dt;
  int n, m, p;
  long long z_off, lam_off, th_off, xs_off, xref_off;
  long long gws_off;   // offset (floats) of this OCP's slot in the stored-Schur buffer
};

struct Options {
  int sqp_iters;
  int line_search;
  int n_alpha;
  float alpha[8];
  float ls_eta;
  float feas_tol;
  float pcg_tol;        // relative residual tolerance: sqrt(eta / eta_0) <= pcg_tol
  int pcg_max_iters;
  float ru_delta;       // reliable-update trigger: eta drops by ru_delta^2
  int pcg_precision;    // 0: FP32 iteration + FP64 reliable updates; 1: double-float throughout
  int exact_hessian;    // backward KKT matrix: 0 Gauss-Newton, 1 exact Hessian of the Lagrangian
  int pcg_variant;      // 0: Algorithm 4 as printed; 1: one-reduction reorganisation (single-warp teams)
};

enum KernelMode : int { MODE_SOLVE = 0, MODE_INSPECT = 1, MODE_VJP = 2 };

struct KParams {
  const OcpRec* ocps;
  const int* order;          // work list (OCP indices), heaviest first
  int n_work;
  unsigned char* cold;       // per-OCP flags (may be null): start this OCP cold, then clear the flag
  int mode;
  Options opt;
  // inputs
  const float* x_s;
  const float* theta;
  const float* x_ref;        // may be null: reference = 0
  const float* z_init;       // may be null
  const float* lam_init_f;   // may be null (float multipliers from the caller)
  const double* lam_init_d;  // may be null (resident multipliers)
  // forward outputs
  float* z_out;
  float* lam_out;
  float* res_z;              // resident warm-start copies (may be null)
  double* res_lam;
  float* res_xs;             // resident copies of the solve's inputs, read again by the vjp
  float* res_th;
  float* res_xref;
  int* status;
  int* pcg_iters;            // [ocp * sqp_iters + k] (may be null)
  float* alpha_hist;         // [ocp * sqp_iters + k] (may be null)
  // backward
  const float* dl_dz;
  const double* lamt_init;   // may be null
  double* res_lamt;          // resident adjoint multipliers (may be null)
  float* dl_dtheta;
  float* dl_dxs;
  float* lamt_out;           // may be null
  // stored Schur mode: forward writes, backward reads (may be null)
  float* store;
  int store_mode;            // 0 recompute in vjp, 1 use stored blocks
  // inspect output: per OCP a record at inspect_off[ocp] (floats)
  float* inspect;
  const long long* inspect_off;
  // workspace
  int ws_floats;             // per team
  float* gws;                // global per-team workspace (used when it does not fit in smem)
  int use_gws;
  int teams_per_block;
  int cl_kc;                 // cluster launches: knot capacity of one CTA's shared-memory layout
};

}  // namespace dmpc
