// The plain one-launch-per-step form of the same method: every step of an SQP iteration
// (load, linearise, Schur blocks, preconditioner, each PCG operation of Algorithm 4, recovery,
// line search, outputs) is its own kernel launch over the batch, the per-OCP workspace (the S
// and Phi^-1 blocks included) lives in HBM and the PCG scalars of each OCP are kept in HBM
// between launches.  The launches of a solve form one CUDA graph; each PCG solve is a
// conditional WHILE node whose body (a few PCG iterations, then plain_pcg_continue) repeats
// until no OCP of the batch is still iterating, so convergence is decided on the device with no
// host round trip.  It reuses the stage functions of the fused form, so both compute the same
// arithmetic; it is the comparator the fused form is measured against.
#pragma once
#include "fused.cuh"

namespace dmpc {

struct PlainState {
  float eta, eta0, eta_ref, eta_true;
  int it, stall, active, converged, folded, status;
};

enum PlainStep : int {
  PS_LOAD = 0, PS_LIN, PS_SCHUR, PS_PREC, PS_PCG_SETUP, PS_MATVEC, PS_AXPY, PS_PRECAPPLY, PS_BETA,
  PS_PCG_FINISH, PS_RECOVER, PS_LS, PS_FWD_OUT, PS_BWD_FINISH
};

// One PCG setup step: initial guess, FP64 true residual, preconditioned residual, eta, eta_0.
template <class M, int TEAM>
__device__ __noinline__ void plain_pcg_setup(Ctx<M, TEAM>& c, PlainState& S) {
  constexpr int NX = M::NX;
  const KParams& P = *c.P;
  const int K = c.K, KP = c.KP;
  if (P.mode == MODE_VJP) stage_bwd_rhs<M, TEAM>(c);
  else copy_lam_to_lamp<M, TEAM>(c);
  float* R = c.F(c.L.r);
  float* Pv = c.F(c.L.p);
  float* Y = c.F(c.L.y);
  float* DL = c.F(c.L.dl);
  const double* G = c.Dp(c.L.d_gam);
  for (int k = c.tm.lane; k < K; k += TEAM)
#pragma unroll
    for (int i = 0; i < NX; ++i) { Y[i * KP + k] = (float)G[i * KP + k]; DL[i * KP + k] = 0.f; }
  hp_residual<M, TEAM>(c, c.Dp(c.L.d_lamp));
  const float* Pd = c.F(c.L.Pd);
  const float* Po = c.F(c.L.Po);
  float red2[2] = {0.f, 0.f};
  for (int k = c.tm.lane; k < K; k += TEAM) {
    float rt[NX], gt[NX];
    btmv_row<NX>(Pd, Po, R, k, K, KP, rt);
    btmv_row<NX>(Pd, Po, Y, k, K, KP, gt);
#pragma unroll
    for (int i = 0; i < NX; ++i) {
      Pv[i * KP + k] = rt[i];
      red2[0] = fmaf(R[i * KP + k], rt[i], red2[0]);
      red2[1] = fmaf(Y[i * KP + k], gt[i], red2[1]);
    }
  }
  c.tm.sum(red2);
  if (c.tm.lane == 0) {
    const float tol2 = P.opt.pcg_tol * P.opt.pcg_tol;
    S.eta = red2[0]; S.eta0 = red2[1]; S.eta_ref = red2[0]; S.eta_true = red2[0];
    S.it = 0; S.stall = 0; S.folded = 1;
    S.converged = !(red2[0] > tol2 * red2[1]);
    S.active = !S.converged;
  }
}

template <class M, int TEAM>
__device__ __noinline__ void plain_step(Ctx<M, TEAM>& c, PlainState& S, int step, int s_iter) {
  constexpr int NX = M::NX;
  const KParams& P = *c.P;
  const int K = c.K, KP = c.KP;
  float* R = c.F(c.L.r);
  float* Pv = c.F(c.L.p);
  float* Y = c.F(c.L.y);
  float* DL = c.F(c.L.dl);
  double* LP = c.Dp(c.L.d_lamp);
  const float* D = c.F(c.L.D);
  const float* O = c.F(c.L.O);
  const float* Pd = c.F(c.L.Pd);
  const float* Po = c.F(c.L.Po);
  switch (step) {
    case PS_LOAD: c.status = 0; stage_load<M, TEAM>(c, P.z_init != nullptr); break;
    case PS_LIN:
      stage_linearise<M, TEAM>(c);
      if (c.exact) stage_exact_hessian<M, TEAM>(c);
      break;
    case PS_SCHUR:  // exact-Hessian backward: the Riccati solve replaces a2-a4
      if (c.exact) {
        stage_riccati_exact<M, TEAM>(c);
        // reduced Hessian not positive definite: the Gauss-Newton gradient instead (the later
        // steps see the flag and take the Gauss-Newton path)
        if (c.status & ST_HESS_INDEF) stage_schur<M, TEAM>(c, false);
      } else {
        stage_schur<M, TEAM>(c, P.mode != MODE_VJP);
      }
      break;
    case PS_PREC:
      if (!c.exact) stage_precond<M, TEAM>(c);
      break;
    case PS_PCG_SETUP:
      if (c.exact) {
        if (c.tm.lane == 0) { S.it = 0; S.stall = 0; S.active = 0; S.converged = 1; S.folded = 1; }
      } else {
        plain_pcg_setup<M, TEAM>(c, S);
      }
      break;
    case PS_MATVEC: {  // y = S p   (Algorithm 4, line 6)
      if (!S.active) break;
      for (int k = c.tm.lane; k < K; k += TEAM) {
        float y[NX];
        btmv_row<NX>(D, O, Pv, k, K, KP, y);
#pragma unroll
        for (int i = 0; i < NX; ++i) Y[i * KP + k] = y[i];
      }
      break;
    }
    case PS_AXPY: {  // v = p^T y, alpha, lambda += alpha p, r -= alpha y   (lines 7-10)
      if (!S.active) break;
      float v[1] = {0.f};
      for (int k = c.tm.lane; k < K; k += TEAM)
#pragma unroll
        for (int i = 0; i < NX; ++i) v[0] = fmaf(Pv[i * KP + k], Y[i * KP + k], v[0]);
      c.tm.sum(v);
      if (!(v[0] > 0.f) || !isfinite(v[0])) {
        if (c.tm.lane == 0) S.active = 0;
        break;
      }
      const float alpha = S.eta / v[0];
      for (int k = c.tm.lane; k < K; k += TEAM)
#pragma unroll
        for (int i = 0; i < NX; ++i) {
          DL[i * KP + k] = fmaf(alpha, Pv[i * KP + k], DL[i * KP + k]);
          R[i * KP + k] = fmaf(-alpha, Y[i * KP + k], R[i * KP + k]);
        }
      if (c.tm.lane == 0) S.folded = 0;
      break;
    }
    case PS_PRECAPPLY: {  // r~ = Phi^-1 r   (line 11)
      if (!S.active) break;
      for (int k = c.tm.lane; k < K; k += TEAM) {
        float rt[NX];
        btmv_row<NX>(Pd, Po, R, k, K, KP, rt);
#pragma unroll
        for (int i = 0; i < NX; ++i) Y[i * KP + k] = rt[i];
      }
      break;
    }
    case PS_BETA: {  // eta' = r^T r~, reliable update, beta, p = r~ + beta p   (lines 12-15)
      if (!S.active) break;
      const float tol2 = P.opt.pcg_tol * P.opt.pcg_tol;
      const float dl2 = P.opt.ru_delta * P.opt.ru_delta;
      float e1[1] = {0.f};
      for (int k = c.tm.lane; k < K; k += TEAM)
#pragma unroll
        for (int i = 0; i < NX; ++i) e1[0] = fmaf(R[i * KP + k], Y[i * KP + k], e1[0]);
      c.tm.sum(e1);
      float eta_new = e1[0];
      const int it = S.it + 1;
      bool active = true, converged = false;
      int stall = S.stall;
      float eta_ref = S.eta_ref, eta_true = S.eta_true;
      bool folded = false;
      if (eta_new < dl2 * eta_ref || !(eta_new > tol2 * S.eta0) || it >= P.opt.pcg_max_iters || !isfinite(eta_new)) {
        for (int k = c.tm.lane; k < K; k += TEAM)
#pragma unroll
          for (int i = 0; i < NX; ++i) { LP[i * KP + k] += (double)DL[i * KP + k]; DL[i * KP + k] = 0.f; }
        folded = true;
        hp_residual<M, TEAM>(c, LP);
        float e2[1] = {0.f};
        for (int k = c.tm.lane; k < K; k += TEAM) {
          float rt[NX];
          btmv_row<NX>(Pd, Po, R, k, K, KP, rt);
#pragma unroll
          for (int i = 0; i < NX; ++i) { Y[i * KP + k] = rt[i]; e2[0] = fmaf(R[i * KP + k], rt[i], e2[0]); }
        }
        c.tm.sum(e2);
        eta_new = e2[0];
        eta_ref = eta_new;
        if (!(eta_new > tol2 * S.eta0)) { converged = true; active = false; }
        else if (!isfinite(eta_new)) active = false;
        else {
          if (eta_new > 0.25f * eta_true) { if (++stall >= 2) active = false; }
          else stall = 0;
          eta_true = eta_new;
          if (it >= P.opt.pcg_max_iters) active = false;
        }
      }
      if (active) {
        const float beta = eta_new / S.eta;
        for (int k = c.tm.lane; k < K; k += TEAM)
#pragma unroll
          for (int i = 0; i < NX; ++i) Pv[i * KP + k] = fmaf(beta, Pv[i * KP + k], Y[i * KP + k]);
      }
      c.tm.sync();
      if (c.tm.lane == 0) {
        S.it = it; S.stall = stall; S.eta_ref = eta_ref; S.eta_true = eta_true; S.eta = eta_new;
        S.active = active; S.converged = converged;
        if (folded) S.folded = 1;
      }
      break;
    }
    case PS_PCG_FINISH: {
      int it = S.it;
      if (!S.folded) {
        for (int k = c.tm.lane; k < K; k += TEAM)
#pragma unroll
          for (int i = 0; i < NX; ++i) { LP[i * KP + k] += (double)DL[i * KP + k]; DL[i * KP + k] = 0.f; }
        hp_residual<M, TEAM>(c, LP);
      }
      if (!S.converged) {
        c.status |= ST_FP64_RESCUE;
        it += stage_pcg_df<M, TEAM>(c, S.eta0, P.opt.pcg_max_iters);
      }
      if (c.tm.lane == 0) {
        S.it = it;
        if (P.mode != MODE_VJP && P.pcg_iters) P.pcg_iters[(long long)c.ocp * P.opt.sqp_iters + s_iter] = it;
      }
      break;
    }
    case PS_RECOVER: stage_recover<M, TEAM>(c); break;
    case PS_LS: {
      const float a = stage_linesearch<M, TEAM>(c);
      if (c.tm.lane == 0 && P.alpha_hist) P.alpha_hist[(long long)c.ocp * P.opt.sqp_iters + s_iter] = a;
      break;
    }
    case PS_FWD_OUT: stage_fwd_outputs<M, TEAM>(c); break;
    case PS_BWD_FINISH: stage_bwd_finish<M, TEAM>(c, S.it); break;
    default: break;
  }
}

template <class M, int TEAM>
__device__ void plain_one(const KParams& P, PlainState* st, int ocp, int step, int s_iter) {
  Ctx<M, TEAM> c;
  c.P = &P;
  c.o = P.ocps[ocp];
  c.ocp = ocp;
  c.T = c.o.T;
  c.K = c.o.T + 1;
  c.dt = c.o.dt;
  c.L = make_layout(M::NX, M::NU, c.K, TEAM, P.opt.exact_hessian, is_implicit<M>::value ? 1 : 0);
  c.exact = !is_lq<M>::value && !is_implicit<M>::value && P.opt.exact_hessian && P.mode == MODE_VJP;
  c.KP = c.L.KP;
  float* ws = P.gws + (size_t)ocp * P.ws_floats;
  c.db = reinterpret_cast<double*>(ws);
  c.fb = ws;
  c.tm.lane = threadIdx.x;
  c.tm.bar_id = 1;
  c.tm.red = ws + c.L.red;
  c.tm.buf = 0;
  PlainState& S = st[ocp];
  c.status = S.status;
  c.df_iters = 0;
  if (step != PS_LOAD && (S.status & ST_HESS_INDEF)) c.exact = false;   // Gauss-Newton fallback
  plain_step<M, TEAM>(c, S, step, s_iter);
  c.status = c.tm.bor(c.status);
  if (c.tm.lane == 0) S.status = c.status;
}

// One block = one team = one OCP; one launch = one step for the whole batch.  The parameters
// live in device memory (written once per solve), so one captured graph serves every solve.
template <int TEAM, class... Ms>
__global__ void __launch_bounds__(256, 1) plain_kernel(const KParams* __restrict__ Pp, PlainState* st, int step,
                                                        int s_iter) {
  const KParams& P = *Pp;
  if ((int)blockIdx.x >= P.n_work) return;
  const int ocp = P.order ? P.order[blockIdx.x] : (int)blockIdx.x;
  const OcpRec& o = P.ocps[ocp];
  bool done = ((o.model == Ms::ID && o.nx == Ms::NX && o.nu == Ms::NU
                    ? (plain_one<Ms, TEAM>(P, st, ocp, step, s_iter), true)
                    : false) || ...);
  (void)done;
}

// Last node of a PCG WHILE body: keeps the loop running while any OCP of the work list is
// still iterating (every OCP stops within pcg_max_iters iterations, so the loop ends).
__global__ void plain_pcg_continue(const PlainState* st, const KParams* P, cudaGraphConditionalHandle cond);

}  // namespace dmpc
