// Fused per-OCP SQP iteration and backward pass of DiffMPC (arXiv 2510.06179), one team
// of threads per OCP, all per-knot data resident in the team's workspace (shared memory,
// or a global-memory slot when an OCP does not fit).
//
// Steps per SQP iteration (Algorithm 2):
//   a1 linearise every knot in parallel (Eq. 4; Delta-form linear terms)     FP32
//   a2 Schur blocks chi_t, phi_t (Eq. 10), gamma (App. A.2)                   FP32 / FP64
//   a3 stair preconditioner Phi^-1 = D^-1 - D^-1 O D^-1 (Eq. 10)              FP32
//   a4 PCG (Algorithm 4) on S_spd lambda = gamma_spd                          FP32 inner loop,
//      FP64 solution accumulation with reliable (true-residual) updates
//   a5 primal recovery (Eq. 11)                                               FP64
//   a6 line search over the alpha set (Algorithm 5) and the step              FP32 / FP64
// Backward (Algorithm 3): a1-a3 at the returned z (or stored blocks), adjoint right-hand
// side from (dl/dz, 0) (Eq. 7), the same PCG, z~ (Eq. 11 form), and
// dl/dtheta = -(dF/dtheta)^T [z~; lambda~] (Eq. 3) contracted per knot.
//
// The A array holds A_t + I (see stage_linearise).
// Data layout in the workspace: element e of knot k of an array lives at arr[e * KP + k]
// (knot-minor), so the threads of a warp, which own consecutive knots, touch consecutive
// words.  Thread `lane` of the team owns knots lane, lane + TEAM, ...; knot k holds x_k,
// u_k, lambda_k, Schur block row k, and the linearisation of dynamics step t = k - 1.
#pragma once
#include "device_util.cuh"
#include "dfloat.cuh"
#include "models.cuh"
#include "params.h"

namespace dmpc {

enum StatusBits : int {
  ST_OK = 0, ST_PCG_MAXITER = 1, ST_NONFINITE = 2, ST_LS_MINSTEP = 4, ST_BAD_INPUT = 8,
  ST_PCG_BREAKDOWN = 16, ST_CHOL_FAIL = 32, ST_FP64_RESCUE = 64, ST_HESS_INDEF = 128
};

constexpr int kMisc = 256;      // per-team scalars (theta, cost weights, reciprocals)
constexpr int kRedMax = 48;     // must equal Team<>::RED_MAX

struct Layout {
  int KP;
  int d_lam, d_lamp, d_gam, d_wx, d_wu, d_r, d_p, d_y, d_W, d_total;  // double arrays (in doubles)
  int x, u, xp, up, f, C, A, Bm, Ap, D, O, Pd, Po, r, p, y, dl, misc, red, bnd, f_total;  // floats
  int total_floats;
};

// exact = 1 adds the exact-Hessian backward's per-knot blocks ((nx+nu)^2 doubles per knot: the
// Hessian block, then the Riccati factors) and its scratch; implicit = 1 adds the A^+ blocks of
// an implicit integrator (nx^2 floats per knot).
__host__ __device__ inline Layout make_layout(int nx, int nu, int K, int team, int exact = 0, int implicit = 0) {
  Layout L;
  L.KP = (K + 1) & ~1;
  const int KP = L.KP;
  int o = 0;
  L.d_lam = o; o += nx * KP;
  L.d_lamp = o; o += nx * KP;
  L.d_gam = o; o += nx * KP;
  L.d_wx = o; o += nx * KP;
  L.d_wu = o; o += nu * KP;
  L.d_r = o; o += nx * KP;
  L.d_p = o; o += nx * KP;
  L.d_y = o; o += nx * KP;
  L.d_W = o; o += exact ? (nx + nu) * (nx + nu) * (KP + 2) + 2 * (nx + nu) : 0;
  L.d_total = o;
  int f = 2 * o;  // floats start after the doubles
  L.x = f; f += nx * KP;
  L.u = f; f += nu * KP;
  L.xp = f; f += nx * KP;
  L.up = f; f += nu * KP;
  L.f = f; f += nx * KP;
  L.C = f; f += nx * KP;
  L.A = f; f += nx * nx * KP;
  L.Bm = f; f += nx * nu * KP;
  L.Ap = f; f += implicit ? nx * nx * KP : 0;
  L.D = f; f += nx * nx * KP;
  L.O = f; f += nx * nx * KP;
  L.Pd = f; f += nx * nx * KP;
  L.Po = f; f += nx * nx * KP;
  L.r = f; f += nx * KP;
  L.p = f; f += nx * KP;
  L.y = f; f += nx * KP;
  L.dl = f; f += nx * KP;
  L.misc = f; f += kMisc;
  L.red = f; f += 2 * ((team + 31) / 32) * kRedMax;
  L.bnd = f; f += 2 * 2 * ((team + 31) / 32) * nx;  // warp-boundary exchange, double-buffered
  L.f_total = f;
  L.total_floats = (f + 3) & ~3;
  return L;
}

// misc layout (floats): [0,16) shared params, [16,32) raw Q, [32,48) raw R, [48,64) raw Q_T,
// [64,80) projected Q, [80,96) projected R, [96,112) projected Q_T
constexpr int MS_TH = 0, MS_Q = 16, MS_R = 32, MS_QT = 48, MS_QP = 64, MS_RP = 80, MS_QTP = 96;
constexpr int MS_BAD = 120;  // nonzero when a weight or parameter is not finite
// double reciprocals of the projected weights (float offset 128, 8-byte aligned):
// [0,16) 1/Q, [16,24) 1/R, [24,40) 1/Q_T  (in doubles)
constexpr int MS_DINV = 128;

template <class M>
struct ClRun;

template <class M, int TEAM>
struct Ctx {
  static constexpr int NX = M::NX, NU = M::NU, NZ = M::NX + M::NU;
  Team<TEAM> tm;
  const KParams* P;
  OcpRec o;
  Layout L;
  int K, T, KP, ocp;
  float dt;
  double* db;
  float* fb;
  int status;
  int df_iters;  // PCG iterations of the current solve run in the double-float rescue (inspect output)
  bool exact;  // backward with the exact Hessian of the Lagrangian (Riccati solve), else Gauss-Newton
  ClRun<M>* cl = nullptr;  // set when the OCP runs on a thread-block cluster (its PCG solves are distributed)
  bool cl_form = false;    // the next cluster PCG forms the S and Phi^-1 blocks itself (a2, a3 skipped here)

  __device__ __forceinline__ float* F(int off) const { return fb + off; }
  __device__ __forceinline__ double* Dp(int off) const { return db + off; }
  __device__ __forceinline__ float misc(int i) const { return fb[L.misc + i]; }
  __device__ __forceinline__ float qraw(int k, int i) const { return misc((k < T ? MS_Q : MS_QT) + i); }
  __device__ __forceinline__ float qproj(int k, int i) const { return misc((k < T ? MS_QP : MS_QTP) + i); }
  __device__ __forceinline__ double qinv(int k, int i) const {
    return reinterpret_cast<const double*>(fb + L.misc + MS_DINV)[(k < T ? 0 : 24) + i];
  }
  __device__ __forceinline__ double rinv(int i) const {
    return reinterpret_cast<const double*>(fb + L.misc + MS_DINV)[16 + i];
  }
  // (vx, vu) = G_k^-1 (wx, wu) over the variables (x_k, u_k) of knot k (u only for k < T),
  // G_k = diag(Q_k, R) with the projected weights.
  template <class V>
  __device__ __forceinline__ void ginv(int k, const V (&wx)[NX], const V (&wu)[NU], double (&vx)[NX],
                                       double (&vu)[NU]) const {
#pragma unroll
    for (int i = 0; i < NX; ++i) vx[i] = (double)wx[i] * qinv(k, i);
#pragma unroll
    for (int i = 0; i < NU; ++i) vu[i] = (k < T) ? (double)wu[i] * rinv(i) : 0.0;
  }
  __device__ __forceinline__ float xref(int k, int i) const {
    return P->x_ref ? __ldg(P->x_ref + o.xref_off + (long long)k * NX + i) : 0.f;
  }
  // Delta-form linear cost terms (Eq. 4 read in absolute z): q_k = grad c(x_k) - Q_k x_k,
  // r_k = grad c(u_k) - R u_k, with grad c from the raw weights and Q_k, R projected.
  __device__ __forceinline__ double qlin(int k, int i, float xk) const {
    return (double)qraw(k, i) * ((double)xk - (double)xref(k, i)) - (double)qproj(k, i) * (double)xk;
  }
  __device__ __forceinline__ double rlin(int i, float uk) const {
    return (double)misc(MS_R + i) * (double)uk - (double)misc(MS_RP + i) * (double)uk;
  }
};

// ---------------------------------------------------------------------------------------
// small dense helpers on element-major blocks
template <int NX>
__device__ __forceinline__ float blk(const float* base, int KP, int k, int i, int j) {
  return base[(i * NX + j) * KP + k];
}

// out = Md_k v_k + Mo_k v_{k-1} + Mo_{k+1}^T v_{k+1}  (symmetric block-tridiagonal row k);
// FP32 blocks, vectors and accumulation in V.
template <int NX, class V>
__device__ __forceinline__ void btmv_row(const float* Md, const float* Mo, const V* v, int k, int K,
                                         int KP, V* out) {
  V vc[NX], vm[NX], vp[NX];
#pragma unroll
  for (int j = 0; j < NX; ++j) {
    vc[j] = v[j * KP + k];
    vm[j] = (k > 0) ? v[j * KP + k - 1] : V(0);
    vp[j] = (k + 1 < K) ? v[j * KP + k + 1] : V(0);
  }
#pragma unroll
  for (int i = 0; i < NX; ++i) {
    V acc = V(0);
#pragma unroll
    for (int j = 0; j < NX; ++j) acc = fma((V)Md[(i * NX + j) * KP + k], vc[j], acc);
    if (k > 0) {
#pragma unroll
      for (int j = 0; j < NX; ++j) acc = fma((V)Mo[(i * NX + j) * KP + k], vm[j], acc);
    }
    if (k + 1 < K) {
#pragma unroll
      for (int j = 0; j < NX; ++j) acc = fma((V)Mo[(j * NX + i) * KP + k + 1], vp[j], acc);
    }
    out[i] = acc;
  }
}

// Inverse of an SPD NX x NX block (Cholesky, then L^-T L^-1), in float or double.  Returns
// false if a pivot is not positive (the block is then replaced by the inverse of its diagonal).
template <int NX, class V = float>
__device__ bool spd_inverse(const V* a, V* inv) {
  V L[NX * NX];
#pragma unroll (NX <= 8 ? 32 : 1)
  for (int i = 0; i < NX * NX; ++i) L[i] = V(0);
  bool ok = true;
#pragma unroll (NX <= 8 ? 32 : 1)
  for (int j = 0; j < NX; ++j) {
    V s = a[j * NX + j];
#pragma unroll (NX <= 8 ? 32 : 1)
    for (int k = 0; k < j; ++k) s -= L[j * NX + k] * L[j * NX + k];
    if (!(s > V(0))) { ok = false; s = fabs(a[j * NX + j]) + V(1e-30); }
    const V d = sqrt(s);
    L[j * NX + j] = d;
    const V id = V(1) / d;
#pragma unroll (NX <= 8 ? 32 : 1)
    for (int i = j + 1; i < NX; ++i) {
      V t = a[i * NX + j];
#pragma unroll (NX <= 8 ? 32 : 1)
      for (int k = 0; k < j; ++k) t -= L[i * NX + k] * L[j * NX + k];
      L[i * NX + j] = t * id;
    }
  }
  if (!ok) {
#pragma unroll (NX <= 8 ? 32 : 1)
    for (int i = 0; i < NX * NX; ++i) inv[i] = V(0);
#pragma unroll (NX <= 8 ? 32 : 1)
    for (int i = 0; i < NX; ++i) inv[i * NX + i] = V(1) / (fabs(a[i * NX + i]) + V(1e-30));
    return false;
  }
  // W = L^-1 (lower triangular), forward substitution column by column
  V W[NX * NX];
#pragma unroll (NX <= 8 ? 32 : 1)
  for (int i = 0; i < NX * NX; ++i) W[i] = V(0);
#pragma unroll (NX <= 8 ? 32 : 1)
  for (int c = 0; c < NX; ++c) {
#pragma unroll (NX <= 8 ? 32 : 1)
    for (int i = c; i < NX; ++i) {
      V t = (i == c) ? V(1) : V(0);
#pragma unroll (NX <= 8 ? 32 : 1)
      for (int k = c; k < i; ++k) t -= L[i * NX + k] * W[k * NX + c];
      W[i * NX + c] = t / L[i * NX + i];
    }
  }
  // inv = W^T W
#pragma unroll (NX <= 8 ? 32 : 1)
  for (int i = 0; i < NX; ++i) {
#pragma unroll (NX <= 8 ? 32 : 1)
    for (int j = 0; j <= i; ++j) {
      V s = V(0);
#pragma unroll (NX <= 8 ? 32 : 1)
      for (int k = (i > j ? i : j); k < NX; ++k) s += W[k * NX + i] * W[k * NX + j];
      inv[i * NX + j] = s;
      inv[j * NX + i] = s;
    }
  }
  return true;
}

// ---------------------------------------------------------------------------------------
// Load per-OCP scalars and the initial iterate.
template <class M, int TEAM>
__device__ __noinline__ void stage_load(Ctx<M, TEAM>& c, bool use_z_init) {
  constexpr int NX = M::NX, NU = M::NU, NZ = NX + NU;
  const KParams& P = *c.P;
  const int T = c.T, K = c.K, KP = c.KP;
  const float* th = P.theta + c.o.th_off;
  int pk = 0;
  if constexpr (is_lq<M>::value) pk = M::PK;
  const int oq = M::NP + T * pk;
  if (c.tm.lane == 0) {
    float* ms = c.F(c.L.misc);
    for (int i = 0; i < M::NP; ++i) ms[MS_TH + i] = th[i];
    float qm = 0.f, rm = 0.f, qtm = 0.f;
    for (int i = 0; i < NX; ++i) { ms[MS_Q + i] = th[oq + i]; qm = fmaxf(qm, th[oq + i]); }
    for (int i = 0; i < NU; ++i) { ms[MS_R + i] = th[oq + NX + i]; rm = fmaxf(rm, th[oq + NX + i]); }
    for (int i = 0; i < NX; ++i) { ms[MS_QT + i] = th[oq + NX + NU + i]; qtm = fmaxf(qtm, th[oq + NX + NU + i]); }
    // PD projection of the diagonal Hessians (Sec. 3.1): clamp at 1e-6 max(1, largest entry)
    float fq = 1e-6f * fmaxf(1.f, qm), fr = 1e-6f * fmaxf(1.f, rm), fqt = 1e-6f * fmaxf(1.f, qtm);
    int bad = 0;
    for (int i = 0; i < NX; ++i) { ms[MS_QP + i] = fmaxf(ms[MS_Q + i], fq); bad |= !isfinite(ms[MS_Q + i]); }
    for (int i = 0; i < NU; ++i) { ms[MS_RP + i] = fmaxf(ms[MS_R + i], fr); bad |= !isfinite(ms[MS_R + i]); }
    for (int i = 0; i < NX; ++i) { ms[MS_QTP + i] = fmaxf(ms[MS_QT + i], fqt); bad |= !isfinite(ms[MS_QT + i]); }
    for (int i = 0; i < M::NP; ++i) bad |= !isfinite(ms[MS_TH + i]);
    ms[MS_BAD] = bad ? 1.f : 0.f;
    double* dinv = reinterpret_cast<double*>(ms + MS_DINV);
    for (int i = 0; i < NX; ++i) { dinv[i] = 1.0 / (double)ms[MS_QP + i]; dinv[24 + i] = 1.0 / (double)ms[MS_QTP + i]; }
    for (int i = 0; i < NU; ++i) dinv[16 + i] = 1.0 / (double)ms[MS_RP + i];
  }
  const float* xs = P.x_s + c.o.xs_off;
  if (P.mode == MODE_SOLVE && P.res_th) {
    // keep the inputs of this solve on the device for the backward pass
    const int p = c.o.p;
    for (int i = c.tm.lane; i < p; i += TEAM) P.res_th[c.o.th_off + i] = th[i];
    for (int i = c.tm.lane; i < NX; i += TEAM) P.res_xs[c.o.xs_off + i] = xs[i];
    if (P.x_ref)
      for (int i = c.tm.lane; i < K * NX; i += TEAM) P.res_xref[c.o.xref_off + i] = P.x_ref[c.o.xref_off + i];
  }
  float* X = c.F(c.L.x);
  float* U = c.F(c.L.u);
  double* LAM = c.Dp(c.L.d_lam);
  // a slot re-assigned to a new problem starts cold (its resident iterate belongs to the old one)
  const bool cold = P.cold != nullptr && P.cold[c.ocp] != 0 && P.mode == MODE_SOLVE;
  const float* zi = (use_z_init && !cold) ? P.z_init : nullptr;
  for (int k = c.tm.lane; k < K; k += TEAM) {
    const long long zb = c.o.z_off + (long long)k * NZ;
#pragma unroll
    for (int i = 0; i < NX; ++i) X[i * KP + k] = zi ? zi[zb + i] : xs[i];
    if (k < T) {
#pragma unroll
      for (int i = 0; i < NU; ++i) U[i * KP + k] = zi ? zi[zb + NX + i] : 0.f;
    }
    const long long lb = c.o.lam_off + (long long)k * NX;
#pragma unroll
    for (int i = 0; i < NX; ++i) {
      double v = 0.0;
      if (P.mode != MODE_VJP) {
        if (cold) v = 0.0;
        else if (P.lam_init_d) v = P.lam_init_d[lb + i];
        else if (P.lam_init_f) v = (double)P.lam_init_f[lb + i];
      } else {
        v = P.lam_init_d ? P.lam_init_d[lb + i] : (P.lam_init_f ? (double)P.lam_init_f[lb + i] : 0.0);
      }
      LAM[i * KP + k] = v;
    }
  }
  c.tm.sync();
  if (cold && c.tm.lane == 0) P.cold[c.ocp] = 0;
  if (c.misc(MS_BAD) != 0.f) c.status |= ST_BAD_INPUT;
}

// a1: linearise dynamics step t = k-1 at knot slot k (FP32): A_t, B_t, C_t, f_t; f_0 = x_0 - x_s.
// The A array holds A_t + I, not A_t: for an integrator step A_t = -dPhi/dx = -I - d(Phi - x)/dx, and
// in FP32 the identity would round away most of the step's own Jacobian (about dt times the
// dynamics' derivatives), which sets the QP solution's precision; every consumer subtracts the
// identity in its own precision (exactly in the FP64 and double-float operators).  C_t and f_t
// are formed from the increment Phi - x, so no term of the size of the state cancels.
template <class M, int TEAM>
__device__ __noinline__ void stage_linearise(Ctx<M, TEAM>& c) {
  constexpr int NX = M::NX, NU = M::NU, NZ = NX + NU;
  const KParams& P = *c.P;
  const int T = c.T, K = c.K, KP = c.KP;
  const float* X = c.F(c.L.x);
  const float* U = c.F(c.L.u);
  float* A = c.F(c.L.A);
  float* Bm = c.F(c.L.Bm);
  float* C = c.F(c.L.C);
  float* Fv = c.F(c.L.f);
  const float* xs = P.x_s + c.o.xs_off;
  for (int k = c.tm.lane; k < K; k += TEAM) {
    if (k == 0) {
#pragma unroll
      for (int i = 0; i < NX; ++i) Fv[i * KP] = X[i * KP] - xs[i];
      continue;
    }
    const int t = k - 1;
    float xt[NX], ut[NU];
#pragma unroll
    for (int i = 0; i < NX; ++i) xt[i] = X[i * KP + t];
#pragma unroll
    for (int i = 0; i < NU; ++i) ut[i] = U[i * KP + t];
    float phi[NX], fres[NX];
    if constexpr (is_lq<M>::value) {
      const float* tk = P.theta + c.o.th_off + (long long)t * M::PK;
#pragma unroll
      for (int i = 0; i < NX; ++i) {
        float acc = tk[NX * NX + NX * NU + i];
#pragma unroll
        for (int j = 0; j < NX; ++j) {
          float a = tk[i * NX + j];
          acc = fmaf(a, xt[j], acc);
          A[(i * NX + j) * KP + k] = (i == j ? 1.f : 0.f) - a;   // A_t + I = I - Abar_t (exact)
        }
#pragma unroll
        for (int j = 0; j < NU; ++j) {
          float b = tk[NX * NX + i * NU + j];
          acc = fmaf(b, ut[j], acc);
          Bm[(i * NU + j) * KP + k] = -b;
        }
        phi[i] = acc;
        C[i * KP + k] = tk[NX * NX + NX * NU + i];
      }
#pragma unroll
      for (int i = 0; i < NX; ++i) fres[i] = X[i * KP + k] - phi[i];
    } else if constexpr (is_implicit<M>::value) {
      // trapezoidal rule: f = x_{t+1} - x_t - dt/2 (F(x_t, u_t) + F(x_{t+1}, u_t)), so
      // A = -I - dt/2 F_x(x_t), B = -dt/2 (F_u(x_t) + F_u(x_{t+1})), A^+ = I - dt/2 F_x(x_{t+1})
      float* Ap = c.F(c.L.Ap);
      constexpr int CH = NZ <= 8 ? NZ : 8;
      float pv[M::NP];
#pragma unroll
      for (int j = 0; j < M::NP; ++j) pv[j] = c.misc(MS_TH + j);
      float xn[NX], fsum[NX], ja[NX * NZ], jb[NX * NZ];
#pragma unroll
      for (int i = 0; i < NX; ++i) xn[i] = X[i * KP + k];
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const float* xe = side == 0 ? xt : xn;
        float* jac = side == 0 ? ja : jb;
#pragma unroll
        for (int c0 = 0; c0 < NZ; c0 += CH) {
          Dual<CH> xd[NX], ud[NU], pd[M::NP], out[NX];
#pragma unroll
          for (int i = 0; i < NX; ++i) xd[i] = Dual<CH>::seed(xe[i], i - c0);
#pragma unroll
          for (int i = 0; i < NU; ++i) ud[i] = Dual<CH>::seed(ut[i], NX + i - c0);
#pragma unroll
          for (int j = 0; j < M::NP; ++j) pd[j] = Dual<CH>(pv[j]);
          M::f(xd, ud, pd, out);
#pragma unroll
          for (int i = 0; i < NX; ++i) {
            if (c0 == 0) fsum[i] = (side == 0 ? 0.f : fsum[i]) + out[i].v;
#pragma unroll
            for (int q = 0; q < CH; ++q)
              if (c0 + q < NZ) jac[i * NZ + c0 + q] = out[i].d[q];
          }
        }
      }
      const float h = 0.5f * c.dt;
#pragma unroll
      for (int i = 0; i < NX; ++i) {
        // C = A^+ x_{t+1} + A x_t + B u_t - f with A = -I + E, A^+ = I + E^+ and
        // f = x_{t+1} - x_t - h (F_a + F_b):  C = E x_t + E^+ x_{t+1} + B u_t + h (F_a + F_b)
        float acc = h * fsum[i];
#pragma unroll
        for (int j = 0; j < NX; ++j) {
          const float e = -h * ja[i * NZ + j];     // A + I
          const float ep = -h * jb[i * NZ + j];    // A^+ - I
          A[(i * NX + j) * KP + k] = e;
          Ap[(i * NX + j) * KP + k] = (i == j ? 1.f : 0.f) + ep;
          acc = fmaf(e, xt[j], fmaf(ep, xn[j], acc));
        }
#pragma unroll
        for (int j = 0; j < NU; ++j) {
          const float b = -h * (ja[i * NZ + NX + j] + jb[i * NZ + NX + j]);
          Bm[(i * NU + j) * KP + k] = b;
          acc = fmaf(b, ut[j], acc);
        }
        C[i * KP + k] = acc;
        fres[i] = (xn[i] - xt[i]) - h * fsum[i];
      }
    } else {
      constexpr int CH = NZ <= 8 ? NZ : 8;
      float pv[M::NP];
#pragma unroll
      for (int j = 0; j < M::NP; ++j) pv[j] = c.misc(MS_TH + j);
      float cacc[NX];
#pragma unroll
      for (int i = 0; i < NX; ++i) cacc[i] = 0.f;
#pragma unroll
      for (int c0 = 0; c0 < NZ; c0 += CH) {
        Dual<CH> xd[NX], ud[NU], pd[M::NP], out[NX];
#pragma unroll
        for (int i = 0; i < NX; ++i) xd[i] = Dual<CH>::seed(xt[i], i - c0);
#pragma unroll
        for (int i = 0; i < NU; ++i) ud[i] = Dual<CH>::seed(ut[i], NX + i - c0);
#pragma unroll
        for (int j = 0; j < M::NP; ++j) pd[j] = Dual<CH>(pv[j]);
        model_increment<M>(xd, ud, pd, c.dt, out);   // d = Phi - x and its derivatives
#pragma unroll
        for (int i = 0; i < NX; ++i) {
          phi[i] = out[i].v;
#pragma unroll
          for (int q = 0; q < CH; ++q) {
            const int col = c0 + q;
            if (col < NZ) {
              const float jv = out[i].d[q];
              if (col < NX) {
                A[(i * NX + col) * KP + k] = -jv;    // A_t + I = -dd/dx
                cacc[i] = fmaf(jv, xt[col], cacc[i]);
              } else {
                Bm[(i * NU + (col - NX)) * KP + k] = -jv;
                cacc[i] = fmaf(jv, ut[col - NX], cacc[i]);
              }
            }
          }
        }
      }
      // C_t = A^+ x_{t+1} + A_t x_t + B_t u_t - f_t = Phi - J_x x_t - J_u u_t = d - (dd/dx) x_t - (dd/du) u_t,
      // f_t = x_{t+1} - Phi = (x_{t+1} - x_t) - d
#pragma unroll
      for (int i = 0; i < NX; ++i) {
        C[i * KP + k] = phi[i] - cacc[i];
        fres[i] = (X[i * KP + k] - xt[i]) - phi[i];
      }
    }
#pragma unroll
    for (int i = 0; i < NX; ++i) Fv[i * KP + k] = fres[i];
  }
  c.tm.sync();
}

// Backward with the exact Hessian of the Lagrangian (Sec. 3.4 contrasts it with the Gauss-
// Newton matrix the method uses): per knot k < T the block of grad^2_zz L over (x_k, u_k) is
//   G_k = diag(Q_k, R) - sum_i lambda_{k+1,i} grad^2 Phi_{k,i}(x_k, u_k)   (f_k = x_{k+1} - Phi_k),
// second derivatives of the integrator step from hyper-dual numbers (one model evaluation per
// pair of seed directions), lambda from the forward solve; G_T = diag(Q_T).  Stored in FP64
// at W[(a * NZ + b) * KP + k].
template <class M, int TEAM>
__device__ __noinline__ void stage_exact_hessian(Ctx<M, TEAM>& c) {
  constexpr int NX = M::NX, NU = M::NU, NZ = NX + NU, NP = M::NP;
  const int T = c.T, KP = c.KP;
  const float* X = c.F(c.L.x);
  const float* U = c.F(c.L.u);
  const double* LAM = c.Dp(c.L.d_lam);
  double* W = c.Dp(c.L.d_W);
  if constexpr (!is_lq<M>::value && !is_implicit<M>::value)  // exact mode is off for these
  for (int k = c.tm.lane; k < T; k += TEAM) {
    float lam1[NX];
#pragma unroll
    for (int i = 0; i < NX; ++i) lam1[i] = (float)LAM[i * KP + k + 1];
#pragma unroll 1
    for (int a = 0; a < NZ; ++a) {
#pragma unroll 1
      for (int b = 0; b <= a; ++b) {
        HDual<1> xh[NX], uh[NU], ph[NP > 0 ? NP : 1], out[NX];
#pragma unroll
        for (int i = 0; i < NX; ++i) {
          xh[i] = HDual<1>(X[i * KP + k]);
          xh[i].e = (i == a) ? 1.f : 0.f;
          xh[i].t[0] = (i == b) ? 1.f : 0.f;
        }
#pragma unroll
        for (int i = 0; i < NU; ++i) {
          uh[i] = HDual<1>(U[i * KP + k]);
          uh[i].e = (NX + i == a) ? 1.f : 0.f;
          uh[i].t[0] = (NX + i == b) ? 1.f : 0.f;
        }
#pragma unroll
        for (int j = 0; j < NP; ++j) ph[j] = HDual<1>(c.misc(MS_TH + j));
        model_step<M>(xh, uh, ph, c.dt, out);
        double h = 0.0;
#pragma unroll
        for (int i = 0; i < NX; ++i) h += (double)lam1[i] * (double)out[i].et[0];
        double g = -h;
        if (a == b) g += (a < NX) ? (double)c.qproj(k, a) : (double)c.misc(MS_RP + a - NX);
        W[(a * NZ + b) * KP + k] = g;
        W[(b * NZ + a) * KP + k] = g;
      }
    }
  }
  c.tm.sync();
}

// The exact-Hessian backward KKT system [G H^T; H 0] [z~; lambda~] = [dl/dz; 0] (Eq. 7 with the
// full G) solved by the discrete-time Riccati recursion in FP64: the per-knot blocks G_k of the
// Lagrangian Hessian are indefinite for most OCPs away from the pure cost, so H G^-1 H^T is not
// positive definite and PCG does not apply; the recursion needs only the reduced Hessian to be
// positive definite (second-order sufficiency at the forward solution).  With the constraint
// rows x~_{k+1} + A_k x~_k + B_k u~_k = 0, x~_0 = 0 and g = dl/dz:
//   backward  P_T = G_T, s_T = -g_T;   for k = T-1..0 with Ab = -A_k, Bb = -B_k:
//     Qxx = G_xx + Ab^T P Ab, Quu = G_uu + Bb^T P Bb, Qux = G_ux + Bb^T P Ab,
//     qx = -g_x + Ab^T s, qu = -g_u + Bb^T s,  K = -Quu^-1 Qux, k = -Quu^-1 qu,
//     P_k = Qxx + Qux^T K, s_k = qx + Qux^T k;
//   forward   u~_k = K x~_k + k, x~_{k+1} = Ab x~_k + Bb u~_k, lambda~_k = -(P_k x~_k + s_k).
// Knot slot k of W (after its G_k is consumed) holds [P_k | s_k | K_k | k_k].  Writes z~ to
// (xp, up) and lambda~ to lamp.  A Quu that is not positive definite sets ST_HESS_INDEF.
template <class M, int TEAM>
__device__ __noinline__ void stage_riccati_exact(Ctx<M, TEAM>& c) {
  constexpr int NX = M::NX, NU = M::NU, NZ = NX + NU;
  constexpr int OP = 0, OS = NX * NX, OK = OS + NX, Ok = OK + NU * NX;  // slot offsets
  const KParams& P = *c.P;
  const int T = c.T, KP = c.KP;
  const float* g = P.dl_dz + c.o.z_off;
  const float* A = c.F(c.L.A);
  const float* Bm = c.F(c.L.Bm);
  double* W = c.Dp(c.L.d_W);
  double* Q = W + (size_t)NZ * NZ * KP;   // scratch: Q block (NZ x NZ, rows x then u)
  double* q = Q + NZ * NZ;                // scratch: q (NZ)
  double* F = q + NZ;                     // scratch: [K | k] (NU x (NX + 1)), then P_k, s_k
  double* LP = c.Dp(c.L.d_lamp);
  float* XT = c.F(c.L.xp);
  float* UT = c.F(c.L.up);
  const int ln = c.tm.lane;
  auto slot = [&](int e, int k) -> double& { return W[e * KP + k]; };
  // entry (i, j) of A_k (dynamics step k, knot slot k + 1) from the stored A_k + I
  auto a_true = [&](int i, int j, int kn) -> double { return (double)A[(i * NX + j) * KP + kn] - (i == j ? 1.0 : 0.0); };
  // P_T, s_T (slot T)
  for (int e = ln; e < NX * NX; e += TEAM) {
    const int i = e / NX, j = e % NX;
    slot(OP + e, T) = (i == j) ? (double)c.qproj(T, i) : 0.0;
  }
  for (int i = ln; i < NX; i += TEAM) slot(OS + i, T) = -(double)g[(long long)T * NZ + i];
  c.tm.sync();
  for (int k = T - 1; k >= 0; --k) {
    const int kn = k + 1;  // dynamics step k lives at knot slot k + 1: A_k = A[.., k + 1]
    // Q = G_k + [Ab Bb]^T P_{k+1} [Ab Bb], q = -g_k + [Ab Bb]^T s_{k+1}
    for (int e = ln; e < NZ * NZ; e += TEAM) {
      const int a = e / NZ, b = e % NZ;
      double acc = W[e * KP + k];
      for (int i = 0; i < NX; ++i) {
        const double mi = -(a < NX ? a_true(i, a, kn) : (double)Bm[(i * NU + a - NX) * KP + kn]);
        double pj = 0.0;
        for (int j = 0; j < NX; ++j) {
          const double mj = -(b < NX ? a_true(j, b, kn) : (double)Bm[(j * NU + b - NX) * KP + kn]);
          pj += slot(OP + i * NX + j, kn) * mj;
        }
        acc += mi * pj;
      }
      Q[e] = acc;
    }
    for (int a = ln; a < NZ; a += TEAM) {
      double acc = -(double)g[(long long)k * NZ + a];
      for (int i = 0; i < NX; ++i)
        acc += -(a < NX ? a_true(i, a, kn) : (double)Bm[(i * NU + a - NX) * KP + kn]) * slot(OS + i, kn);
      q[a] = acc;
    }
    c.tm.sync();
    // [K | k] = -Quu^-1 [Qux | qu]  (one thread: NU <= 4)
    if (ln == 0) {
      double quu[NU * NU], qi[NU * NU];
#pragma unroll
      for (int a = 0; a < NU; ++a)
#pragma unroll
        for (int b = 0; b < NU; ++b) quu[a * NU + b] = Q[(NX + a) * NZ + NX + b];
      if (!spd_inverse<NU, double>(quu, qi)) c.status |= ST_HESS_INDEF;
      for (int a = 0; a < NU; ++a) {
        for (int j = 0; j <= NX; ++j) {
          double acc = 0.0;
          for (int b = 0; b < NU; ++b) acc += qi[a * NU + b] * (j < NX ? Q[(NX + b) * NZ + j] : q[NX + b]);
          F[a * (NX + 1) + j] = -acc;
        }
      }
    }
    c.tm.sync();
    // P_k = Qxx + Qux^T K, s_k = qx + Qux^T k  (into scratch, then into slot k over G_k)
    double* Pn = F + NU * (NX + 1);
    for (int e = ln; e < NX * NX + NX; e += TEAM) {
      const int i = e / NX, j = e % NX;
      double acc;
      if (e < NX * NX) {
        acc = 0.5 * (Q[i * NZ + j] + Q[j * NZ + i]);
        for (int a = 0; a < NU; ++a)
          acc += 0.5 * (Q[(NX + a) * NZ + i] * F[a * (NX + 1) + j] + Q[(NX + a) * NZ + j] * F[a * (NX + 1) + i]);
      } else {
        const int r = e - NX * NX;
        acc = q[r];
        for (int a = 0; a < NU; ++a) acc += Q[(NX + a) * NZ + r] * F[a * (NX + 1) + NX];
      }
      Pn[e] = acc;
    }
    c.tm.sync();
    for (int e = ln; e < NX * NX + NX; e += TEAM) slot(OP + e, k) = Pn[e];  // OS = NX * NX follows OP
    for (int e = ln; e < NU * (NX + 1); e += TEAM) {
      const int a = e / (NX + 1), j = e % (NX + 1);
      if (j < NX) slot(OK + a * NX + j, k) = F[e];
      else slot(Ok + a, k) = F[e];
    }
    c.tm.sync();
  }
  // forward: x~_0 = 0 (one thread; O(T nz^2))
  if (ln == 0) {
    double x[NX], xn[NX], u[NU];
#pragma unroll
    for (int i = 0; i < NX; ++i) x[i] = 0.0;
    for (int k = 0; k <= T; ++k) {
#pragma unroll
      for (int i = 0; i < NX; ++i) {
        double acc = slot(OS + i, k);
#pragma unroll
        for (int j = 0; j < NX; ++j) acc += slot(OP + i * NX + j, k) * x[j];
        LP[i * KP + k] = -acc;
        XT[i * KP + k] = (float)x[i];
      }
      if (k == T) break;
#pragma unroll
      for (int a = 0; a < NU; ++a) {
        double acc = slot(Ok + a, k);
#pragma unroll
        for (int j = 0; j < NX; ++j) acc += slot(OK + a * NX + j, k) * x[j];
        u[a] = acc;
        UT[a * KP + k] = (float)acc;
      }
#pragma unroll
      for (int i = 0; i < NX; ++i) {
        double acc = 0.0;
#pragma unroll
        for (int j = 0; j < NX; ++j) acc -= a_true(i, j, k + 1) * x[j];
#pragma unroll
        for (int a = 0; a < NU; ++a) acc -= (double)Bm[(i * NU + a) * KP + k + 1] * u[a];
        xn[i] = acc;
      }
#pragma unroll
      for (int i = 0; i < NX; ++i) x[i] = xn[i];
    }
  }
  c.status = c.tm.bor(c.status);
  c.tm.sync();
}

// a2: Schur blocks of S_spd = H G^-1 H^T (Eq. 10) in FP32:  D_0 = Q_0^-1,
// D_k = chi_{k-1} = A Q_{k-1}^-1 A^T + B R^-1 B^T + Q_k^-1,  O_k = phi_{k-1} = A Q_{k-1}^-1.
// With rhs_from_qp, also gamma_spd = -(d + H G^-1 b) (App. A.2) in FP64.
template <class M, int TEAM>
// blocks = false: gamma only (the blocks are formed by the cluster PCG).
__device__ __noinline__ void stage_schur(Ctx<M, TEAM>& c, bool rhs_from_qp, bool blocks = true) {
  constexpr int NX = M::NX, NU = M::NU;
  const KParams& P = *c.P;
  const int T = c.T, K = c.K, KP = c.KP;
  const float* A = c.F(c.L.A);
  const float* Bm = c.F(c.L.Bm);
  const float* C = c.F(c.L.C);
  const float* X = c.F(c.L.x);
  const float* U = c.F(c.L.u);
  float* D = c.F(c.L.D);
  float* O = c.F(c.L.O);
  double* G = c.Dp(c.L.d_gam);
  const float* xs = P.x_s + c.o.xs_off;
  for (int k = c.tm.lane; k < K; k += TEAM) {
    float qi[NX];
#pragma unroll (NX <= 8 ? 32 : 1)
    for (int i = 0; i < NX; ++i) qi[i] = 1.f / c.qproj(k, i);
    if (k == 0) {
      if (blocks) {
#pragma unroll (NX <= 8 ? 32 : 1)
        for (int i = 0; i < NX; ++i)
#pragma unroll (NX <= 8 ? 32 : 1)
          for (int j = 0; j < NX; ++j) D[(i * NX + j) * KP] = (i == j) ? qi[i] : 0.f;
      }
      if (rhs_from_qp) {
#pragma unroll (NX <= 8 ? 32 : 1)
        for (int i = 0; i < NX; ++i)
          G[i * KP] = -(double)xs[i] - c.qlin(0, i, X[i * KP]) * c.qinv(0, i);
      }
      continue;
    }
    const int t = k - 1;
    if constexpr (is_implicit<M>::value) {
      // general A^+ (Eq. 10): D_k = A Q_t^-1 A^T + B R^-1 B^T + A^+_k Q_k^-1 A^+_k^T,
      // O_k = A_k Q_t^-1 (A^+_{k-1})^T (A^+_0 = I: row 0 is x_0 - x_s)
      const float* Ap = c.F(c.L.Ap);
      float qt[NX], ri[NU];
#pragma unroll
      for (int i = 0; i < NX; ++i) qt[i] = 1.f / c.qproj(t, i);
#pragma unroll
      for (int i = 0; i < NU; ++i) ri[i] = 1.f / c.misc(MS_RP + i);
#pragma unroll
      for (int i = 0; i < NX; ++i) {
#pragma unroll
        for (int j = 0; j <= i; ++j) {
          float sum = 0.f;
#pragma unroll
          for (int l = 0; l < NX; ++l) {
            const float ail = A[(i * NX + l) * KP + k] - (i == l ? 1.f : 0.f);
            const float ajl = A[(j * NX + l) * KP + k] - (j == l ? 1.f : 0.f);
            sum = fmaf(ail * qt[l], ajl, sum);
            sum = fmaf(Ap[(i * NX + l) * KP + k] * qi[l], Ap[(j * NX + l) * KP + k], sum);
          }
#pragma unroll
          for (int l = 0; l < NU; ++l) sum = fmaf(Bm[(i * NU + l) * KP + k] * ri[l], Bm[(j * NU + l) * KP + k], sum);
          D[(i * NX + j) * KP + k] = sum;
          D[(j * NX + i) * KP + k] = sum;
        }
#pragma unroll
        for (int j = 0; j < NX; ++j) {
          float sum = 0.f;
#pragma unroll
          for (int l = 0; l < NX; ++l) {
            const float apv = (t == 0) ? (j == l ? 1.f : 0.f) : Ap[(j * NX + l) * KP + t];
            sum = fmaf((A[(i * NX + l) * KP + k] - (i == l ? 1.f : 0.f)) * qt[l], apv, sum);
          }
          O[(i * NX + j) * KP + k] = sum;
        }
      }
      if (rhs_from_qp) {
        double vq[NX], vk[NX], vr[NU];
#pragma unroll
        for (int j = 0; j < NX; ++j) {
          vq[j] = c.qlin(t, j, X[j * KP + t]) * c.qinv(t, j);
          vk[j] = c.qlin(k, j, X[j * KP + k]) * c.qinv(k, j);
        }
#pragma unroll
        for (int j = 0; j < NU; ++j) vr[j] = c.rlin(j, U[j * KP + t]) * c.rinv(j);
#pragma unroll
        for (int i = 0; i < NX; ++i) {
          double z = 0.0;
#pragma unroll
          for (int j = 0; j < NX; ++j)
            z += ((double)A[(i * NX + j) * KP + k] - (i == j ? 1.0 : 0.0)) * vq[j] +
                 (double)Ap[(i * NX + j) * KP + k] * vk[j];
#pragma unroll
          for (int j = 0; j < NU; ++j) z += (double)Bm[(i * NU + j) * KP + k] * vr[j];
          G[i * KP + k] = -(double)C[i * KP + k] - z;
        }
      }
      continue;
    }
    float qt[NX], ri[NU];
#pragma unroll (NX <= 8 ? 32 : 1)
    for (int i = 0; i < NX; ++i) qt[i] = 1.f / c.qproj(t, i);
#pragma unroll (NX <= 8 ? 32 : 1)
    for (int i = 0; i < NU; ++i) ri[i] = 1.f / c.misc(MS_RP + i);
    float a[NX * NX], b[NX * NU];   // a: A_t in FP32 (the stored A_t + I minus the identity)
#pragma unroll (NX <= 8 ? 32 : 1)
    for (int i = 0; i < NX * NX; ++i) a[i] = A[i * KP + k] - ((i / NX) == (i % NX) ? 1.f : 0.f);
#pragma unroll (NX <= 8 ? 32 : 1)
    for (int i = 0; i < NX * NU; ++i) b[i] = Bm[i * KP + k];
#pragma unroll (NX <= 8 ? 32 : 1)
    for (int i = 0; i < NX && blocks; ++i) {
#pragma unroll (NX <= 8 ? 32 : 1)
      for (int j = 0; j <= i; ++j) {
        float s = (i == j) ? qi[i] : 0.f;
#pragma unroll (NX <= 8 ? 32 : 1)
        for (int l = 0; l < NX; ++l) s = fmaf(a[i * NX + l] * qt[l], a[j * NX + l], s);
#pragma unroll (NX <= 8 ? 32 : 1)
        for (int l = 0; l < NU; ++l) s = fmaf(b[i * NU + l] * ri[l], b[j * NU + l], s);
        D[(i * NX + j) * KP + k] = s;
        D[(j * NX + i) * KP + k] = s;
      }
#pragma unroll (NX <= 8 ? 32 : 1)
      for (int j = 0; j < NX; ++j) O[(i * NX + j) * KP + k] = a[i * NX + j] * qt[j];
    }
    if (rhs_from_qp) {
      double vq[NX], vr[NU];
#pragma unroll (NX <= 8 ? 32 : 1)
      for (int j = 0; j < NX; ++j) vq[j] = c.qlin(t, j, X[j * KP + t]) * c.qinv(t, j);
#pragma unroll (NX <= 8 ? 32 : 1)
      for (int j = 0; j < NU; ++j) vr[j] = c.rlin(j, U[j * KP + t]) * c.rinv(j);
#pragma unroll (NX <= 8 ? 32 : 1)
      for (int i = 0; i < NX; ++i) {
        double z = c.qlin(k, i, X[i * KP + k]) * c.qinv(k, i) - vq[i];
#pragma unroll (NX <= 8 ? 32 : 1)
        for (int j = 0; j < NX; ++j) z += (double)A[(i * NX + j) * KP + k] * vq[j];   // exact A_t + I
#pragma unroll (NX <= 8 ? 32 : 1)
        for (int j = 0; j < NU; ++j) z += (double)b[i * NU + j] * vr[j];
        G[i * KP + k] = -(double)C[i * KP + k] - z;
      }
    }
  }
  c.tm.sync();
}

// a3: Phi^-1 blocks (FP32): Pd_k = D_k^-1, Po_k = -D_k^-1 O_k D_{k-1}^-1 (Eq. 10).
template <class M, int TEAM>
__device__ __noinline__ void stage_precond(Ctx<M, TEAM>& c) {
  constexpr int NX = M::NX;
  const int K = c.K, KP = c.KP;
  const float* D = c.F(c.L.D);
  const float* O = c.F(c.L.O);
  float* Pd = c.F(c.L.Pd);
  float* Po = c.F(c.L.Po);
  for (int k = c.tm.lane; k < K; k += TEAM) {
    float a[NX * NX], inv[NX * NX];
#pragma unroll (NX <= 8 ? 32 : 1)
    for (int i = 0; i < NX * NX; ++i) a[i] = D[i * KP + k];
    if (!spd_inverse<NX>(a, inv)) c.status |= ST_CHOL_FAIL;
#pragma unroll (NX <= 8 ? 32 : 1)
    for (int i = 0; i < NX * NX; ++i) Pd[i * KP + k] = inv[i];
  }
  c.tm.sync();
  for (int k = c.tm.lane; k < K; k += TEAM) {
    if (k == 0) continue;
    float t1[NX * NX];
    // t1 = O_k Pd_{k-1}
#pragma unroll (NX <= 8 ? 32 : 1)
    for (int i = 0; i < NX; ++i)
#pragma unroll (NX <= 8 ? 32 : 1)
      for (int j = 0; j < NX; ++j) {
        float s = 0.f;
#pragma unroll (NX <= 8 ? 32 : 1)
        for (int l = 0; l < NX; ++l) s = fmaf(O[(i * NX + l) * KP + k], Pd[(l * NX + j) * KP + k - 1], s);
        t1[i * NX + j] = s;
      }
#pragma unroll (NX <= 8 ? 32 : 1)
    for (int i = 0; i < NX; ++i)
#pragma unroll (NX <= 8 ? 32 : 1)
      for (int j = 0; j < NX; ++j) {
        float s = 0.f;
#pragma unroll (NX <= 8 ? 32 : 1)
        for (int l = 0; l < NX; ++l) s = fmaf(Pd[(i * NX + l) * KP + k], t1[l * NX + j], s);
        Po[(i * NX + j) * KP + k] = -s;
      }
  }
  c.tm.sync();
}

// FP64 product S_spd * src evaluated from the factors (H, G^-1) of the current QP data:
// w = H^T src, then (H G^-1 w).  With res = true it writes the float residual
// r = float(gamma - S src); otherwise the double product dst = S src.  Leaves w = H^T src in
// the wx/wu arrays (used by the recovery step).
template <class M, int TEAM>
__device__ __noinline__ void hp_apply(Ctx<M, TEAM>& c, const double* src, bool res, double* dst) {
  constexpr int NX = M::NX, NU = M::NU;
  const int T = c.T, K = c.K, KP = c.KP;
  const float* A = c.F(c.L.A);
  const float* Bm = c.F(c.L.Bm);
  double* WX = c.Dp(c.L.d_wx);
  double* WU = c.Dp(c.L.d_wu);
  const double* G = c.Dp(c.L.d_gam);
  float* R = c.F(c.L.r);
  c.tm.sync();
  for (int k = c.tm.lane; k < K; k += TEAM) {
    double wx[NX];
#pragma unroll
    for (int i = 0; i < NX; ++i) wx[i] = src[i * KP + k];
    if constexpr (is_implicit<M>::value) {
      if (k > 0) {  // row k's coefficient of x_k is A^+ (slot k); row 0's is I
        const float* Ap = c.F(c.L.Ap);
        double w2[NX];
#pragma unroll
        for (int i = 0; i < NX; ++i) {
          double acc = 0.0;
#pragma unroll
          for (int j = 0; j < NX; ++j) acc += (double)Ap[(j * NX + i) * KP + k] * wx[j];
          w2[i] = acc;
        }
#pragma unroll
        for (int i = 0; i < NX; ++i) wx[i] = w2[i];
      }
    }
    if (k < T) {
      double ln[NX];
#pragma unroll
      for (int j = 0; j < NX; ++j) ln[j] = src[j * KP + k + 1];
      // A_k lives at slot k + 1 (stored as A_k + I)
#pragma unroll
      for (int i = 0; i < NX; ++i) {
        double s = wx[i] - ln[i];
#pragma unroll
        for (int j = 0; j < NX; ++j) s += (double)A[(j * NX + i) * KP + k + 1] * ln[j];
        wx[i] = s;
      }
#pragma unroll
      for (int i = 0; i < NU; ++i) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < NX; ++j) s += (double)Bm[(j * NU + i) * KP + k + 1] * ln[j];
        WU[i * KP + k] = s;
      }
    }
#pragma unroll
    for (int i = 0; i < NX; ++i) WX[i * KP + k] = wx[i];
  }
  c.tm.sync();
  for (int k = c.tm.lane; k < K; k += TEAM) {
    double s[NX], su[NU], wx[NX], wu[NU];
#pragma unroll
    for (int i = 0; i < NX; ++i) wx[i] = WX[i * KP + k];
#pragma unroll
    for (int i = 0; i < NU; ++i) wu[i] = (k < T) ? WU[i * KP + k] : 0.0;
    c.ginv(k, wx, wu, s, su);
    if constexpr (is_implicit<M>::value) {
      if (k > 0) {
        const float* Ap = c.F(c.L.Ap);
        double s2[NX];
#pragma unroll
        for (int i = 0; i < NX; ++i) {
          double acc = 0.0;
#pragma unroll
          for (int j = 0; j < NX; ++j) acc += (double)Ap[(i * NX + j) * KP + k] * s[j];
          s2[i] = acc;
        }
#pragma unroll
        for (int i = 0; i < NX; ++i) s[i] = s2[i];
      }
    }
    if (k > 0) {
      const int t = k - 1;
      double vx[NX], vu[NU];
#pragma unroll
      for (int j = 0; j < NX; ++j) wx[j] = WX[j * KP + t];
#pragma unroll
      for (int j = 0; j < NU; ++j) wu[j] = WU[j * KP + t];
      c.ginv(t, wx, wu, vx, vu);
#pragma unroll
      for (int i = 0; i < NX; ++i) {
        double acc = s[i] - vx[i];
#pragma unroll
        for (int j = 0; j < NX; ++j) acc += (double)A[(i * NX + j) * KP + k] * vx[j];
#pragma unroll
        for (int j = 0; j < NU; ++j) acc += (double)Bm[(i * NU + j) * KP + k] * vu[j];
        s[i] = acc;
      }
    }
    if (res) {
#pragma unroll
      for (int i = 0; i < NX; ++i) R[i * KP + k] = (float)(G[i * KP + k] - s[i]);
    } else {
#pragma unroll
      for (int i = 0; i < NX; ++i) dst[i * KP + k] = s[i];
    }
  }
  c.tm.sync();
}

template <class M, int TEAM>
__device__ __forceinline__ void hp_residual(Ctx<M, TEAM>& c, const double* src) {
  hp_apply<M, TEAM>(c, src, true, nullptr);
}

// Double-float rescue for any team size (workspace vectors): Algorithm 4 continued from the
// folded solution with the vectors, the scalars and every sum in double-float (compensated
// accumulation, FP32 instructions), the operator S = H G^-1 H^T applied from the FP32 factors
// and the reciprocal weights (the FP64 true-residual operator), and the preconditioner from its
// FP32 blocks (exactly symmetric: the diagonal blocks are formed symmetric).  Replaces an FP64
// rescue whose cost on this GPU's FP64 pipe dominated large OCPs.  Vectors live in the double
// arrays of the workspace, one (hi, lo) pair per double slot.
template <int TEAM>
__device__ __forceinline__ dfl team_df_sum(Team<TEAM>& tm, dfl v) {
  v = df_warp_sum(v);
  if (TEAM <= 32) {
    __syncwarp();
    return v;
  }
  constexpr int NW = TEAM / 32, RM = Team<TEAM>::RED_MAX;
  float* rb = tm.red + tm.buf * (NW * RM);
  const int w = tm.lane >> 5;
  if ((tm.lane & 31) == 0) { rb[w * RM] = v.hi; rb[w * RM + 1] = v.lo; }
  tm.sync();
  dfl s = {rb[0], rb[1]};
  for (int q = 1; q < NW; ++q) s = df_add(s, dfl{rb[q * RM], rb[q * RM + 1]});
  tm.buf ^= 1;
  return s;
}

// out = S v in double-float; leaves w = H^T v in (WX, WU).
template <class M, int TEAM>
__device__ __noinline__ void df_apply(Ctx<M, TEAM>& c, const dfl* v, dfl* out, dfl* WX, dfl* WU,
                                      const dfl (&qx)[M::NX], const dfl (&qT)[M::NX], const dfl (&ri)[M::NU]) {
  constexpr int NX = M::NX, NU = M::NU;
  const int T = c.T, K = c.K, KP = c.KP;
  const float* A = c.F(c.L.A);
  const float* Bm = c.F(c.L.Bm);
  c.tm.sync();
  for (int k = c.tm.lane; k < K; k += TEAM) {
#pragma unroll (NX <= 8 ? 32 : 1)
    for (int i = 0; i < NX; ++i) {
      dacc a = dacc_zero();
      if constexpr (is_implicit<M>::value) {
        if (k > 0) {
#pragma unroll
          for (int j = 0; j < NX; ++j) dacc_fma(a, c.F(c.L.Ap)[(j * NX + i) * KP + k], v[j * KP + k]);
        } else {
          dacc_add(a, v[i * KP + k]);
        }
      } else {
        dacc_add(a, v[i * KP + k]);
      }
      if (k < T) {   // (A_k + I)^T v_{k+1} - v_{k+1}
#pragma unroll
        for (int j = 0; j < NX; ++j) dacc_fma(a, A[(j * NX + i) * KP + k + 1], v[j * KP + k + 1]);
        dacc_add(a, df_neg(v[i * KP + k + 1]));
      }
      WX[i * KP + k] = dacc_get(a);
    }
    if (k < T) {
#pragma unroll
      for (int i = 0; i < NU; ++i) {
        dacc a = dacc_zero();
#pragma unroll
        for (int j = 0; j < NX; ++j) dacc_fma(a, Bm[(j * NU + i) * KP + k + 1], v[j * KP + k + 1]);
        WU[i * KP + k] = dacc_get(a);
      }
    }
  }
  c.tm.sync();
  for (int k = c.tm.lane; k < K; k += TEAM) {
    dfl vx[NX], vu[NU];
    if (k > 0) {
#pragma unroll
      for (int j = 0; j < NX; ++j) vx[j] = df_mul(WX[j * KP + k - 1], qx[j]);  // k - 1 < T
#pragma unroll
      for (int j = 0; j < NU; ++j) vu[j] = df_mul(WU[j * KP + k - 1], ri[j]);
    }
#pragma unroll (NX <= 8 ? 32 : 1)
    for (int i = 0; i < NX; ++i) {
      dacc a = dacc_zero();
      if constexpr (is_implicit<M>::value) {
        if (k > 0) {
#pragma unroll
          for (int j = 0; j < NX; ++j)
            dacc_fma(a, c.F(c.L.Ap)[(i * NX + j) * KP + k], df_mul(WX[j * KP + k], k < T ? qx[j] : qT[j]));
        } else {
          dacc_add(a, df_mul(WX[i * KP + k], qx[i]));
        }
      } else {
        dacc_add(a, df_mul(WX[i * KP + k], k < T ? qx[i] : qT[i]));
      }
      if (k > 0) {
#pragma unroll
        for (int j = 0; j < NX; ++j) dacc_fma(a, A[(i * NX + j) * KP + k], vx[j]);
        dacc_add(a, df_neg(vx[i]));
#pragma unroll
        for (int j = 0; j < NU; ++j) dacc_fma(a, Bm[(i * NU + j) * KP + k], vu[j]);
      }
      out[i * KP + k] = dacc_get(a);
    }
  }
  c.tm.sync();
}

template <int NX>
__device__ __forceinline__ void btmv_row_df(const float* Md, const float* Mo, const dfl* v, int k, int K, int KP,
                                            dfl (&out)[NX]) {
#pragma unroll (NX <= 8 ? 32 : 1)
  for (int i = 0; i < NX; ++i) {
    dacc a = dacc_zero();
#pragma unroll
    for (int j = 0; j < NX; ++j) dacc_fma(a, Md[(i * NX + j) * KP + k], v[j * KP + k]);
    if (k > 0) {
#pragma unroll
      for (int j = 0; j < NX; ++j) dacc_fma(a, Mo[(i * NX + j) * KP + k], v[j * KP + k - 1]);
    }
    if (k + 1 < K) {
#pragma unroll
      for (int j = 0; j < NX; ++j) dacc_fma(a, Mo[(j * NX + i) * KP + k + 1], v[j * KP + k + 1]);
    }
    out[i] = dacc_get(a);
  }
}

template <class M, int TEAM>
__device__ __noinline__ int stage_pcg_df(Ctx<M, TEAM>& c, float eta0f, int maxit) {
  constexpr int NX = M::NX, NU = M::NU;
  const KParams& P = *c.P;
  const int K = c.K, KP = c.KP;
  const float* Pd = c.F(c.L.Pd);
  const float* Po = c.F(c.L.Po);
  double* LP = c.Dp(c.L.d_lamp);
  const double* G = c.Dp(c.L.d_gam);
  // double-float vectors: x in d_y, r in d_r, p in d_p (one pair per double slot); y = S p in
  // the FP32 scratch arrays r and p, which are contiguous (2 NX KP floats = NX KP pairs)
  dfl* X = reinterpret_cast<dfl*>(c.Dp(c.L.d_y));
  dfl* R = reinterpret_cast<dfl*>(c.Dp(c.L.d_r));
  dfl* Pv = reinterpret_cast<dfl*>(c.Dp(c.L.d_p));
  dfl* Y = reinterpret_cast<dfl*>(c.F(c.L.r));  // spans the FP32 arrays r and p (contiguous)
  dfl* WX = reinterpret_cast<dfl*>(c.Dp(c.L.d_wx));
  dfl* WU = reinterpret_cast<dfl*>(c.Dp(c.L.d_wu));
  dfl qx[NX], qT[NX], ri[NU];
#pragma unroll
  for (int i = 0; i < NX; ++i) { qx[i] = df_from(c.qinv(0, i)); qT[i] = df_from(c.qinv(c.T, i)); }
#pragma unroll
  for (int i = 0; i < NU; ++i) ri[i] = df_from(c.rinv(i));
  const dfl thr = df_mulf(df_make(eta0f), P.opt.pcg_tol * P.opt.pcg_tol);
  for (int k = c.tm.lane; k < K; k += TEAM)
#pragma unroll
    for (int i = 0; i < NX; ++i) X[i * KP + k] = df_from(LP[i * KP + k]);
  df_apply<M, TEAM>(c, X, Pv, WX, WU, qx, qT, ri);  // Pv = S x (temporarily)
  for (int k = c.tm.lane; k < K; k += TEAM)
#pragma unroll
    for (int i = 0; i < NX; ++i) R[i * KP + k] = df_sub(df_from(G[i * KP + k]), Pv[i * KP + k]);
  c.tm.sync();
  dacc ea = dacc_zero();
  for (int k = c.tm.lane; k < K; k += TEAM) {
    dfl z[NX];
    btmv_row_df<NX>(Pd, Po, R, k, K, KP, z);
#pragma unroll
    for (int i = 0; i < NX; ++i) { Pv[i * KP + k] = z[i]; dacc_fma(ea, R[i * KP + k], z[i]); }
  }
  dfl eta = team_df_sum<TEAM>(c.tm, dacc_get(ea));
  int it = 0;
  bool converged = !(eta.hi > thr.hi);
  while (!converged && it < maxit) {
    df_apply<M, TEAM>(c, Pv, Y, WX, WU, qx, qT, ri);
    dacc va = dacc_zero();
    for (int k = c.tm.lane; k < K; k += TEAM)
#pragma unroll
      for (int i = 0; i < NX; ++i) dacc_fma(va, Pv[i * KP + k], Y[i * KP + k]);
    const dfl v = team_df_sum<TEAM>(c.tm, dacc_get(va));
    if (!(v.hi > 0.f) || !isfinite(v.hi)) { c.status |= ST_PCG_BREAKDOWN; break; }
    const dfl alpha = df_div(eta, v);
    for (int k = c.tm.lane; k < K; k += TEAM)
#pragma unroll
      for (int i = 0; i < NX; ++i) {
        X[i * KP + k] = df_add(X[i * KP + k], df_mul(alpha, Pv[i * KP + k]));
        R[i * KP + k] = df_sub(R[i * KP + k], df_mul(alpha, Y[i * KP + k]));
      }
    c.tm.sync();
    dacc na = dacc_zero();
    for (int k = c.tm.lane; k < K; k += TEAM) {
      dfl z[NX];
      btmv_row_df<NX>(Pd, Po, R, k, K, KP, z);
#pragma unroll
      for (int i = 0; i < NX; ++i) { Y[i * KP + k] = z[i]; dacc_fma(na, R[i * KP + k], z[i]); }
    }
    const dfl eta_new = team_df_sum<TEAM>(c.tm, dacc_get(na));
    ++it;
    if (!(eta_new.hi > thr.hi)) { converged = true; break; }
    if (!isfinite(eta_new.hi)) break;
    const dfl beta = df_div(eta_new, eta);
    eta = eta_new;
    for (int k = c.tm.lane; k < K; k += TEAM)
#pragma unroll
      for (int i = 0; i < NX; ++i) Pv[i * KP + k] = df_add(Y[i * KP + k], df_mul(beta, Pv[i * KP + k]));
    c.tm.sync();
  }
  for (int k = c.tm.lane; k < K; k += TEAM)
#pragma unroll
    for (int i = 0; i < NX; ++i) LP[i * KP + k] = df_to(X[i * KP + k]);
  hp_residual<M, TEAM>(c, LP);  // leaves w = H^T lambda (FP64) for the recovery
  if (!converged) c.status |= ST_PCG_MAXITER;
  return it;
}

// a4: PCG (Algorithm 4) on S_spd lambda = gamma_spd.  The iteration runs in FP32 on the
// FP32 blocks; the solution is accumulated in FP64 (lamp) and the residual is replaced by
// the FP64 true residual whenever eta has dropped by ru_delta^2 since the last
// replacement, and before convergence is declared (a "reliable update" scheme).
// Stops when eta <= pcg_tol^2 * eta_0, eta_0 = gamma^T Phi^-1 gamma, on a true residual.
// On entry lamp holds the initial guess.  Returns the iteration count.
template <class M, int TEAM>
__device__ __noinline__ int stage_pcg(Ctx<M, TEAM>& c) {
  constexpr int NX = M::NX;
  const KParams& P = *c.P;
  const int K = c.K, KP = c.KP;
  const float* D = c.F(c.L.D);
  const float* O = c.F(c.L.O);
  const float* Pd = c.F(c.L.Pd);
  const float* Po = c.F(c.L.Po);
  float* R = c.F(c.L.r);
  float* Pv = c.F(c.L.p);
  float* Y = c.F(c.L.y);
  float* DL = c.F(c.L.dl);
  double* LP = c.Dp(c.L.d_lamp);
  const double* G = c.Dp(c.L.d_gam);
  const float tol2 = P.opt.pcg_tol * P.opt.pcg_tol;
  const float dl2 = P.opt.ru_delta * P.opt.ru_delta;

  for (int k = c.tm.lane; k < K; k += TEAM) {
#pragma unroll
    for (int i = 0; i < NX; ++i) { Y[i * KP + k] = (float)G[i * KP + k]; DL[i * KP + k] = 0.f; }
  }
  hp_residual<M, TEAM>(c, LP);
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
  float eta = red2[0];
  const float eta0 = red2[1];
  float eta_ref = eta;       // eta at the last true-residual replacement
  float eta_true = eta;      // last true eta
  int it = 0, stall = 0;
  bool converged = !(eta > tol2 * eta0);
  bool rescue = false;
  const int maxit = P.opt.pcg_max_iters;
  bool folded = true;
  while (!converged && it < maxit) {
    // y = S p,  v = p^T y
    float v[1] = {0.f};
    for (int k = c.tm.lane; k < K; k += TEAM) {
      float y[NX];
      btmv_row<NX>(D, O, Pv, k, K, KP, y);
#pragma unroll
      for (int i = 0; i < NX; ++i) { Y[i * KP + k] = y[i]; v[0] = fmaf(Pv[i * KP + k], y[i], v[0]); }
    }
    c.tm.sum(v);
    if (!(v[0] > 0.f) || !isfinite(v[0])) { rescue = true; break; }
    const float alpha = eta / v[0];
    for (int k = c.tm.lane; k < K; k += TEAM) {
#pragma unroll
      for (int i = 0; i < NX; ++i) {
        DL[i * KP + k] = fmaf(alpha, Pv[i * KP + k], DL[i * KP + k]);
        R[i * KP + k] = fmaf(-alpha, Y[i * KP + k], R[i * KP + k]);
      }
    }
    folded = false;
    c.tm.sync();
    float e1[1] = {0.f};
    for (int k = c.tm.lane; k < K; k += TEAM) {
      float rt[NX];
      btmv_row<NX>(Pd, Po, R, k, K, KP, rt);
#pragma unroll
      for (int i = 0; i < NX; ++i) { Y[i * KP + k] = rt[i]; e1[0] = fmaf(R[i * KP + k], rt[i], e1[0]); }
    }
    c.tm.sum(e1);
    float eta_new = e1[0];
    ++it;
    if (eta_new < dl2 * eta_ref || !(eta_new > tol2 * eta0) || it >= maxit || !isfinite(eta_new)) {
      // reliable update: fold the FP32 correction into the FP64 solution, true residual
      for (int k = c.tm.lane; k < K; k += TEAM) {
#pragma unroll
        for (int i = 0; i < NX; ++i) { LP[i * KP + k] += (double)DL[i * KP + k]; DL[i * KP + k] = 0.f; }
      }
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
      if (!(eta_new > tol2 * eta0)) { converged = true; break; }
      if (!isfinite(eta_new)) { rescue = true; break; }
      // stagnation: a whole update cycle (meant to gain ru_delta^-2) gained less than 4x on the
      // true residual twice in a row -> the FP32 operator cannot resolve this system
      if (eta_new > 0.25f * eta_true) {
        if (++stall >= 2) { rescue = true; break; }
      } else {
        stall = 0;
      }
      eta_true = eta_new;
      if (it >= maxit) { rescue = true; break; }
    }
    const float beta = eta_new / eta;
    eta = eta_new;
    for (int k = c.tm.lane; k < K; k += TEAM) {
#pragma unroll
      for (int i = 0; i < NX; ++i) Pv[i * KP + k] = fmaf(beta, Pv[i * KP + k], Y[i * KP + k]);
    }
    c.tm.sync();
  }
  if (!folded) {
    for (int k = c.tm.lane; k < K; k += TEAM) {
#pragma unroll
      for (int i = 0; i < NX; ++i) { LP[i * KP + k] += (double)DL[i * KP + k]; DL[i * KP + k] = 0.f; }
    }
    hp_residual<M, TEAM>(c, LP);
  }
  if (!converged) {
    // per-OCP double-float rescue of this solve, continuing from the folded solution
    c.status |= ST_FP64_RESCUE;
    const int d = stage_pcg_df<M, TEAM>(c, eta0, maxit);
    c.df_iters += d;
    it += d;
  }
  return it;
}

// Neighbour terms of a block-tridiagonal row for one-knot-per-lane ownership (knot k = lane):
// vm = v_{k-1} and tn = (M_{k+1})^T v_{k+1}, where every lane provides its own v_k and
// t_k = M_k^T v_k.  Inside a warp they move by shuffles; across warps lane 31 / lane 0 go through
// a small shared buffer (double-buffered by `buf`, barrier of the team).
template <int NX, int TEAM>
__device__ __forceinline__ void neighbour_terms(const float (&v)[NX], const float (&t)[NX], float (&vm)[NX],
                                                float (&tn)[NX], Team<TEAM>& tm, float* bnd, int buf) {
  constexpr int NW = TEAM / 32;
  const int ln = tm.lane & 31, wid = tm.lane >> 5;
#pragma unroll
  for (int i = 0; i < NX; ++i) {
    vm[i] = __shfl_up_sync(0xffffffffu, v[i], 1);
    tn[i] = __shfl_down_sync(0xffffffffu, t[i], 1);
  }
  if (NW > 1) {
    float* B = bnd + buf * (NW * 2 * NX);
    if (ln == 0) {
#pragma unroll
      for (int i = 0; i < NX; ++i) B[(wid * 2 + 0) * NX + i] = t[i];
    }
    if (ln == 31) {
#pragma unroll
      for (int i = 0; i < NX; ++i) B[(wid * 2 + 1) * NX + i] = v[i];
    }
    tm.sync();
    if (ln == 0) {
#pragma unroll
      for (int i = 0; i < NX; ++i) vm[i] = wid > 0 ? B[((wid - 1) * 2 + 1) * NX + i] : 0.f;
    }
    if (ln == 31) {
#pragma unroll
      for (int i = 0; i < NX; ++i) tn[i] = wid < NW - 1 ? B[((wid + 1) * 2 + 0) * NX + i] : 0.f;
    }
  } else {
    if (ln == 0) {
#pragma unroll
      for (int i = 0; i < NX; ++i) vm[i] = 0.f;
    }
    if (ln == 31) {
#pragma unroll
      for (int i = 0; i < NX; ++i) tn[i] = 0.f;
    }
  }
}

// out = Md v + Mo vm + tn, and t = Mo^T v (the part lane k-1 needs), with register blocks.
template <int NX>
__device__ __forceinline__ void reg_row(const float (&Md)[NX * NX], const float (&Mo)[NX * NX], const float (&v)[NX],
                                        float (&t)[NX]) {
#pragma unroll
  for (int j = 0; j < NX; ++j) {
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < NX; ++i) s = fmaf(Mo[i * NX + j], v[i], s);
    t[j] = s;
  }
}

// a4, register-resident variant (one knot per lane, K <= TEAM, nx <= 6): the same algorithm
// as stage_pcg (FP32 iteration, FP64 solution with reliable updates, double-float rescue), with the
// S and Phi^-1 blocks of the lane's knot held in registers for the whole solve and the neighbour
// coupling done with shuffles (a small shared buffer across warps), so the loop reads no blocks.
template <class M, int TEAM>
__device__ __noinline__ int stage_pcg_reg(Ctx<M, TEAM>& c) {
  constexpr int NX = M::NX;
  const KParams& P = *c.P;
  const int K = c.K, KP = c.KP;
  const int k = c.tm.lane;
  const bool live = k < K;
  float* R = c.F(c.L.r);
  float* Y = c.F(c.L.y);
  float* bnd = c.F(c.L.bnd);
  double* LP = c.Dp(c.L.d_lamp);
  const double* G = c.Dp(c.L.d_gam);
  const float* Pdm = c.F(c.L.Pd);
  const float* Pom = c.F(c.L.Po);
  const float tol2 = P.opt.pcg_tol * P.opt.pcg_tol;
  const float dl2 = P.opt.ru_delta * P.opt.ru_delta;
  Team<TEAM> tm = c.tm;  // team state in registers for the loop (c lives in local memory)
  float Dk[NX * NX], Ok[NX * NX], Pdk[NX * NX], Pok[NX * NX];
#pragma unroll
  for (int e = 0; e < NX * NX; ++e) {
    Dk[e] = live ? c.F(c.L.D)[e * KP + k] : 0.f;
    Ok[e] = (live && k > 0) ? c.F(c.L.O)[e * KP + k] : 0.f;
    Pdk[e] = live ? Pdm[e * KP + k] : 0.f;
    Pok[e] = (live && k > 0) ? Pom[e * KP + k] : 0.f;
  }
  if (live) {
#pragma unroll
    for (int i = 0; i < NX; ++i) Y[i * KP + k] = (float)G[i * KP + k];
  }
  hp_residual<M, TEAM>(c, LP);
  float r[NX], p[NX], dl[NX], rt[NX], t[NX], vm[NX], tn[NX];
  float red2[2] = {0.f, 0.f};
  if (live) {
    float gt[NX];
    btmv_row<NX>(Pdm, Pom, R, k, K, KP, rt);
    btmv_row<NX>(Pdm, Pom, Y, k, K, KP, gt);
#pragma unroll
    for (int i = 0; i < NX; ++i) {
      r[i] = R[i * KP + k];
      red2[0] = fmaf(r[i], rt[i], red2[0]);
      red2[1] = fmaf(Y[i * KP + k], gt[i], red2[1]);
    }
  } else {
#pragma unroll
    for (int i = 0; i < NX; ++i) { r[i] = 0.f; rt[i] = 0.f; }
  }
#pragma unroll
  for (int i = 0; i < NX; ++i) { p[i] = rt[i]; dl[i] = 0.f; }
  tm.sum(red2);
  float eta = red2[0];
  const float eta0 = red2[1];
  float eta_ref = eta, eta_true = eta;
  int it = 0, stall = 0, xb = 0;
  bool converged = !(eta > tol2 * eta0);
  const int maxit = P.opt.pcg_max_iters;
  bool folded = true;
  while (!converged && it < maxit) {
    // y = S p
    reg_row<NX>(Dk, Ok, p, t);
    neighbour_terms<NX, TEAM>(p, t, vm, tn, tm, bnd, xb); xb ^= 1;
    float y[NX];
    float v[1] = {0.f};
#pragma unroll
    for (int i = 0; i < NX; ++i) {
      float s = tn[i];
#pragma unroll
      for (int j = 0; j < NX; ++j) s = fmaf(Dk[i * NX + j], p[j], fmaf(Ok[i * NX + j], vm[j], s));
      y[i] = s;
      v[0] = fmaf(p[i], s, v[0]);
    }
    tm.sum(v);
    if (!(v[0] > 0.f) || !isfinite(v[0])) break;
    const float alpha = __fdividef(eta, v[0]);
#pragma unroll
    for (int i = 0; i < NX; ++i) { dl[i] = fmaf(alpha, p[i], dl[i]); r[i] = fmaf(-alpha, y[i], r[i]); }
    folded = false;
    // rt = Phi^-1 r
    reg_row<NX>(Pdk, Pok, r, t);
    neighbour_terms<NX, TEAM>(r, t, vm, tn, tm, bnd, xb); xb ^= 1;
    float e1[1] = {0.f};
#pragma unroll
    for (int i = 0; i < NX; ++i) {
      float s = tn[i];
#pragma unroll
      for (int j = 0; j < NX; ++j) s = fmaf(Pdk[i * NX + j], r[j], fmaf(Pok[i * NX + j], vm[j], s));
      rt[i] = s;
      e1[0] = fmaf(r[i], s, e1[0]);
    }
    tm.sum(e1);
    float eta_new = e1[0];
    ++it;
    if (eta_new < dl2 * eta_ref || !(eta_new > tol2 * eta0) || it >= maxit || !isfinite(eta_new)) {
      if (live) {
#pragma unroll
        for (int i = 0; i < NX; ++i) { LP[i * KP + k] += (double)dl[i]; dl[i] = 0.f; }
      }
      folded = true;
      hp_residual<M, TEAM>(c, LP);
      float e2[1] = {0.f};
      if (live) {
        btmv_row<NX>(Pdm, Pom, R, k, K, KP, rt);
#pragma unroll
        for (int i = 0; i < NX; ++i) { r[i] = R[i * KP + k]; e2[0] = fmaf(r[i], rt[i], e2[0]); }
      }
      tm.sum(e2);
      eta_new = e2[0];
      eta_ref = eta_new;
      if (!(eta_new > tol2 * eta0)) { converged = true; break; }
      if (!isfinite(eta_new)) break;
      if (eta_new > 0.25f * eta_true) {
        if (++stall >= 2) break;
      } else {
        stall = 0;
      }
      eta_true = eta_new;
      if (it >= maxit) break;
    }
    const float beta = __fdividef(eta_new, eta);
    eta = eta_new;
#pragma unroll
    for (int i = 0; i < NX; ++i) p[i] = fmaf(beta, p[i], rt[i]);
  }
  if (!folded) {
    if (live) {
#pragma unroll
      for (int i = 0; i < NX; ++i) LP[i * KP + k] += (double)dl[i];
    }
    hp_residual<M, TEAM>(c, LP);
  }
  c.tm.buf = tm.buf;
  if (!converged) {
    c.status |= ST_FP64_RESCUE;
    const int d = stage_pcg_df<M, TEAM>(c, eta0, maxit);
    c.df_iters += d;
    it += d;
  }
  return it;
}

// Block-tridiagonal row product for KPL contiguous knots per lane (knots l*KPL + j) of one
// warp, blocks in registers: out_j = Md_j v_j + Mo_j v_{j-1} + Mo_{j+1}^T v_{j+1}.  The
// transposed products t_j = Mo_j^T v_j travel to the previous knot; across lanes both move by
// shuffles (lane 0 receives zeros, lane 31 receives zeros).
template <int NX, int KPL>
__device__ __forceinline__ void warp_btmv(const float (&Md)[KPL][NX * NX], const float (&Mo)[KPL][NX * NX],
                                          const float (&v)[KPL][NX], float (&out)[KPL][NX], int ln) {
  float t[KPL][NX];
#pragma unroll
  for (int j = 0; j < KPL; ++j)
#pragma unroll
    for (int b = 0; b < NX; ++b) {
      float a = 0.f;
#pragma unroll
      for (int i = 0; i < NX; ++i) a = fmaf(Mo[j][i * NX + b], v[j][i], a);
      t[j][b] = a;
    }
  float vm[NX], tn[NX];
#pragma unroll
  for (int i = 0; i < NX; ++i) {
    vm[i] = __shfl_up_sync(0xffffffffu, v[KPL - 1][i], 1);
    tn[i] = __shfl_down_sync(0xffffffffu, t[0][i], 1);
    if (ln == 0) vm[i] = 0.f;
    if (ln == 31) tn[i] = 0.f;
  }
#pragma unroll
  for (int j = 0; j < KPL; ++j)
#pragma unroll
    for (int i = 0; i < NX; ++i) {
      float a = (j + 1 < KPL) ? t[j + 1 < KPL ? j + 1 : 0][i] : tn[i];
#pragma unroll
      for (int q = 0; q < NX; ++q) {
        const float prev = (j > 0) ? v[j > 0 ? j - 1 : 0][q] : vm[q];
        a = fmaf(Md[j][i * NX + q], v[j][q], fmaf(Mo[j][i * NX + q], prev, a));
      }
      out[j][i] = a;
    }
}

template <int NV>
__device__ __forceinline__ void warp_sum(float (&v)[NV]) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] += __shfl_xor_sync(0xffffffffu, v[j], off);
}

// Double-float PCG for the single-warp path (Algorithm 4 in about 48-bit arithmetic built from
// FP32 instructions): the operator S = H G^-1 H^T is applied from the FP32 factors A_t, B_t and
// the reciprocal weights (the same operator as the FP64 true residual), the preconditioner from
// its FP32 blocks with the diagonal blocks symmetrised (so it is exactly symmetric), and the
// vectors and the scalars alpha, beta, eta are double-float.  All state in registers,
// neighbour exchanges by shuffles.  Used as the rescue of a stagnated FP32 iteration, or for
// the whole solve when the options ask for it.

// out = M v for a block-tridiagonal symmetric M (diagonal blocks Md, sub-diagonal blocks Mo),
// v and out double-float; same data movement as warp_btmv.
template <int NX, int KPL>
__device__ __forceinline__ void warp_btmv_df(const float (&Md)[KPL][NX * NX], const float (&Mo)[KPL][NX * NX],
                                             const dfl (&v)[KPL][NX], dfl (&out)[KPL][NX], int ln) {
  dfl t[KPL][NX];
#pragma unroll
  for (int j = 0; j < KPL; ++j)
#pragma unroll
    for (int b = 0; b < NX; ++b) {
      dacc a = dacc_zero();
#pragma unroll
      for (int i = 0; i < NX; ++i) dacc_fma(a, Mo[j][i * NX + b], v[j][i]);
      t[j][b] = dacc_get(a);
    }
  dfl vm[NX], tn[NX];
#pragma unroll
  for (int i = 0; i < NX; ++i) {
    vm[i].hi = __shfl_up_sync(0xffffffffu, v[KPL - 1][i].hi, 1);
    vm[i].lo = __shfl_up_sync(0xffffffffu, v[KPL - 1][i].lo, 1);
    tn[i].hi = __shfl_down_sync(0xffffffffu, t[0][i].hi, 1);
    tn[i].lo = __shfl_down_sync(0xffffffffu, t[0][i].lo, 1);
    if (ln == 0) vm[i] = df_make(0.f);
    if (ln == 31) tn[i] = df_make(0.f);
  }
#pragma unroll
  for (int j = 0; j < KPL; ++j)
#pragma unroll
    for (int i = 0; i < NX; ++i) {
      dacc a = dacc_zero();
      dacc_add(a, (j + 1 < KPL) ? t[j + 1 < KPL ? j + 1 : 0][i] : tn[i]);
#pragma unroll
      for (int q = 0; q < NX; ++q) {
        dacc_fma(a, Mo[j][i * NX + q], (j > 0) ? v[j > 0 ? j - 1 : 0][q] : vm[q]);
        dacc_fma(a, Md[j][i * NX + q], v[j][q]);
      }
      out[j][i] = dacc_get(a);
    }
}

template <class M, int KPL>
__device__ __forceinline__ void warp_S_df(const float (&Ak)[KPL][M::NX * M::NX], const float (&Bk)[KPL][M::NX * M::NU],
                                          const float (&Apk)[KPL][M::NX * M::NX],
                                          const dfl (&qi)[KPL][M::NX], const dfl (&ri)[M::NU], const bool (&has_u)[KPL],
                                          const bool (&has_a)[KPL], const dfl (&v)[KPL][M::NX], dfl (&out)[KPL][M::NX],
                                          int ln) {
  // Ak: A_k + I of the knots that carry a dynamics row (has_a), else 0; Apk: A^+ of the lane's
  // knots (identity at knot 0), read only for implicit integrators
  constexpr int NX = M::NX, NU = M::NU;
  // pass 1: w = H^T v.  Knot k+1 owns A_k (slot k+1) and sends A_k^T v_{k+1}, B_k^T v_{k+1}.
  dfl t[KPL][NX], ub[KPL][NU];
#pragma unroll
  for (int j = 0; j < KPL; ++j) {
#pragma unroll
    for (int b = 0; b < NX; ++b) {
      dacc a = dacc_zero();
#pragma unroll
      for (int i = 0; i < NX; ++i) dacc_fma(a, Ak[j][i * NX + b], v[j][i]);
      if (has_a[j]) dacc_add(a, df_neg(v[j][b]));
      t[j][b] = dacc_get(a);
    }
#pragma unroll
    for (int b = 0; b < NU; ++b) {
      dacc a = dacc_zero();
#pragma unroll
      for (int i = 0; i < NX; ++i) dacc_fma(a, Bk[j][i * NU + b], v[j][i]);
      ub[j][b] = dacc_get(a);
    }
  }
  dfl tn[NX], ubn[NU];
#pragma unroll
  for (int i = 0; i < NX; ++i) {
    tn[i].hi = __shfl_down_sync(0xffffffffu, t[0][i].hi, 1);
    tn[i].lo = __shfl_down_sync(0xffffffffu, t[0][i].lo, 1);
    if (ln == 31) tn[i] = df_make(0.f);
  }
#pragma unroll
  for (int i = 0; i < NU; ++i) {
    ubn[i].hi = __shfl_down_sync(0xffffffffu, ub[0][i].hi, 1);
    ubn[i].lo = __shfl_down_sync(0xffffffffu, ub[0][i].lo, 1);
    if (ln == 31) ubn[i] = df_make(0.f);
  }
  // pass 2: G^-1 w, then H (G^-1 w); knot k needs the scaled w of knot k-1
  dfl vx[KPL][NX], vu[KPL][NU];
#pragma unroll
  for (int j = 0; j < KPL; ++j) {
    dfl own[NX];  // the knot's own row term of H^T v: v_k, or A^+_k^T v_k for implicit integrators
#pragma unroll
    for (int i = 0; i < NX; ++i) {
      if constexpr (is_implicit<M>::value) {
        dacc a = dacc_zero();
#pragma unroll
        for (int q = 0; q < NX; ++q) dacc_fma(a, Apk[j][q * NX + i], v[j][q]);
        own[i] = dacc_get(a);
      } else {
        own[i] = v[j][i];
      }
    }
#pragma unroll
    for (int i = 0; i < NX; ++i) vx[j][i] = df_mul(df_add(own[i], (j + 1 < KPL) ? t[j + 1 < KPL ? j + 1 : 0][i] : tn[i]), qi[j][i]);
#pragma unroll
    for (int i = 0; i < NU; ++i)
      vu[j][i] = has_u[j] ? df_mul((j + 1 < KPL) ? ub[j + 1 < KPL ? j + 1 : 0][i] : ubn[i], ri[i]) : df_make(0.f);
  }
  dfl vxm[NX], vum[NU];
#pragma unroll
  for (int i = 0; i < NX; ++i) {
    vxm[i].hi = __shfl_up_sync(0xffffffffu, vx[KPL - 1][i].hi, 1);
    vxm[i].lo = __shfl_up_sync(0xffffffffu, vx[KPL - 1][i].lo, 1);
    if (ln == 0) vxm[i] = df_make(0.f);
  }
#pragma unroll
  for (int i = 0; i < NU; ++i) {
    vum[i].hi = __shfl_up_sync(0xffffffffu, vu[KPL - 1][i].hi, 1);
    vum[i].lo = __shfl_up_sync(0xffffffffu, vu[KPL - 1][i].lo, 1);
    if (ln == 0) vum[i] = df_make(0.f);
  }
#pragma unroll
  for (int j = 0; j < KPL; ++j)
#pragma unroll
    for (int i = 0; i < NX; ++i) {
      dacc a = dacc_zero();
      if constexpr (is_implicit<M>::value) {
#pragma unroll
        for (int q = 0; q < NX; ++q) dacc_fma(a, Apk[j][i * NX + q], vx[j][q]);
      } else {
        dacc_add(a, vx[j][i]);
      }
#pragma unroll
      for (int q = 0; q < NX; ++q) dacc_fma(a, Ak[j][i * NX + q], (j > 0) ? vx[j > 0 ? j - 1 : 0][q] : vxm[q]);
      if (has_a[j]) dacc_add(a, df_neg((j > 0) ? vx[j > 0 ? j - 1 : 0][i] : vxm[i]));
#pragma unroll
      for (int q = 0; q < NU; ++q) dacc_fma(a, Bk[j][i * NU + q], (j > 0) ? vu[j > 0 ? j - 1 : 0][q] : vum[q]);
      out[j][i] = dacc_get(a);
    }
}

template <class M, int KPL>
__device__ __noinline__ int stage_pcg_warp_df(Ctx<M, 32>& c, float eta0f, int maxit) {
  constexpr int NX = M::NX, NU = M::NU;
  const KParams& P = *c.P;
  const int K = c.K, KP = c.KP, T = c.T;
  const int ln = c.tm.lane;
  double* LP = c.Dp(c.L.d_lamp);
  const double* G = c.Dp(c.L.d_gam);
  float Pdk[KPL][NX * NX], Pok[KPL][NX * NX], Ak[KPL][NX * NX], Bk[KPL][NX * NU], Apk[KPL][NX * NX];
  dfl qi[KPL][NX], ri[NU];
  bool live[KPL], has_u[KPL], has_a[KPL];
#pragma unroll
  for (int j = 0; j < KPL; ++j) {
    const int k = ln * KPL + j;
    live[j] = k < K;
    has_u[j] = k < T;
    has_a[j] = live[j] && k > 0;
#pragma unroll
    for (int a = 0; a < NX; ++a)
#pragma unroll
      for (int b = 0; b < NX; ++b) {
        // symmetrised diagonal block: exactly symmetric operator
        const float pab = live[j] ? c.F(c.L.Pd)[(a * NX + b) * KP + k] : 0.f;
        const float pba = live[j] ? c.F(c.L.Pd)[(b * NX + a) * KP + k] : 0.f;
        Pdk[j][a * NX + b] = 0.5f * (pab + pba);
      }
#pragma unroll
    for (int e = 0; e < NX * NX; ++e) {
      Pok[j][e] = (live[j] && k > 0) ? c.F(c.L.Po)[e * KP + k] : 0.f;
      Ak[j][e] = (live[j] && k > 0) ? c.F(c.L.A)[e * KP + k] : 0.f;
    }
#pragma unroll
    for (int e = 0; e < NX * NU; ++e) Bk[j][e] = (live[j] && k > 0) ? c.F(c.L.Bm)[e * KP + k] : 0.f;
#pragma unroll
    for (int e = 0; e < NX * NX; ++e) {
      if constexpr (is_implicit<M>::value)
        Apk[j][e] = (k == 0) ? ((e / NX == e % NX) ? 1.f : 0.f) : (live[j] ? c.F(c.L.Ap)[e * KP + k] : 0.f);
      else
        Apk[j][e] = 0.f;
    }
#pragma unroll
    for (int i = 0; i < NX; ++i) qi[j][i] = live[j] ? df_from(c.qinv(k, i)) : df_make(0.f);
  }
#pragma unroll
  for (int i = 0; i < NU; ++i) ri[i] = df_from(c.rinv(i));
  // stop when eta <= tol^2 eta_0, compared in double-float
  const dfl thr = df_mulf(df_make(eta0f), P.opt.pcg_tol * P.opt.pcg_tol);
  dfl x[KPL][NX], r[KPL][NX], p[KPL][NX], y[KPL][NX], z[KPL][NX];
#pragma unroll
  for (int j = 0; j < KPL; ++j)
#pragma unroll
    for (int i = 0; i < NX; ++i) x[j][i] = live[j] ? df_from(LP[i * KP + ln * KPL + j]) : df_make(0.f);
  // r = gamma - S x, z = Phi^-1 r, p = z, eta = r^T z
  warp_S_df<M, KPL>(Ak, Bk, Apk, qi, ri, has_u, has_a, x, y, ln);
#pragma unroll
  for (int j = 0; j < KPL; ++j)
#pragma unroll
    for (int i = 0; i < NX; ++i) r[j][i] = live[j] ? df_sub(df_from(G[i * KP + ln * KPL + j]), y[j][i]) : df_make(0.f);
  warp_btmv_df<NX, KPL>(Pdk, Pok, r, z, ln);
  dacc ea = dacc_zero();
#pragma unroll
  for (int j = 0; j < KPL; ++j)
#pragma unroll
    for (int i = 0; i < NX; ++i) { p[j][i] = z[j][i]; dacc_fma(ea, r[j][i], z[j][i]); }
  dfl eta = df_warp_sum(dacc_get(ea));
  int it = 0;
  bool converged = !(eta.hi > thr.hi);
  while (!converged && it < maxit) {
    warp_S_df<M, KPL>(Ak, Bk, Apk, qi, ri, has_u, has_a, p, y, ln);
    dacc va = dacc_zero();
#pragma unroll
    for (int j = 0; j < KPL; ++j)
#pragma unroll
      for (int i = 0; i < NX; ++i) dacc_fma(va, p[j][i], y[j][i]);
    const dfl v = df_warp_sum(dacc_get(va));
    if (!(v.hi > 0.f) || !isfinite(v.hi)) { c.status |= ST_PCG_BREAKDOWN; break; }
    const dfl alpha = df_div(eta, v);
#pragma unroll
    for (int j = 0; j < KPL; ++j)
#pragma unroll
      for (int i = 0; i < NX; ++i) {
        x[j][i] = df_add(x[j][i], df_mul(alpha, p[j][i]));
        r[j][i] = df_sub(r[j][i], df_mul(alpha, y[j][i]));
      }
    warp_btmv_df<NX, KPL>(Pdk, Pok, r, z, ln);
    dacc na = dacc_zero();
#pragma unroll
    for (int j = 0; j < KPL; ++j)
#pragma unroll
      for (int i = 0; i < NX; ++i) dacc_fma(na, r[j][i], z[j][i]);
    const dfl eta_new = df_warp_sum(dacc_get(na));
    ++it;
    if (!(eta_new.hi > thr.hi)) { converged = true; break; }
    if (!isfinite(eta_new.hi)) break;
    const dfl beta = df_div(eta_new, eta);
    eta = eta_new;
#pragma unroll
    for (int j = 0; j < KPL; ++j)
#pragma unroll
      for (int i = 0; i < NX; ++i) p[j][i] = df_add(z[j][i], df_mul(beta, p[j][i]));
  }
#pragma unroll
  for (int j = 0; j < KPL; ++j)
    if (live[j])
#pragma unroll
      for (int i = 0; i < NX; ++i) LP[i * KP + ln * KPL + j] = df_to(x[j][i]);
  hp_residual<M, 32>(c, LP);  // leaves w = H^T lambda for the recovery
  if (!converged) c.status |= ST_PCG_MAXITER;
  return it;
}

// a4, single-warp variant (TEAM = 32, KPL contiguous knots per lane, K <= 32 KPL, nx <= 4):
// the same algorithm as stage_pcg (Algorithm 4 in FP32 with FP64 reliable updates and the
// double-float rescue), with the S and Phi^-1 blocks of the lane's knots in registers for the whole
// solve and every neighbour exchange and reduction done with warp shuffles: no shared memory
// and no barrier inside the iteration.
template <class M, int KPL>
__device__ __noinline__ int stage_pcg_warp(Ctx<M, 32>& c) {
  constexpr int NX = M::NX;
  const KParams& P = *c.P;
  const int K = c.K, KP = c.KP;
  const int ln = c.tm.lane;
  float* R = c.F(c.L.r);
  double* LP = c.Dp(c.L.d_lamp);
  const double* G = c.Dp(c.L.d_gam);
  const float tol2 = P.opt.pcg_tol * P.opt.pcg_tol;
  const float dl2 = P.opt.ru_delta * P.opt.ru_delta;
  float Dk[KPL][NX * NX], Ok[KPL][NX * NX], Pdk[KPL][NX * NX], Pok[KPL][NX * NX];
  bool live[KPL];
#pragma unroll
  for (int j = 0; j < KPL; ++j) {
    const int k = ln * KPL + j;
    live[j] = k < K;
#pragma unroll
    for (int e = 0; e < NX * NX; ++e) {
      Dk[j][e] = live[j] ? c.F(c.L.D)[e * KP + k] : 0.f;
      Ok[j][e] = (live[j] && k > 0) ? c.F(c.L.O)[e * KP + k] : 0.f;
      Pdk[j][e] = live[j] ? c.F(c.L.Pd)[e * KP + k] : 0.f;
      Pok[j][e] = (live[j] && k > 0) ? c.F(c.L.Po)[e * KP + k] : 0.f;
    }
  }
  // eta_0 = gamma^T Phi^-1 gamma, from the FP32-rounded gamma
  float r[KPL][NX], z[KPL][NX], p[KPL][NX], y[KPL][NX], dl[KPL][NX];
#pragma unroll
  for (int j = 0; j < KPL; ++j)
#pragma unroll
    for (int i = 0; i < NX; ++i) r[j][i] = live[j] ? (float)G[i * KP + ln * KPL + j] : 0.f;
  warp_btmv<NX, KPL>(Pdk, Pok, r, z, ln);
  float e0[1] = {0.f};
#pragma unroll
  for (int j = 0; j < KPL; ++j)
#pragma unroll
    for (int i = 0; i < NX; ++i) e0[0] = fmaf(r[j][i], z[j][i], e0[0]);
  warp_sum(e0);
  const float eta0 = e0[0];
  if (P.opt.pcg_precision == 1) {
    const int d = stage_pcg_warp_df<M, KPL>(c, eta0, P.opt.pcg_max_iters);
    c.df_iters += d;
    return d;
  }
  // true residual of the initial guess, preconditioned residual, first direction
  hp_residual<M, 32>(c, LP);
#pragma unroll
  for (int j = 0; j < KPL; ++j)
#pragma unroll
    for (int i = 0; i < NX; ++i) { r[j][i] = live[j] ? R[i * KP + ln * KPL + j] : 0.f; dl[j][i] = 0.f; }
  warp_btmv<NX, KPL>(Pdk, Pok, r, z, ln);
  float e1[1] = {0.f};
#pragma unroll
  for (int j = 0; j < KPL; ++j)
#pragma unroll
    for (int i = 0; i < NX; ++i) { p[j][i] = z[j][i]; e1[0] = fmaf(r[j][i], z[j][i], e1[0]); }
  warp_sum(e1);
  float eta = e1[0];
  float eta_ref = eta, eta_true = eta;
  int it = 0, stall = 0;
  bool converged = !(eta > tol2 * eta0);
  bool folded = true;
  const int maxit = P.opt.pcg_max_iters;
  while (!converged && it < maxit) {
    warp_btmv<NX, KPL>(Dk, Ok, p, y, ln);          // y = S p
    float v[1] = {0.f};
#pragma unroll
    for (int j = 0; j < KPL; ++j)
#pragma unroll
      for (int i = 0; i < NX; ++i) v[0] = fmaf(p[j][i], y[j][i], v[0]);
    warp_sum(v);
    if (!(v[0] > 0.f) || !isfinite(v[0])) break;
    const float alpha = __fdividef(eta, v[0]);
#pragma unroll
    for (int j = 0; j < KPL; ++j)
#pragma unroll
      for (int i = 0; i < NX; ++i) { dl[j][i] = fmaf(alpha, p[j][i], dl[j][i]); r[j][i] = fmaf(-alpha, y[j][i], r[j][i]); }
    folded = false;
    warp_btmv<NX, KPL>(Pdk, Pok, r, z, ln);        // z = Phi^-1 r
    float e2[1] = {0.f};
#pragma unroll
    for (int j = 0; j < KPL; ++j)
#pragma unroll
      for (int i = 0; i < NX; ++i) e2[0] = fmaf(r[j][i], z[j][i], e2[0]);
    warp_sum(e2);
    float eta_new = e2[0];
    ++it;
    if (eta_new < dl2 * eta_ref || !(eta_new > tol2 * eta0) || it >= maxit || !isfinite(eta_new)) {
      // reliable update: fold the FP32 correction into the FP64 solution, true residual
#pragma unroll
      for (int j = 0; j < KPL; ++j)
        if (live[j])
#pragma unroll
          for (int i = 0; i < NX; ++i) { LP[i * KP + ln * KPL + j] += (double)dl[j][i]; dl[j][i] = 0.f; }
      folded = true;
      hp_residual<M, 32>(c, LP);
#pragma unroll
      for (int j = 0; j < KPL; ++j)
#pragma unroll
        for (int i = 0; i < NX; ++i) r[j][i] = live[j] ? R[i * KP + ln * KPL + j] : 0.f;
      warp_btmv<NX, KPL>(Pdk, Pok, r, z, ln);
      float e3[1] = {0.f};
#pragma unroll
      for (int j = 0; j < KPL; ++j)
#pragma unroll
        for (int i = 0; i < NX; ++i) e3[0] = fmaf(r[j][i], z[j][i], e3[0]);
      warp_sum(e3);
      eta_new = e3[0];
      eta_ref = eta_new;
      if (!(eta_new > tol2 * eta0)) { converged = true; break; }
      if (!isfinite(eta_new)) break;
      if (eta_new > 0.25f * eta_true) {
        if (++stall >= 2) break;
      } else {
        stall = 0;
      }
      eta_true = eta_new;
      if (it >= maxit) break;
    }
    const float beta = __fdividef(eta_new, eta);
    eta = eta_new;
#pragma unroll
    for (int j = 0; j < KPL; ++j)
#pragma unroll
      for (int i = 0; i < NX; ++i) p[j][i] = fmaf(beta, p[j][i], z[j][i]);
  }
  if (!folded) {
#pragma unroll
    for (int j = 0; j < KPL; ++j)
      if (live[j])
#pragma unroll
        for (int i = 0; i < NX; ++i) LP[i * KP + ln * KPL + j] += (double)dl[j][i];
    hp_residual<M, 32>(c, LP);
  }
  if (!converged) {
    c.status |= ST_FP64_RESCUE;
    const int d = stage_pcg_warp_df<M, KPL>(c, eta0, maxit);
    c.df_iters += d;
    it += d;
  }
  return it;
}

// a4, single-warp variant with ONE reduction per iteration (pcg_variant = 1): Algorithm 4
// reorganised as Chronopoulos and Gear's conjugate gradient (1989).  In exact arithmetic it
// produces the same iterates: with u = Phi^-1 r and w = S u, the two inner products
// gamma = r^T u (Algorithm 4's eta) and delta = w^T u are formed together, beta = gamma / gamma_old,
// alpha = gamma / (delta - beta gamma / alpha_old), p = u + beta p and s = w + beta s (s = S p by
// recurrence), lambda += alpha p, r -= alpha s.  One fused warp reduction of two values replaces
// Algorithm 4's two dependent reductions, which shortens the serial chain of an iteration; the two
// block-tridiagonal products (Phi^-1 r, then S u) stay dependent.  Reliable updates, stagnation
// test and double-float rescue as in stage_pcg_warp; at each true-residual replacement s is
// recomputed as S p so the recurrence does not drift.
template <class M, int KPL>
__device__ __noinline__ int stage_pcg_warp_cg(Ctx<M, 32>& c) {
  constexpr int NX = M::NX;
  const KParams& P = *c.P;
  const int K = c.K, KP = c.KP;
  const int ln = c.tm.lane;
  float* R = c.F(c.L.r);
  double* LP = c.Dp(c.L.d_lamp);
  const double* G = c.Dp(c.L.d_gam);
  const float tol2 = P.opt.pcg_tol * P.opt.pcg_tol;
  const float dl2 = P.opt.ru_delta * P.opt.ru_delta;
  float Dk[KPL][NX * NX], Ok[KPL][NX * NX], Pdk[KPL][NX * NX], Pok[KPL][NX * NX];
  bool live[KPL];
#pragma unroll
  for (int j = 0; j < KPL; ++j) {
    const int k = ln * KPL + j;
    live[j] = k < K;
#pragma unroll
    for (int e = 0; e < NX * NX; ++e) {
      Dk[j][e] = live[j] ? c.F(c.L.D)[e * KP + k] : 0.f;
      Ok[j][e] = (live[j] && k > 0) ? c.F(c.L.O)[e * KP + k] : 0.f;
      Pdk[j][e] = live[j] ? c.F(c.L.Pd)[e * KP + k] : 0.f;
      Pok[j][e] = (live[j] && k > 0) ? c.F(c.L.Po)[e * KP + k] : 0.f;
    }
  }
  // eta_0 = gamma^T Phi^-1 gamma, from the FP32-rounded gamma
  float r[KPL][NX], u[KPL][NX], w[KPL][NX], p[KPL][NX], sv[KPL][NX], dl[KPL][NX];
#pragma unroll
  for (int j = 0; j < KPL; ++j)
#pragma unroll
    for (int i = 0; i < NX; ++i) r[j][i] = live[j] ? (float)G[i * KP + ln * KPL + j] : 0.f;
  warp_btmv<NX, KPL>(Pdk, Pok, r, u, ln);
  float e0[1] = {0.f};
#pragma unroll
  for (int j = 0; j < KPL; ++j)
#pragma unroll
    for (int i = 0; i < NX; ++i) e0[0] = fmaf(r[j][i], u[j][i], e0[0]);
  warp_sum(e0);
  const float eta0 = e0[0];
  if (P.opt.pcg_precision == 1) {
    const int d = stage_pcg_warp_df<M, KPL>(c, eta0, P.opt.pcg_max_iters);
    c.df_iters += d;
    return d;
  }
  // true residual of the initial guess; u = Phi^-1 r, w = S u, gamma = r^T u, delta = w^T u
  hp_residual<M, 32>(c, LP);
#pragma unroll
  for (int j = 0; j < KPL; ++j)
#pragma unroll
    for (int i = 0; i < NX; ++i) { r[j][i] = live[j] ? R[i * KP + ln * KPL + j] : 0.f; dl[j][i] = 0.f; }
  warp_btmv<NX, KPL>(Pdk, Pok, r, u, ln);
  warp_btmv<NX, KPL>(Dk, Ok, u, w, ln);
  float gd[2] = {0.f, 0.f};
#pragma unroll
  for (int j = 0; j < KPL; ++j)
#pragma unroll
    for (int i = 0; i < NX; ++i) { gd[0] = fmaf(r[j][i], u[j][i], gd[0]); gd[1] = fmaf(w[j][i], u[j][i], gd[1]); }
  warp_sum(gd);
  float gam = gd[0];
  float eta_ref = gam, eta_true = gam;
  int it = 0, stall = 0;
  bool converged = !(gam > tol2 * eta0);
  bool folded = true;
  const int maxit = P.opt.pcg_max_iters;
  // first direction: p = u, s = w, alpha = gamma / delta
  float alpha = __fdividef(gam, gd[1]);
#pragma unroll
  for (int j = 0; j < KPL; ++j)
#pragma unroll
    for (int i = 0; i < NX; ++i) { p[j][i] = u[j][i]; sv[j][i] = w[j][i]; }
  bool broke = !(gd[1] > 0.f) || !isfinite(gd[1]);
  while (!converged && !broke && it < maxit) {
#pragma unroll
    for (int j = 0; j < KPL; ++j)
#pragma unroll
      for (int i = 0; i < NX; ++i) { dl[j][i] = fmaf(alpha, p[j][i], dl[j][i]); r[j][i] = fmaf(-alpha, sv[j][i], r[j][i]); }
    folded = false;
    warp_btmv<NX, KPL>(Pdk, Pok, r, u, ln);        // u = Phi^-1 r
    warp_btmv<NX, KPL>(Dk, Ok, u, w, ln);          // w = S u
    float q[2] = {0.f, 0.f};
#pragma unroll
    for (int j = 0; j < KPL; ++j)
#pragma unroll
      for (int i = 0; i < NX; ++i) { q[0] = fmaf(r[j][i], u[j][i], q[0]); q[1] = fmaf(w[j][i], u[j][i], q[1]); }
    warp_sum(q);
    float gam_new = q[0], del = q[1];
    ++it;
    bool recompute_s = false;
    if (gam_new < dl2 * eta_ref || !(gam_new > tol2 * eta0) || it >= maxit || !isfinite(gam_new)) {
      // reliable update: fold the FP32 correction into the FP64 solution, true residual
#pragma unroll
      for (int j = 0; j < KPL; ++j)
        if (live[j])
#pragma unroll
          for (int i = 0; i < NX; ++i) { LP[i * KP + ln * KPL + j] += (double)dl[j][i]; dl[j][i] = 0.f; }
      folded = true;
      hp_residual<M, 32>(c, LP);
#pragma unroll
      for (int j = 0; j < KPL; ++j)
#pragma unroll
        for (int i = 0; i < NX; ++i) r[j][i] = live[j] ? R[i * KP + ln * KPL + j] : 0.f;
      warp_btmv<NX, KPL>(Pdk, Pok, r, u, ln);
      warp_btmv<NX, KPL>(Dk, Ok, u, w, ln);
      float q2[2] = {0.f, 0.f};
#pragma unroll
      for (int j = 0; j < KPL; ++j)
#pragma unroll
        for (int i = 0; i < NX; ++i) { q2[0] = fmaf(r[j][i], u[j][i], q2[0]); q2[1] = fmaf(w[j][i], u[j][i], q2[1]); }
      warp_sum(q2);
      gam_new = q2[0];
      del = q2[1];
      eta_ref = gam_new;
      if (!(gam_new > tol2 * eta0)) { converged = true; break; }
      if (!isfinite(gam_new)) break;
      if (gam_new > 0.25f * eta_true) {
        if (++stall >= 2) break;
      } else {
        stall = 0;
      }
      eta_true = gam_new;
      if (it >= maxit) break;
      recompute_s = true;
    }
    const float beta = __fdividef(gam_new, gam);
    const float den = del - beta * __fdividef(gam_new, alpha);
    if (!(den > 0.f) || !isfinite(den)) break;
    alpha = __fdividef(gam_new, den);
    gam = gam_new;
#pragma unroll
    for (int j = 0; j < KPL; ++j)
#pragma unroll
      for (int i = 0; i < NX; ++i) { p[j][i] = fmaf(beta, p[j][i], u[j][i]); sv[j][i] = fmaf(beta, sv[j][i], w[j][i]); }
    if (recompute_s) {
      // s = S p exactly after a residual replacement, and alpha from it (Algorithm 4's form)
      warp_btmv<NX, KPL>(Dk, Ok, p, sv, ln);
      float v[1] = {0.f};
#pragma unroll
      for (int j = 0; j < KPL; ++j)
#pragma unroll
        for (int i = 0; i < NX; ++i) v[0] = fmaf(p[j][i], sv[j][i], v[0]);
      warp_sum(v);
      if (!(v[0] > 0.f) || !isfinite(v[0])) break;
      alpha = __fdividef(gam, v[0]);
    }
  }
  if (!folded) {
#pragma unroll
    for (int j = 0; j < KPL; ++j)
      if (live[j])
#pragma unroll
        for (int i = 0; i < NX; ++i) LP[i * KP + ln * KPL + j] += (double)dl[j][i];
    hp_residual<M, 32>(c, LP);
  }
  if (!converged) {
    c.status |= ST_FP64_RESCUE;
    const int d = stage_pcg_warp_df<M, KPL>(c, eta0, maxit);
    c.df_iters += d;
    it += d;
  }
  return it;
}

// PCG entry: the register-resident inner loop when one knot per lane fits (nx <= 6).
}  // namespace dmpc
#include "dpcg.cuh"
namespace dmpc {

// Leader side of the distributed PCG: hand the solve to every CTA of the cluster and take part in
// it (a stagnated solve is finished by the cluster's double-float rescue).
template <class M>
__device__ __noinline__ int stage_pcg_cluster(Ctx<M, kClThreads>& c) {
  ClRun<M>& r = *c.cl;
  cl_command<M>(r, CL_PCG, c.ocp, c.K, c.T, c.cl_form ? 1 : 0);
  const ClResult res = cl_pcg<M>(r, *c.P, c.K, c.T, c.fb, c.cl_form);
  __threadfence();
  int it = res.it;
  if (r.broken) {
    c.status |= ST_SYNC_TIMEOUT;
    return it;
  }
  if (res.chol_fail) c.status |= ST_CHOL_FAIL;
  if (!res.converged) {   // finished by the cluster's double-float rescue
    c.status |= ST_FP64_RESCUE;
    if (res.df_breakdown) c.status |= ST_PCG_BREAKDOWN;
    if (!res.df_converged) c.status |= ST_PCG_MAXITER;
    c.df_iters += res.df_it;
    it += res.df_it;
  }
  return it;
}

// Whether this OCP's PCG solves run on its thread-block cluster.
template <class M, int TEAM>
__device__ __forceinline__ bool cl_active(const Ctx<M, TEAM>& c) {
  if constexpr (kClusterPcg && TEAM == kClThreads && M::NX % kClRows == 0 && !is_implicit<M>::value)
    return c.cl != nullptr && !c.cl->broken;
  return false;
}

template <class M, int TEAM>
__device__ __forceinline__ int run_pcg(Ctx<M, TEAM>& c) {
  if constexpr (kClusterPcg && TEAM == kClThreads && M::NX % kClRows == 0 && !is_implicit<M>::value) {
    if (cl_active(c)) return stage_pcg_cluster<M>(c);
  }
  if constexpr (M::NX <= 4) {
    if constexpr (TEAM == 32) {
      if (c.P->opt.pcg_variant == 1) {
        if (c.K <= 32) return stage_pcg_warp_cg<M, 1>(c);
        if (c.K <= 64) return stage_pcg_warp_cg<M, 2>(c);
      }
      if (c.K <= 32) return stage_pcg_warp<M, 1>(c);
      if (c.K <= 64) return stage_pcg_warp<M, 2>(c);
    } else {
      if (c.K <= TEAM) return stage_pcg_reg<M, TEAM>(c);
    }
  } else if constexpr (M::NX <= 6 && TEAM > 32) {
    if (c.K <= TEAM) return stage_pcg_reg<M, TEAM>(c);
  }
  return stage_pcg<M, TEAM>(c);
}

// a5: primal recovery (Eq. 11) from lamp and w = H^T lamp (left by the last hp_residual):
// x_k = -Q_k^-1 (q_k + w_x,k), u_k = -R^-1 (r_k + w_u,k).  Writes float z+ (xp, up).
template <class M, int TEAM>
__device__ __noinline__ void stage_recover(Ctx<M, TEAM>& c) {
  constexpr int NX = M::NX, NU = M::NU;
  const int T = c.T, K = c.K, KP = c.KP;
  const float* X = c.F(c.L.x);
  const float* U = c.F(c.L.u);
  float* XP = c.F(c.L.xp);
  float* UP = c.F(c.L.up);
  const double* WX = c.Dp(c.L.d_wx);
  const double* WU = c.Dp(c.L.d_wu);
  for (int k = c.tm.lane; k < K; k += TEAM) {
#pragma unroll
    for (int i = 0; i < NX; ++i)
      XP[i * KP + k] = (float)(-(c.qlin(k, i, X[i * KP + k]) + WX[i * KP + k]) * c.qinv(k, i));
    if (k < T) {
#pragma unroll
      for (int i = 0; i < NU; ++i)
        UP[i * KP + k] = (float)(-(c.rlin(i, U[i * KP + k]) + WU[i * KP + k]) * c.rinv(i));
    }
  }
  c.tm.sync();
}

template <class M>
__device__ __forceinline__ void plain_step(const float* tk_lq, const float* pv, float dt, const float* x,
                                           const float* u, float* xn) {
  if constexpr (is_lq<M>::value) {
    constexpr int NX = M::NX, NU = M::NU;
#pragma unroll
    for (int i = 0; i < NX; ++i) {
      float acc = tk_lq[NX * NX + NX * NU + i];
#pragma unroll
      for (int j = 0; j < NX; ++j) acc = fmaf(tk_lq[i * NX + j], x[j], acc);
#pragma unroll
      for (int j = 0; j < NU; ++j) acc = fmaf(tk_lq[NX * NX + i * NU + j], u[j], acc);
      xn[i] = acc;
    }
  } else {
    model_step<M>(x, u, pv, dt, xn);
  }
}

// a6: line search (Algorithm 5; merit Eq. 12, penalty Eq. 13, decrease Eq. 14, descent
// Eq. 15) over the alpha set, then z <- z + alpha (z+ - z), lambda <- lambda + alpha
// (lambda+ - lambda).  Cost differences use the exact quadratic expansion, so no large
// cost values are subtracted.  Returns alpha.
template <class M, int TEAM>
__device__ __noinline__ float stage_linesearch(Ctx<M, TEAM>& c) {
  constexpr int NX = M::NX, NU = M::NU;
  const KParams& P = *c.P;
  const int T = c.T, K = c.K, KP = c.KP;
  float* X = c.F(c.L.x);
  float* U = c.F(c.L.u);
  const float* XP = c.F(c.L.xp);
  const float* UP = c.F(c.L.up);
  const float* Fv = c.F(c.L.f);
  double* LAM = c.Dp(c.L.d_lam);
  const double* LP = c.Dp(c.L.d_lamp);
  const int na = P.opt.line_search ? P.opt.n_alpha : 0;
  float alpha = 1.f;
  if (na > 0) {
    const float* xs = P.x_s + c.o.xs_off;
    float pv[M::NP > 0 ? M::NP : 1];
#pragma unroll
    for (int j = 0; j < M::NP; ++j) pv[j] = c.misc(MS_TH + j);
    // red: [num, g0, xabs, dc_0..dc_7, g_0..g_7]
    double red[19];
#pragma unroll
    for (int j = 0; j < 19; ++j) red[j] = 0.0;
    for (int k = c.tm.lane; k < K; k += TEAM) {
      double num = 0.0, quad = 0.0;
#pragma unroll
      for (int i = 0; i < NX; ++i) {
        const double xk = X[i * KP + k], dx = (double)XP[i * KP + k] - xk;
        const double w = c.qraw(k, i);
        num += w * (xk - (double)c.xref(k, i)) * dx;
        quad += w * dx * dx;
        red[1] += fabs((double)Fv[i * KP + k]);
        red[2] += fabs(xk);
      }
      if (k < T) {
#pragma unroll
        for (int i = 0; i < NU; ++i) {
          const double uk = U[i * KP + k], du = (double)UP[i * KP + k] - uk;
          const double w = c.misc(MS_R + i);
          num += w * uk * du;
          quad += w * du * du;
        }
      }
      red[0] += num;
      const float* tk = nullptr;
      if constexpr (is_lq<M>::value) {
        if (k > 0) tk = P.theta + c.o.th_off + (long long)(k - 1) * M::PK;
      }
      for (int j = 0; j < na; ++j) {
        const float a = P.opt.alpha[j];
        red[3 + j] += (double)a * num + 0.5 * (double)a * (double)a * quad;
        double g = 0.0;
        if (k == 0) {
#pragma unroll
          for (int i = 0; i < NX; ++i) g += fabs((double)(X[i * KP] + a * (XP[i * KP] - X[i * KP])) - (double)xs[i]);
        } else {
          const int t = k - 1;
          float xa[NX], ua[NU], xn[NX];
#pragma unroll
          for (int i = 0; i < NX; ++i) xa[i] = X[i * KP + t] + a * (XP[i * KP + t] - X[i * KP + t]);
#pragma unroll
          for (int i = 0; i < NU; ++i) ua[i] = U[i * KP + t] + a * (UP[i * KP + t] - U[i * KP + t]);
          if constexpr (is_implicit<M>::value) {
#pragma unroll
            for (int i = 0; i < NX; ++i) xn[i] = X[i * KP + k] + a * (XP[i * KP + k] - X[i * KP + k]);
            float rr[NX];
            trap_residual<M>(xa, ua, xn, pv, c.dt, rr);
#pragma unroll
            for (int i = 0; i < NX; ++i) g += fabs((double)rr[i]);
          } else if constexpr (is_lq<M>::value) {
            plain_step<M>(tk, pv, c.dt, xa, ua, xn);
#pragma unroll
            for (int i = 0; i < NX; ++i)
              g += fabs((double)(X[i * KP + k] + a * (XP[i * KP + k] - X[i * KP + k])) - (double)xn[i]);
          } else {
            // f_t = (x_{t+1} - x_t) - (Phi - x_t), the increment formed without adding x_t
            model_increment<M>(xa, ua, pv, c.dt, xn);
#pragma unroll
            for (int i = 0; i < NX; ++i)
              g += fabs((double)((X[i * KP + k] + a * (XP[i * KP + k] - X[i * KP + k])) - xa[i]) - (double)xn[i]);
          }
        }
        red[11 + j] += g;
      }
    }
    c.tm.sum(red);
    const double num = red[0], g0 = red[1], xabs = red[2];
    const bool feasible = g0 <= (double)P.opt.feas_tol * ((double)(K * NX) + xabs);
    const double mu = feasible ? 0.0 : fmax(num, 0.0) / (0.5 * g0);
    const double Dmu = num - mu * g0;
    float amin = P.opt.alpha[0];
    for (int j = 0; j < na; ++j) amin = fminf(amin, P.opt.alpha[j]);
    alpha = amin;
    bool found = false;
    for (int j = 0; j < na; ++j) {
      const double a = P.opt.alpha[j];
      const double dphi = red[3 + j] + mu * (red[11 + j] - g0) - (double)P.opt.ls_eta * a * Dmu;
      if (dphi < 0.0) { alpha = P.opt.alpha[j]; found = true; break; }
    }
    if (!found) c.status |= ST_LS_MINSTEP;
    c.tm.sync();
  }
  for (int k = c.tm.lane; k < K; k += TEAM) {
#pragma unroll
    for (int i = 0; i < NX; ++i) {
      X[i * KP + k] += alpha * (XP[i * KP + k] - X[i * KP + k]);
      LAM[i * KP + k] += (double)alpha * (LP[i * KP + k] - LAM[i * KP + k]);
    }
    if (k < T) {
#pragma unroll
      for (int i = 0; i < NU; ++i) U[i * KP + k] += alpha * (UP[i * KP + k] - U[i * KP + k]);
    }
  }
  c.tm.sync();
  return alpha;
}

template <class M, int TEAM>
__device__ void copy_lam_to_lamp(Ctx<M, TEAM>& c) {
  constexpr int NX = M::NX;
  const double* LAM = c.Dp(c.L.d_lam);
  double* LP = c.Dp(c.L.d_lamp);
  for (int k = c.tm.lane; k < c.K; k += TEAM)
#pragma unroll
    for (int i = 0; i < NX; ++i) LP[i * c.KP + k] = LAM[i * c.KP + k];
  c.tm.sync();
}

// Write the stored-Schur record of this OCP (A, B, D, O, Pd, Po at the returned z).
template <class M, int TEAM>
__device__ __noinline__ void store_blocks(Ctx<M, TEAM>& c, bool load) {
  constexpr int NX = M::NX, NU = M::NU;
  float* dst = c.P->store + c.o.gws_off;
  const int K = c.K, KP = c.KP;
  const int offs[6] = {c.L.A, c.L.Bm, c.L.D, c.L.O, c.L.Pd, c.L.Po};
  const int sizes[6] = {NX * NX, NX * NU, NX * NX, NX * NX, NX * NX, NX * NX};
  long long base = 0;
  for (int a = 0; a < 6; ++a) {
    float* w = c.F(offs[a]);
    for (int e = 0; e < sizes[a]; ++e) {
      for (int k = c.tm.lane; k < K; k += TEAM) {
        if (load) w[e * KP + k] = dst[base + (long long)e * K + k];
        else dst[base + (long long)e * K + k] = w[e * KP + k];
      }
    }
    base += (long long)sizes[a] * K;
  }
  c.tm.sync();
}

template <class M, int TEAM>
__device__ __noinline__ void write_inspect(Ctx<M, TEAM>& c, int iters) {
  constexpr int NX = M::NX, NU = M::NU, NZ = NX + NU;
  const int T = c.T, K = c.K, KP = c.KP;
  float* out = c.P->inspect + c.P->inspect_off[c.ocp];
  // record: A (T nx nx), B (T nx nu), C (T nx), f (K nx), D, O, Pd, Po (K nx nx each),
  // gamma (K nx), lambda+ (K nx), z+ (n), pcg iterations (1), of them in the double-float
  // rescue (1); knot-major, row-major blocks
  long long o = 0;
  for (int k = c.tm.lane; k < K; k += TEAM) {
    if (k >= 1) {
      const int t = k - 1;
      for (int e = 0; e < NX * NX; ++e)
        out[o + (long long)t * NX * NX + e] = c.F(c.L.A)[e * KP + k] - ((e / NX) == (e % NX) ? 1.f : 0.f);
      for (int e = 0; e < NX * NU; ++e) out[o + (long long)T * NX * NX + (long long)t * NX * NU + e] = c.F(c.L.Bm)[e * KP + k];
      for (int e = 0; e < NX; ++e) out[o + (long long)T * (NX * NX + NX * NU) + (long long)t * NX + e] = c.F(c.L.C)[e * KP + k];
    }
  }
  o += (long long)T * (NX * NX + NX * NU + NX);
  const int blks[4] = {c.L.D, c.L.O, c.L.Pd, c.L.Po};
  for (int k = c.tm.lane; k < K; k += TEAM) {
    for (int e = 0; e < NX; ++e) out[o + (long long)k * NX + e] = c.F(c.L.f)[e * KP + k];
    for (int b = 0; b < 4; ++b)
      for (int e = 0; e < NX * NX; ++e)
        out[o + (long long)K * NX + (long long)b * K * NX * NX + (long long)k * NX * NX + e] = c.F(blks[b])[e * KP + k];
    const long long og = o + (long long)K * NX + 4LL * K * NX * NX;
    for (int e = 0; e < NX; ++e) {
      out[og + (long long)k * NX + e] = (float)c.Dp(c.L.d_gam)[e * KP + k];
      out[og + (long long)K * NX + (long long)k * NX + e] = (float)c.Dp(c.L.d_lamp)[e * KP + k];
    }
    const long long oz = og + 2LL * K * NX;
    for (int e = 0; e < NX; ++e) out[oz + (long long)k * NZ + e] = c.F(c.L.xp)[e * KP + k];
    if (k < T)
      for (int e = 0; e < NU; ++e) out[oz + (long long)k * NZ + NX + e] = c.F(c.L.up)[e * KP + k];
    if (k == 0) {
      out[oz + (long long)K * NX + (long long)T * NU] = (float)iters;
      out[oz + (long long)K * NX + (long long)T * NU + 1] = (float)c.df_iters;
    }
  }
}

// Forward outputs: optional stored blocks at the returned z, then z, lambda, the resident
// warm-start copies and the status.
template <class M, int TEAM>
__device__ __noinline__ void stage_fwd_outputs(Ctx<M, TEAM>& c) {
  constexpr int NX = M::NX, NU = M::NU, NZ = NX + NU;
  const KParams& P = *c.P;
  const int T = c.T, K = c.K, KP = c.KP;
  if (P.store_mode && P.store) {
    // stored-Schur mode: re-linearise at the returned z and keep the blocks for the vjp
    stage_linearise<M, TEAM>(c);
    stage_schur<M, TEAM>(c, false);
    stage_precond<M, TEAM>(c);
    store_blocks<M, TEAM>(c, false);
  }
  const float* X = c.F(c.L.x);
  const float* U = c.F(c.L.u);
  const double* LAM = c.Dp(c.L.d_lam);
  int bad = 0;
  for (int k = c.tm.lane; k < K; k += TEAM) {
    const long long zb = c.o.z_off + (long long)k * NZ;
    const long long lb = c.o.lam_off + (long long)k * NX;
#pragma unroll
    for (int i = 0; i < NX; ++i) {
      const float xv = X[i * KP + k];
      bad |= !isfinite(xv);
      P.z_out[zb + i] = xv;
      if (P.res_z) P.res_z[zb + i] = xv;
      const double lv = LAM[i * KP + k];
      bad |= !isfinite(lv);
      if (P.lam_out) P.lam_out[lb + i] = (float)lv;
      if (P.res_lam) P.res_lam[lb + i] = lv;
    }
    if (k < T) {
#pragma unroll
      for (int i = 0; i < NU; ++i) {
        const float uv = U[i * KP + k];
        bad |= !isfinite(uv);
        P.z_out[zb + NX + i] = uv;
        if (P.res_z) P.res_z[zb + NX + i] = uv;
      }
    }
  }
  if (bad) c.status |= ST_NONFINITE;
  c.status = c.tm.bor(c.status);
  if (c.tm.lane == 0 && P.status) P.status[c.ocp] = c.status;
}

// ---------------------------------------------------------------------------------------
// Forward: the SQP iterations of one OCP (or one QP in inspect mode).
template <class M, int TEAM>
__device__ void run_forward(Ctx<M, TEAM>& c) {
  constexpr int NX = M::NX, NU = M::NU, NZ = NX + NU;
  const KParams& P = *c.P;
  const int T = c.T, K = c.K, KP = c.KP;
  stage_load<M, TEAM>(c, P.z_init != nullptr);
  const int iters = (P.mode == MODE_INSPECT) ? 1 : P.opt.sqp_iters;
  for (int s = 0; s < iters; ++s) {
    const bool clf = cl_active(c);   // the cluster PCG forms the blocks (a2, a3) itself
    stage_linearise<M, TEAM>(c);
    stage_schur<M, TEAM>(c, true, !clf);
    if (!clf) stage_precond<M, TEAM>(c);
    copy_lam_to_lamp<M, TEAM>(c);
    c.cl_form = clf;
    const int it = run_pcg<M, TEAM>(c);
    c.cl_form = false;
    stage_recover<M, TEAM>(c);
    if (P.mode == MODE_INSPECT) { write_inspect<M, TEAM>(c, it); break; }
    const float a = stage_linesearch<M, TEAM>(c);
    if (c.tm.lane == 0) {
      if (P.pcg_iters) P.pcg_iters[(long long)c.ocp * P.opt.sqp_iters + s] = it;
      if (P.alpha_hist) P.alpha_hist[(long long)c.ocp * P.opt.sqp_iters + s] = a;
    }
  }
  if (P.mode == MODE_INSPECT) return;
  stage_fwd_outputs<M, TEAM>(c);
}

// Backward right-hand side (Eq. 7 with (-b, d) <- (dl/dz, 0)): gamma~_spd = H G^-1 dl/dz,
// and the adjoint PCG's initial guess (the previous adjoint multipliers or 0).
template <class M, int TEAM>
__device__ __noinline__ void stage_bwd_rhs(Ctx<M, TEAM>& c) {
  constexpr int NX = M::NX, NU = M::NU, NZ = NX + NU;
  const KParams& P = *c.P;
  const int K = c.K, KP = c.KP;
  const float* g = P.dl_dz + c.o.z_off;
  const float* A = c.F(c.L.A);
  const float* Bm = c.F(c.L.Bm);
  double* G = c.Dp(c.L.d_gam);
  double* LP = c.Dp(c.L.d_lamp);
  const int T = c.T;
  for (int k = c.tm.lane; k < K; k += TEAM) {
    double s[NX], su[NU];
    float gx[NX], gu[NU];
#pragma unroll
    for (int i = 0; i < NX; ++i) gx[i] = g[(long long)k * NZ + i];
#pragma unroll
    for (int i = 0; i < NU; ++i) gu[i] = (k < T) ? g[(long long)k * NZ + NX + i] : 0.f;
    c.ginv(k, gx, gu, s, su);
    if constexpr (is_implicit<M>::value) {
      if (k > 0) {  // row k's coefficient of x_k is A^+ (slot k)
        const float* Ap = c.F(c.L.Ap);
        double s2[NX];
#pragma unroll
        for (int i = 0; i < NX; ++i) {
          double acc = 0.0;
#pragma unroll
          for (int j = 0; j < NX; ++j) acc += (double)Ap[(i * NX + j) * KP + k] * s[j];
          s2[i] = acc;
        }
#pragma unroll
        for (int i = 0; i < NX; ++i) s[i] = s2[i];
      }
    }
    if (k > 0) {
      const int t = k - 1;
      double vx[NX], vu[NU];
#pragma unroll
      for (int j = 0; j < NX; ++j) gx[j] = g[(long long)t * NZ + j];
#pragma unroll
      for (int j = 0; j < NU; ++j) gu[j] = g[(long long)t * NZ + NX + j];
      c.ginv(t, gx, gu, vx, vu);
#pragma unroll
      for (int i = 0; i < NX; ++i) {
        s[i] -= vx[i];   // A_t = (stored A_t + I) - I
#pragma unroll
        for (int j = 0; j < NX; ++j) s[i] += (double)A[(i * NX + j) * KP + k] * vx[j];
#pragma unroll
        for (int j = 0; j < NU; ++j) s[i] += (double)Bm[(i * NU + j) * KP + k] * vu[j];
      }
    }
    const long long lb = c.o.lam_off + (long long)k * NX;
#pragma unroll
    for (int i = 0; i < NX; ++i) {
      G[i * KP + k] = s[i];
      LP[i * KP + k] = P.lamt_init ? P.lamt_init[lb + i] : 0.0;
    }
  }
  c.tm.sync();
}

// Backward finish: z~ = G^-1 (dl/dz - H^T lambda~) (Eq. 11 form), then
// dl/dtheta = -(dF/dtheta)^T [z~; lambda~] contracted per knot (Eq. 3), dl/dx_s = lambda~_0.
template <class M, int TEAM>
__device__ __noinline__ void stage_bwd_finish(Ctx<M, TEAM>& c, int it) {
  constexpr int NX = M::NX, NU = M::NU, NZ = NX + NU, NP = M::NP;
  const KParams& P = *c.P;
  const int T = c.T, K = c.K, KP = c.KP;
  const float* g = P.dl_dz + c.o.z_off;
  double* LP = c.Dp(c.L.d_lamp);
  // z~ = G^-1 (dl/dz - H^T lambda~)  (stored in xp, up)
  const double* WX = c.Dp(c.L.d_wx);
  const double* WU = c.Dp(c.L.d_wu);
  float* XT = c.F(c.L.xp);
  float* UT = c.F(c.L.up);
  for (int k = c.tm.lane; k < K && !c.exact; k += TEAM) {  // exact Hessian: the Riccati solve wrote z~
    double dx[NX], du[NU], vx[NX], vu[NU];
#pragma unroll
    for (int i = 0; i < NX; ++i) dx[i] = (double)g[(long long)k * NZ + i] - WX[i * KP + k];
#pragma unroll
    for (int i = 0; i < NU; ++i) du[i] = (k < T) ? (double)g[(long long)k * NZ + NX + i] - WU[i * KP + k] : 0.0;
    c.ginv(k, dx, du, vx, vu);
#pragma unroll
    for (int i = 0; i < NX; ++i) XT[i * KP + k] = (float)vx[i];
    if (k < T) {
#pragma unroll
      for (int i = 0; i < NU; ++i) UT[i * KP + k] = (float)vu[i];
    }
  }
  c.tm.sync();
  // theta contraction: dl/dtheta = -(dF/dtheta)^T [z~; lambda~]
  const float* X = c.F(c.L.x);
  const float* U = c.F(c.L.u);
  const double* LAM = c.Dp(c.L.d_lam);
  constexpr int NR = NP + NX + NU + NX;
  float red[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) red[j] = 0.f;
  float* dth = P.dl_dtheta + c.o.th_off;
  int pk = 0;
  if constexpr (is_lq<M>::value) pk = M::PK;
  const int oq = NP + T * pk;
  for (int k = c.tm.lane; k < K; k += TEAM) {
    // cost part: grad c^x = Q (x - xref), grad c^u = R u
#pragma unroll
    for (int i = 0; i < NX; ++i) {
      const float v = XT[i * KP + k] * (X[i * KP + k] - c.xref(k, i));
      if (k < T) red[NP + i] -= v; else red[NP + NX + NU + i] -= v;
    }
    if (k < T) {
#pragma unroll
      for (int i = 0; i < NU; ++i) red[NP + NX + i] -= UT[i * KP + k] * U[i * KP + k];
    }
    if (k == 0) continue;
    const int t = k - 1;
    if constexpr (is_lq<M>::value) {
      float* dk = dth + (long long)t * M::PK;
#pragma unroll
      for (int i = 0; i < NX; ++i) {
        const float li = (float)LAM[i * KP + k], lti = (float)LP[i * KP + k];
#pragma unroll
        for (int j = 0; j < NX; ++j) dk[i * NX + j] = li * XT[j * KP + t] + lti * X[j * KP + t];
#pragma unroll
        for (int j = 0; j < NU; ++j) dk[NX * NX + i * NU + j] = li * UT[j * KP + t] + lti * U[j * KP + t];
        dk[NX * NX + NX * NU + i] = lti;
      }
    } else if constexpr (is_implicit<M>::value) {
      // f_t = x_{t+1} - x_t - h (F(x_t, u_t) + F(x_{t+1}, u_t)), h = dt/2: the contraction
      // -(lambda^T f_{z theta} z~ + lambda~^T f_theta) = h sum over both evaluations of F
      HDual<NP> xa[NX], xb[NX], uh[NU], ph[NP], fa[NX], fb[NX];
#pragma unroll
      for (int i = 0; i < NX; ++i) {
        xa[i] = HDual<NP>(X[i * KP + t]); xa[i].e = XT[i * KP + t];
        xb[i] = HDual<NP>(X[i * KP + k]); xb[i].e = XT[i * KP + k];
      }
#pragma unroll
      for (int i = 0; i < NU; ++i) { uh[i] = HDual<NP>(U[i * KP + t]); uh[i].e = UT[i * KP + t]; }
#pragma unroll
      for (int j = 0; j < NP; ++j) { ph[j] = HDual<NP>(c.misc(MS_TH + j)); ph[j].t[j] = 1.f; }
      M::f(xa, uh, ph, fa);
      M::f(xb, uh, ph, fb);
      const float h = 0.5f * c.dt;
#pragma unroll
      for (int i = 0; i < NX; ++i) {
        const float li = h * (float)LAM[i * KP + k], lti = h * (float)LP[i * KP + k];
#pragma unroll
        for (int j = 0; j < NP; ++j)
          red[j] = fmaf(li, fa[i].et[j] + fb[i].et[j], fmaf(lti, fa[i].t[j] + fb[i].t[j], red[j]));
      }
    } else {
      HDual<NP> xh[NX], uh[NU], ph[NP], out[NX];
#pragma unroll
      for (int i = 0; i < NX; ++i) { xh[i] = HDual<NP>(X[i * KP + t]); xh[i].e = XT[i * KP + t]; }
#pragma unroll
      for (int i = 0; i < NU; ++i) { uh[i] = HDual<NP>(U[i * KP + t]); uh[i].e = UT[i * KP + t]; }
#pragma unroll
      for (int j = 0; j < NP; ++j) { ph[j] = HDual<NP>(c.misc(MS_TH + j)); ph[j].t[j] = 1.f; }
      model_step<M>(xh, uh, ph, c.dt, out);
#pragma unroll
      for (int i = 0; i < NX; ++i) {
        const float li = (float)LAM[i * KP + k], lti = (float)LP[i * KP + k];
#pragma unroll
        for (int j = 0; j < NP; ++j) red[j] = fmaf(li, out[i].et[j], fmaf(lti, out[i].t[j], red[j]));
      }
    }
  }
  c.tm.sum(red);
  c.status = c.tm.bor(c.status);
  if (c.tm.lane == 0) {
#pragma unroll
    for (int j = 0; j < NP; ++j) dth[j] = red[j];
#pragma unroll
    for (int i = 0; i < NX; ++i) { dth[oq + i] = red[NP + i]; dth[oq + NX + NU + i] = red[NP + NX + NU + i]; }
#pragma unroll
    for (int i = 0; i < NU; ++i) dth[oq + NX + i] = red[NP + NX + i];
    if (P.status) P.status[c.ocp] = c.status;
    if (P.pcg_iters) P.pcg_iters[c.ocp] = it;
  }
  for (int k = c.tm.lane; k < K; k += TEAM) {
    const long long lb = c.o.lam_off + (long long)k * NX;
#pragma unroll
    for (int i = 0; i < NX; ++i) {
      const double v = LP[i * KP + k];
      if (k == 0) P.dl_dxs[c.o.xs_off + i] = (float)v;   // dl/dx_s = lambda~_0
      if (P.lamt_out) P.lamt_out[lb + i] = (float)v;
      if (P.res_lamt) P.res_lamt[lb + i] = v;
    }
  }
}

// Backward (Algorithm 3): adjoint PCG with the same S, z~, and the theta contraction.
template <class M, int TEAM>
__device__ __noinline__ void run_backward(Ctx<M, TEAM>& c) {
  const KParams& P = *c.P;
  stage_load<M, TEAM>(c, true);   // z (returned solution) and lambda (forward multipliers)
  if (c.exact) {
    stage_linearise<M, TEAM>(c);
    stage_exact_hessian<M, TEAM>(c);
    stage_riccati_exact<M, TEAM>(c);
    if (!(c.status & ST_HESS_INDEF)) {
      stage_bwd_finish<M, TEAM>(c, 0);
      return;
    }
    // the exact reduced Hessian is not positive definite at some knot (the point is not a strict
    // local minimum in the exact second-order sense): this OCP gets the Gauss-Newton gradient,
    // flagged, from the linearisation already in the workspace
    c.exact = false;
    const bool clf = cl_active(c);
    stage_schur<M, TEAM>(c, false, !clf);
    if (!clf) stage_precond<M, TEAM>(c);
    stage_bwd_rhs<M, TEAM>(c);
    c.cl_form = clf;
    const int it = run_pcg<M, TEAM>(c);
    c.cl_form = false;
    stage_bwd_finish<M, TEAM>(c, it);
    return;
  }
  bool clf = false;
  if (P.store_mode && P.store && !is_implicit<M>::value) {  // stored records carry no A^+
    store_blocks<M, TEAM>(c, true);
  } else {
    clf = cl_active(c);
    stage_linearise<M, TEAM>(c);
    stage_schur<M, TEAM>(c, false, !clf);
    if (!clf) stage_precond<M, TEAM>(c);
  }
  stage_bwd_rhs<M, TEAM>(c);
  c.cl_form = clf;
  const int it = run_pcg<M, TEAM>(c);
  c.cl_form = false;
  stage_bwd_finish<M, TEAM>(c, it);
}

template <class M, int TEAM>
__device__ void run_one(const KParams& P, int ocp, float* ws, int lane, int team_in_block, ClRun<M>* cl = nullptr) {
  Ctx<M, TEAM> c;
  c.cl = cl;
  c.P = &P;
  c.o = P.ocps[ocp];
  c.ocp = ocp;
  c.T = c.o.T;
  c.K = c.o.T + 1;
  c.dt = c.o.dt;
  c.L = make_layout(M::NX, M::NU, c.K, TEAM, P.opt.exact_hessian, is_implicit<M>::value ? 1 : 0);
  c.KP = c.L.KP;
  c.db = reinterpret_cast<double*>(ws);
  c.fb = ws;
  c.status = 0;
  c.df_iters = 0;
  c.exact = !is_lq<M>::value && !is_implicit<M>::value && P.opt.exact_hessian && P.mode == MODE_VJP;
  c.tm.lane = lane;
  c.tm.bar_id = team_in_block + 1;
  c.tm.red = ws + c.L.red;
  c.tm.buf = 0;
  if (P.mode == MODE_VJP) run_backward<M, TEAM>(c);
  else run_forward<M, TEAM>(c);
}

template <int TEAM, class... Ms>
__device__ __forceinline__ void dispatch(const KParams& P, int ocp, float* ws, int lane, int tib) {
  const OcpRec& o = P.ocps[ocp];
  bool done = ((o.model == Ms::ID && o.nx == Ms::NX && o.nu == Ms::NU
                    ? (run_one<Ms, TEAM>(P, ocp, ws, lane, tib), true)
                    : false) || ...);
  (void)done;
}

// One launch processes the work list: team g takes items g, g + G, g + 2G, ... (the list
// is sorted heaviest first, so this is a longest-processing-time-first assignment).
template <int TEAM, class... Ms>
__global__ void __launch_bounds__(256, 1) fused_kernel(const __grid_constant__ KParams P) {
  extern __shared__ __align__(16) float smem[];
  const int tib = threadIdx.x / TEAM;
  const int lane = threadIdx.x % TEAM;
  const int gteam = blockIdx.x * P.teams_per_block + tib;
  const int nteams = gridDim.x * P.teams_per_block;
  float* ws = P.use_gws ? P.gws + (size_t)gteam * P.ws_floats : smem + (size_t)tib * P.ws_floats;
  for (int w = gteam; w < P.n_work; w += nteams) dispatch<TEAM, Ms...>(P, P.order[w], ws, lane, tib);
}

#ifdef DMPC_CLUSTER_PCG
// One cluster of CTAs per OCP (persistent over the work list: cluster g takes items g, g + G, ...).
// CTA 0 runs the OCP from its global workspace slot; all CTAs run its PCG solves from their
// shared memory.  Launched with a cluster dimension of 2..8 CTAs of kClThreads threads.
template <class M>
__global__ void __launch_bounds__(kClThreads, 1) fused_cluster_kernel(const __grid_constant__ KParams P) {
  extern __shared__ __align__(16) float smem[];
  ClRun<M> r;
  r.init(smem, P.cl_kc);
  if (threadIdx.x == 0) {
    cl::bar_init(r.bar(CB_RED0), 1);   // one local arrival per phase; the data completes its bytes
    cl::bar_init(r.bar(CB_RED1), 1);
    cl::bar_init(r.bar(CB_CMD), 1);    // the leader's command
    cl::bar_init(r.bar(CB_REL), r.ncta);
    cl::fence_bar_init();
  }
  __syncthreads();
  cl::sync_all();
  const int cid = (int)cl::id(), ncl = (int)cl::nclusters();
  float* ws = P.gws + (size_t)cid * P.ws_floats;
  if (r.rank == 0) {
    for (int w = cid; w < P.n_work; w += ncl) run_one<M, kClThreads>(P, P.order[w], ws, threadIdx.x, 0, &r);
    if (!r.broken) cl_command<M>(r, CL_EXIT, 0, 0, 0, 0);
  } else {
    cl_follower<M>(r, P, ws);
  }
  __syncthreads();
  cl::sync_all();
}
#endif

}  // namespace dmpc
