// Dynamics models f_t(x_{t+1}, x_t, u_t) = x_{t+1} - Phi_t(x_t, u_t; theta) of the OCP
// (paper Sec. 3, OCP statement).  Each model gives continuous dynamics templated on the
// scalar type (float, double, Dual<N>, HDual<P>) and an integrator; Phi_t is one
// integrator step, so A_t^+ = I, A_t = -dPhi/dx, B_t = -dPhi/du in Eq. 4.  Trap<Model>
// integrates the same continuous model by the implicit trapezoidal rule,
// f_t = x_{t+1} - x_t - dt/2 (F(x_t, u_t) + F(x_{t+1}, u_t)), whose A_t^+ = I - dt/2 dF/dx(x_{t+1})
// is a general matrix (Eq. 4 and 10 with A^+ != I).
// The LQ model (affine x_{t+1} = Abar_t x_t + Bbar_t u_t + c_t, App. B.1) carries per-knot
// parameters and is handled in closed form by the solver.
#pragma once
#include "device_util.cuh"

namespace dmpc {

enum ModelId : int {
  M_LQ = 0, M_PENDULUM = 1, M_CARTPOLE = 2, M_KIN_BICYCLE = 3,
  M_SINGLE_TRACK = 4, M_RIGID_BODY12 = 5, M_ATTITUDE = 6,
  M_SINGLE_TRACK_RATE = 7,
  // internal ids of the trapezoidal (implicit) variants: model id + kTrapIdOffset
  M_PENDULUM_TRAP = 17, M_CARTPOLE_TRAP = 18
};
constexpr int kTrapIdOffset = 16;
enum Integrator : int { I_RK4 = 0, I_EULER = 1, I_AFFINE = 2, I_TRAP = 3, I_RATE = 4 };

constexpr float kGravity = 9.81f;

// Pendulum, angle from upright: m L^2 phi'' = m g L sin(phi) + u.  params (m, L).
struct Pendulum {
  static constexpr int ID = M_PENDULUM, NX = 2, NU = 1, NP = 2, INTEG = I_RK4;
  template <class S>
  __device__ static void f(const S* x, const S* u, const S* p, S* xd) {
    xd[0] = x[1];
    xd[1] = (kGravity * m_sin(x[0])) / p[1] + u[0] / (p[0] * p[1] * p[1]);
  }
};

// Cart-pole, phi = 0 upright, tip at (p + L sin phi, L cos phi), frictionless, m_c = 1.
//   p''   = (u + m_p sin(phi) (L phi'^2 - g cos(phi))) / (m_c + m_p sin^2 phi)
//   phi'' = ((m_c + m_p) g sin(phi) - u cos(phi) - m_p L phi'^2 sin(phi) cos(phi))
//           / (L (m_c + m_p sin^2 phi))
// params (m_p, L).
struct CartPole {
  static constexpr int ID = M_CARTPOLE, NX = 4, NU = 1, NP = 2, INTEG = I_RK4;
  template <class S>
  __device__ static void f(const S* x, const S* u, const S* p, S* xd) {
    const float mc = 1.0f;
    S s = m_sin(x[2]), c = m_cos(x[2]);
    S w2 = x[3] * x[3];
    S den = mc + p[0] * s * s;
    S num_p = u[0] + p[0] * s * (p[1] * w2 - kGravity * c);
    S num_w = (mc + p[0]) * kGravity * s - u[0] * c - p[0] * p[1] * w2 * s * c;
    xd[0] = x[1];
    xd[1] = num_p / den;
    xd[2] = x[3];
    xd[3] = num_w / (p[1] * den);
  }
};

// Kinematic bicycle: state (px, py, psi, v), input (delta, a); param wheelbase.
struct KinBicycle {
  static constexpr int ID = M_KIN_BICYCLE, NX = 4, NU = 2, NP = 1, INTEG = I_RK4;
  template <class S>
  __device__ static void f(const S* x, const S* u, const S* p, S* xd) {
    xd[0] = x[3] * m_cos(x[2]);
    xd[1] = x[3] * m_sin(x[2]);
    xd[2] = x[3] * m_tan(u[0]) / p[0];
    xd[3] = u[1];
  }
};

// Uncoupled Fiala brush lateral force: below alpha_sl = atan(3 mu Fz / C),
// F = -C t + C^2/(3 mu Fz)|t| t - C^3/(27 mu^2 Fz^2) t^3 (t = tan alpha); beyond, -mu Fz sign.
template <class S>
__device__ __forceinline__ S fiala(const S& alpha, const S& mu, const S& ca, float fz) {
  S t = m_tan(alpha);
  S tsat = 3.0f * fz * mu / ca;
  if (fabsf(m_val(t)) < fabsf(m_val(tsat))) {
    S k2 = ca * ca / (3.0f * fz * mu);
    S k3 = ca * ca * ca / (27.0f * fz * fz * mu * mu);
    return -1.0f * (ca * t) + k2 * m_abs(t) * t - k3 * t * t * t;
  }
  float sg = m_val(t) < 0.f ? -1.f : 1.f;
  return (-sg * fz) * mu;
}

// Dynamic single-track vehicle with Fiala tyres: state (px, py, psi, r, Vy, Vx),
// input (delta, rear drive force Fx); params (mu, C_alpha).  a, b, m from the paper's
// nominal vehicle table, Iz = m a b.
struct SingleTrack {
  static constexpr int ID = M_SINGLE_TRACK, NX = 6, NU = 2, NP = 2, INTEG = I_RK4;
  template <class S>
  __device__ static void f(const S* x, const S* u, const S* p, S* xd) {
    const float a = 1.239f, b = 1.209f, m = 1476.0f;
    const float iz = m * a * b;
    const float fzf = m * kGravity * b / (a + b);
    const float fzr = m * kGravity * a / (a + b);
    S af = m_atan((x[4] + a * x[3]) / x[5]) - u[0];
    S ar = m_atan((x[4] - b * x[3]) / x[5]);
    S fyf = fiala(af, p[0], p[1], fzf);
    S fyr = fiala(ar, p[0], p[1], fzr);
    S cd = m_cos(u[0]), sd = m_sin(u[0]);
    S cp = m_cos(x[2]), sp = m_sin(x[2]);
    xd[0] = x[5] * cp - x[4] * sp;
    xd[1] = x[5] * sp + x[4] * cp;
    xd[2] = x[3];
    xd[3] = (a * (fyf * cd) - b * fyr) / iz;
    xd[4] = (fyf * cd + fyr) / m - x[3] * x[5];
    xd[5] = (u[1] - fyf * sd) / m + x[3] * x[4];
  }
};

// Quadrotor-like rigid body: p, v (world), ZYX Euler angles (roll, pitch, yaw), body rates w;
// input (thrust deviation from hover, torques); params (m, Jx, Jy, Jz).
struct RigidBody12 {
  static constexpr int ID = M_RIGID_BODY12, NX = 12, NU = 4, NP = 4, INTEG = I_RK4;
  template <class S>
  __device__ static void f(const S* x, const S* u, const S* p, S* xd) {
    S sro = m_sin(x[6]), cro = m_cos(x[6]);
    S spi = m_sin(x[7]), cpi = m_cos(x[7]);
    S sya = m_sin(x[8]), cya = m_cos(x[8]);
    S acc = (kGravity * p[0] + u[0]) / p[0];
    S tpi = spi / cpi;
    xd[0] = x[3]; xd[1] = x[4]; xd[2] = x[5];
    xd[3] = acc * (cya * spi * cro + sya * sro);
    xd[4] = acc * (sya * spi * cro - cya * sro);
    xd[5] = acc * (cpi * cro) - kGravity;
    xd[6] = x[9] + sro * tpi * x[10] + cro * tpi * x[11];
    xd[7] = cro * x[10] - sro * x[11];
    xd[8] = (sro * x[10] + cro * x[11]) / cpi;
    S hx = p[1] * x[9], hy = p[2] * x[10], hz = p[3] * x[11];
    xd[9] = (u[1] - (x[10] * hz - x[11] * hy)) / p[1];
    xd[10] = (u[2] - (x[11] * hx - x[9] * hz)) / p[2];
    xd[11] = (u[3] - (x[9] * hy - x[10] * hx)) / p[3];
  }
};

// Attitude rates (App. B.1): J w' = (J w) x w + tau, forward Euler; params diag J.
struct Attitude {
  static constexpr int ID = M_ATTITUDE, NX = 3, NU = 3, NP = 3, INTEG = I_EULER;
  template <class S>
  __device__ static void f(const S* x, const S* u, const S* p, S* xd) {
    S h0 = p[0] * x[0], h1 = p[1] * x[1], h2 = p[2] * x[2];
    xd[0] = (h1 * x[2] - h2 * x[1] + u[0]) / p[0];
    xd[1] = (h2 * x[0] - h0 * x[2] + u[1]) / p[1];
    xd[2] = (h0 * x[1] - h1 * x[0] + u[2]) / p[2];
  }
};

// The increment Phi(x, u; p) - x of one integrator step of model M, formed without adding x
// (dt k1 for Euler, dt/6 (k1 + 2 k2 + 2 k3 + k4) for RK4): its value and derivatives are small
// next to x, so they keep their FP32 precision where Phi itself would round them away.
template <class M, class S>
__device__ __forceinline__ void model_increment(const S* x, const S* u, const S* p, float dt, S* dx) {
  if constexpr (M::INTEG == I_RATE) {
    // control-rate augmentation: the base model's increment with the input held in the state,
    // and dt times the rate for the input part
    using Bm = typename M::Base;
    model_increment<Bm>(x, x + Bm::NX, p, dt, dx);
#pragma unroll
    for (int i = 0; i < M::NU; ++i) dx[Bm::NX + i] = dt * u[i];
    return;
  } else if constexpr (M::INTEG == I_EULER) {
    S k1[M::NX];
    M::f(x, u, p, k1);
#pragma unroll
    for (int i = 0; i < M::NX; ++i) dx[i] = dt * k1[i];
    return;
  } else {
  S k[M::NX], acc[M::NX], xt[M::NX];
  M::f(x, u, p, k);
#pragma unroll
  for (int i = 0; i < M::NX; ++i) { acc[i] = k[i]; xt[i] = x[i] + (0.5f * dt) * k[i]; }
  M::f(xt, u, p, k);
#pragma unroll
  for (int i = 0; i < M::NX; ++i) { acc[i] = acc[i] + 2.0f * k[i]; xt[i] = x[i] + (0.5f * dt) * k[i]; }
  M::f(xt, u, p, k);
#pragma unroll
  for (int i = 0; i < M::NX; ++i) { acc[i] = acc[i] + 2.0f * k[i]; xt[i] = x[i] + dt * k[i]; }
  M::f(xt, u, p, k);
#pragma unroll
  for (int i = 0; i < M::NX; ++i) dx[i] = (dt / 6.0f) * (acc[i] + k[i]);
  }
}

// One integrator step Phi(x, u; p) of model M.
template <class M, class S>
__device__ __forceinline__ void model_step(const S* x, const S* u, const S* p, float dt, S* xn) {
  if constexpr (M::INTEG == I_RATE) {
    S dx[M::NX];
    model_increment<M>(x, u, p, dt, dx);
#pragma unroll
    for (int i = 0; i < M::NX; ++i) xn[i] = x[i] + dx[i];
    return;
  } else {
  if (M::INTEG == I_EULER) {
    S k1[M::NX];
    M::f(x, u, p, k1);
#pragma unroll
    for (int i = 0; i < M::NX; ++i) xn[i] = x[i] + dt * k1[i];
    return;
  }
  S k[M::NX], acc[M::NX], xt[M::NX];
  M::f(x, u, p, k);
#pragma unroll
  for (int i = 0; i < M::NX; ++i) { acc[i] = k[i]; xt[i] = x[i] + (0.5f * dt) * k[i]; }
  M::f(xt, u, p, k);
#pragma unroll
  for (int i = 0; i < M::NX; ++i) { acc[i] = acc[i] + 2.0f * k[i]; xt[i] = x[i] + (0.5f * dt) * k[i]; }
  M::f(xt, u, p, k);
#pragma unroll
  for (int i = 0; i < M::NX; ++i) { acc[i] = acc[i] + 2.0f * k[i]; xt[i] = x[i] + dt * k[i]; }
  M::f(xt, u, p, k);
#pragma unroll
  for (int i = 0; i < M::NX; ++i) xn[i] = x[i] + (dt / 6.0f) * (acc[i] + k[i]);
  }
}

// Control-rate augmentation of a base model (App. B.3): state (x, u), input u_dot, with
// x_{t+1} = Phi_t(x_t, u_t) of the base model and u_{t+1} = u_t + dt u_dot_t, so the input cost
// penalises the rate of the base model's input.  Same parameters as the base model.
template <class B_, int ID_>
struct Rate {
  using Base = B_;
  static constexpr int ID = ID_, NX = B_::NX + B_::NU, NU = B_::NU, NP = B_::NP, INTEG = I_RATE;
};

// A continuous model integrated by the implicit trapezoidal rule.
template <class Base>
struct Trap : Base {
  static constexpr int ID = Base::ID + kTrapIdOffset, INTEG = I_TRAP;
};

template <class M> struct is_implicit { static constexpr bool value = M::INTEG == I_TRAP; };

// f_t(x_t, u_t, x_{t+1}) of the trapezoidal rule.
template <class M, class S>
__device__ __forceinline__ void trap_residual(const S* x, const S* u, const S* xn, const S* p, float dt, S* r) {
  S fa[M::NX], fb[M::NX];
  M::f(x, u, p, fa);
  M::f(xn, u, p, fb);
#pragma unroll
  for (int i = 0; i < M::NX; ++i) r[i] = (xn[i] - x[i]) - (0.5f * dt) * (fa[i] + fb[i]);
}

// The LQ model: per-knot Abar (nx*nx, row-major), Bbar (nx*nu), c (nx).  NX/NU are
// template parameters of the solver instance.
template <int NX_, int NU_>
struct LQ {
  static constexpr int ID = M_LQ, NX = NX_, NU = NU_, NP = 0, INTEG = I_AFFINE;
  static constexpr int PK = NX_ * NX_ + NX_ * NU_ + NX_;
};

template <class M> struct is_lq { static constexpr bool value = false; };
template <int A, int B> struct is_lq<LQ<A, B>> { static constexpr bool value = true; };

}  // namespace dmpc
