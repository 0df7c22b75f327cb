"""Dynamics models f_t^theta of the OCP (Sec. 3, OCP statement) for the FP64 oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

By default a model is explicit: the constraint is f_t(x_{t+1}, x_t, u_t) = x_{t+1} - Phi_t(x_t, u_t)
with Phi_t a one-step integrator of continuous dynamics (RK4 or forward Euler), or the
affine map of the LQ benchmark (App. B.1, "QP problems").  Hence A_t^+ = I,
A_t = -dPhi/dx, B_t = -dPhi/du in Eq. 4.  A continuous model can instead use the implicit
trapezoidal rule (integrator "trapezoid"): f_t = x_{t+1} - x_t - dt/2 (F(x_t, u_t) + F(x_{t+1}, u_t)),
which makes A_t^+ = I - dt/2 dF/dx(x_{t+1}, u_t) a general matrix (the A^+ of Eq. 4 and 10).

Parameters theta of a model are split into `p_shared` entries common to all knots and
`p_knot` entries that belong to one knot t (only the LQ model has those: its A_t, B_t, c_t).

All functions take lists of components (Jets or numpy arrays of equal shape), so the
same code gives plain values and derivatives.  The equations are written out in the
project design notes; this file is an independent transcription of them.
"""
import numpy as np

from .jet import sin, cos, tan, atan, absval, where, value

GRAVITY = 9.81


def rk4(fc, x, u, ths, dt):
    """Classical 4-stage Runge-Kutta step of x' = fc(x, u, ths) with zero-order-hold u."""
    k1 = fc(x, u, ths)
    k2 = fc([xi + 0.5 * dt * ki for xi, ki in zip(x, k1)], u, ths)
    k3 = fc([xi + 0.5 * dt * ki for xi, ki in zip(x, k2)], u, ths)
    k4 = fc([xi + dt * ki for xi, ki in zip(x, k3)], u, ths)
    return [xi + (dt / 6.0) * (a + 2.0 * b + 2.0 * c + d)
            for xi, a, b, c, d in zip(x, k1, k2, k3, k4)]


def euler(fc, x, u, ths, dt):
    k1 = fc(x, u, ths)
    return [xi + dt * ki for xi, ki in zip(x, k1)]


class Model:
    name = "base"
    nx = nu = 0
    p_shared = 0
    p_knot = 0
    integrator = "rk4"

    def __init__(self, dt):
        self.dt = float(dt)

    def fc(self, x, u, ths):  # continuous-time dynamics
        raise NotImplementedError

    def step(self, x, u, ths, thk):
        """Phi_t(x_t, u_t; theta): the discrete one-step map (explicit integrators)."""
        integ = rk4 if self.integrator == "rk4" else euler
        return integ(self.fc, x, u, ths, self.dt)

    @property
    def implicit(self):
        return self.integrator == "trapezoid"

    def residual(self, x, u, xn, ths, thk):
        """f_t(x_t, u_t, x_{t+1}; theta), the dynamics constraint written implicitly."""
        if self.implicit:
            fa = self.fc(x, u, ths)
            fb = self.fc(xn, u, ths)
            return [xn[i] - x[i] - (0.5 * self.dt) * (fa[i] + fb[i]) for i in range(self.nx)]
        phi = self.step(x, u, ths, thk)
        return [xn[i] - phi[i] for i in range(self.nx)]


class LQ(Model):
    """Affine dynamics x_{t+1} = Abar_t x_t + Bbar_t u_t + c_t (App. B.1).

    Per-knot parameters, row-major: Abar_t (nx*nx), Bbar_t (nx*nu), c_t (nx)."""
    name = "lq"
    integrator = "affine"

    def __init__(self, nx, nu, dt=1.0):
        super().__init__(dt)
        self.nx, self.nu = nx, nu
        self.p_knot = nx * nx + nx * nu + nx

    def step(self, x, u, ths, thk):
        nx, nu = self.nx, self.nu
        out = []
        for i in range(nx):
            acc = thk[nx * nx + nx * nu + i]
            for j in range(nx):
                acc = acc + thk[i * nx + j] * x[j]
            for j in range(nu):
                acc = acc + thk[nx * nx + i * nu + j] * u[j]
            out.append(acc)
        return out


class Pendulum(Model):
    """Point-mass pendulum, angle phi measured from upright, torque input.

    m L^2 phi'' = m g L sin(phi) + u.   theta_shared = (m, L)."""
    name = "pendulum"
    nx, nu, p_shared = 2, 1, 2

    def fc(self, x, u, ths):
        phi, w = x
        m, L = ths
        return [w, (GRAVITY / L) * sin(phi) + u[0] / (m * L * L)]


class CartPole(Model):
    """Cart-pole, frictionless, point-mass pole of length L on a massless rod.

    State (p, p', phi, phi'), phi = 0 upright, pole tip at (p + L sin phi, L cos phi);
    input: horizontal force on the cart.  Lagrangian equations of motion:
      p''   = (u + m_p sin(phi) (L phi'^2 - g cos(phi))) / (m_c + m_p sin^2 phi)
      phi'' = ((m_c + m_p) g sin(phi) - u cos(phi) - m_p L phi'^2 sin(phi) cos(phi))
              / (L (m_c + m_p sin^2 phi))
    m_c = 1, g = 9.81 (App. B.2); theta_shared = (m_p, L)."""
    name = "cartpole"
    nx, nu, p_shared = 4, 1, 2
    m_c = 1.0

    def fc(self, x, u, ths):
        p, v, phi, w = x
        m_p, L = ths
        s, c = sin(phi), cos(phi)
        den = self.m_c + m_p * s * s
        pdd = (u[0] + m_p * s * (L * w * w - GRAVITY * c)) / den
        wdd = ((self.m_c + m_p) * GRAVITY * s - u[0] * c - m_p * L * w * w * s * c) / (L * den)
        return [v, pdd, w, wdd]


class KinematicBicycle(Model):
    """Kinematic bicycle: state (px, py, psi, v), input (steer delta, acceleration a).

    px' = v cos psi, py' = v sin psi, psi' = v tan(delta) / l_wb, v' = a.
    theta_shared = (l_wb,)."""
    name = "kin_bicycle"
    nx, nu, p_shared = 4, 2, 1

    def fc(self, x, u, ths):
        px, py, psi, v = x
        delta, a = u
        (lwb,) = ths
        return [v * cos(psi), v * sin(psi), v * tan(delta) / lwb, a]


def fiala_lateral_force(alpha, mu, c_alpha, fz):
    """Uncoupled Fiala brush lateral force F_y(alpha) (Svendenius 2007).

    Below the full-slide angle alpha_sl = atan(3 mu Fz / C):
      F = -C t + C^2/(3 mu Fz) |t| t - C^3/(27 mu^2 Fz^2) t^3,  t = tan(alpha);
    beyond it the force saturates at -mu Fz sign(alpha)."""
    t = tan(alpha)
    sat = 3.0 * mu * fz / c_alpha  # tan(alpha_sl)
    lin = (-1.0 * c_alpha * t + (c_alpha * c_alpha / (3.0 * mu * fz)) * absval(t) * t
           - (c_alpha * c_alpha * c_alpha / (27.0 * mu * mu * fz * fz)) * t * t * t)
    slide = -1.0 * mu * fz * np.sign(value(t))
    return where(np.abs(value(t)) < np.abs(value(sat)), lin, slide)


class SingleTrackFiala(Model):
    """Dynamic single-track vehicle with Fiala tyres.

    State (px, py, psi, r, Vy, Vx) (body-frame velocities), input (steer delta, rear drive force Fx).
      px' = Vx cos psi - Vy sin psi,  py' = Vx sin psi + Vy cos psi,  psi' = r
      r'  = (a Fyf cos delta - b Fyr) / Iz
      Vy' = (Fyf cos delta + Fyr) / m - r Vx
      Vx' = (Fx - Fyf sin delta) / m + r Vy
      slip: alpha_f = atan((Vy + a r)/Vx) - delta,  alpha_r = atan((Vy - b r)/Vx)
      static loads Fzf = m g b/(a+b), Fzr = m g a/(a+b).
    a, b, m from the paper's nominal vehicle table; Iz = m a b (synthetic constant).
    theta_shared = (mu, C_alpha), one friction and one cornering stiffness for both axles."""
    name = "single_track"
    nx, nu, p_shared = 6, 2, 2
    a, b, m = 1.239, 1.209, 1476.0

    @property
    def Iz(self):
        return self.m * self.a * self.b

    def fc(self, x, u, ths):
        px, py, psi, r, vy, vx = x
        delta, fx = u
        mu, ca = ths
        a, b, m = self.a, self.b, self.m
        fzf = m * GRAVITY * b / (a + b)
        fzr = m * GRAVITY * a / (a + b)
        alpha_f = atan((vy + a * r) / vx) - delta
        alpha_r = atan((vy - b * r) / vx)
        fyf = fiala_lateral_force(alpha_f, mu, ca, fzf)
        fyr = fiala_lateral_force(alpha_r, mu, ca, fzr)
        cd, sd = cos(delta), sin(delta)
        return [vx * cos(psi) - vy * sin(psi),
                vx * sin(psi) + vy * cos(psi),
                r,
                (a * fyf * cd - b * fyr) / self.Iz,
                (fyf * cd + fyr) / m - r * vx,
                (fx - fyf * sd) / m + r * vy]


class RigidBody12(Model):
    """Quadrotor-like rigid body, 12 states, 4 inputs.

    State (p[3], v[3] world frame, Euler angles (roll, pitch, yaw) ZYX, body rates w[3]);
    input (thrust deviation from hover dT, body torques tau[3]).
      p' = v,  v' = (m g + dT)/m * R(eta) e3 - g e3,
      roll'  = wx + sin(roll) tan(pitch) wy + cos(roll) tan(pitch) wz
      pitch' = cos(roll) wy - sin(roll) wz
      yaw'   = (sin(roll) wy + cos(roll) wz) / cos(pitch)
      J w' = tau - w x (J w),  J = diag(Jx, Jy, Jz).
    R(eta) e3 = (cos yaw sin pitch cos roll + sin yaw sin roll,
                 sin yaw sin pitch cos roll - cos yaw sin roll, cos pitch cos roll).
    theta_shared = (m, Jx, Jy, Jz)."""
    name = "rigid_body12"
    nx, nu, p_shared = 12, 4, 4

    def fc(self, x, u, ths):
        vx, vy, vz = x[3:6]
        ro, pi, ya = x[6:9]
        wx, wy, wz = x[9:12]
        dT, tx, ty, tz = u
        m, jx, jy, jz = ths
        acc = (m * GRAVITY + dT) / m
        sro, cro, spi, cpi, sya, cya = sin(ro), cos(ro), sin(pi), cos(pi), sin(ya), cos(ya)
        tpi = spi / cpi
        ax = acc * (cya * spi * cro + sya * sro)
        ay = acc * (sya * spi * cro - cya * sro)
        az = acc * (cpi * cro) - GRAVITY
        dro = wx + sro * tpi * wy + cro * tpi * wz
        dpi = cro * wy - sro * wz
        dya = (sro * wy + cro * wz) / cpi
        dwx = (tx - (wy * (jz * wz) - wz * (jy * wy))) / jx
        dwy = (ty - (wz * (jx * wx) - wx * (jz * wz))) / jy
        dwz = (tz - (wx * (jy * wy) - wy * (jx * wx))) / jz
        return [vx, vy, vz, ax, ay, az, dro, dpi, dya, dwx, dwy, dwz]


class Attitude(Model):
    """Rigid-body attitude rates (App. B.1, nonlinear attitude stabilisation):
    J w' = (J w) x w + tau, J = diag(J1, J2, J3), forward Euler.  theta_shared = (J1, J2, J3)."""
    name = "attitude"
    nx, nu, p_shared = 3, 3, 3
    integrator = "euler"

    def fc(self, x, u, ths):
        w1, w2, w3 = x
        j1, j2, j3 = ths
        h1, h2, h3 = j1 * w1, j2 * w2, j3 * w3
        c1 = h2 * w3 - h3 * w2
        c2 = h3 * w1 - h1 * w3
        c3 = h1 * w2 - h2 * w1
        return [(c1 + u[0]) / j1, (c2 + u[1]) / j2, (c3 + u[2]) / j3]


class ControlRate(Model):
    """Control-rate augmentation of a base model (App. B.3: the vehicle's cost on control rates
    is implemented by augmenting the state with the input, x <- (x, u), and taking the rate of the
    input as the new input, u <- u_dot).  State (x, u) of size nx_b + nu_b, input v (nu_b):
      x_{t+1} = Phi_t(x_t, u_t)   (the base model's step, with the input held in the state),
      u_{t+1} = u_t + dt v_t,
    so v_t = (u_{t+1} - u_t) / dt, and the input cost 1/2 v^T diag(R) v penalises the rate while
    diag(Q) over (x, u) weighs the state and the input itself.  Same parameters as the base."""
    integrator = "rate"

    def __init__(self, base):
        super().__init__(base.dt)
        self.base = base
        self.name = base.name + "_rate"
        self.nx = base.nx + base.nu
        self.nu = base.nu
        self.p_shared = base.p_shared
        self.p_knot = base.p_knot

    def step(self, x, u, ths, thk):
        nb = self.base.nx
        xb, ub = list(x[:nb]), list(x[nb:])
        return list(self.base.step(xb, ub, ths, thk)) + [ub[i] + self.dt * u[i] for i in range(self.nu)]


def make_model(name, nx=None, nu=None, dt=0.05, integrator=None):
    """integrator: None (the model's own) or "trapezoid" (implicit trapezoidal rule).  A name
    ending in "_rate" is the control-rate augmentation of the named model."""
    if name.endswith("_rate"):
        return ControlRate(make_model(name[:-len("_rate")], dt=dt, integrator=integrator))
    if name == "lq":
        return LQ(nx, nu)
    table = {"pendulum": Pendulum, "cartpole": CartPole, "kin_bicycle": KinematicBicycle,
             "single_track": SingleTrackFiala, "rigid_body12": RigidBody12, "attitude": Attitude}
    m = table[name](dt)
    if integrator is not None:
        m.integrator = integrator
    return m
