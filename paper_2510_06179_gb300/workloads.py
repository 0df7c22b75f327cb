"""Seeded synthetic workloads (inputs only).

This module draws problem instances; it contains none of the solver's arithmetic and is
shared by the tests, the benchmark and the CUDA path's callers.  Every array it returns
is float32 (the solver's input precision); FP64 checks upcast these same values.

Distributions follow the paper's synthetic problems (random LQ problems of App. B.1,
cart-pole of App. B.2, attitude problem of App. B.1, vehicle of App. B.3) as restated
for the workloads below; a draw N(m, v) takes v as the variance.
"""
from dataclasses import dataclass, field

import numpy as np

# model registry: id, nx, nu, shared params, per-knot params (LQ: nx*nx + nx*nu + nx)
MODELS = {
    "lq":           dict(id=0, nx=None, nu=None, p_shared=0, integrator="affine"),
    "pendulum":     dict(id=1, nx=2, nu=1, p_shared=2, integrator="rk4"),
    "cartpole":     dict(id=2, nx=4, nu=1, p_shared=2, integrator="rk4"),
    "kin_bicycle":  dict(id=3, nx=4, nu=2, p_shared=1, integrator="rk4"),
    "single_track": dict(id=4, nx=6, nu=2, p_shared=2, integrator="rk4"),
    "rigid_body12": dict(id=5, nx=12, nu=4, p_shared=4, integrator="rk4"),
    "attitude":     dict(id=6, nx=3, nu=3, p_shared=3, integrator="euler"),
    "single_track_rate": dict(id=7, nx=8, nu=2, p_shared=2, integrator="rk4"),
}
MODEL_NAMES = {v["id"]: k for k, v in MODELS.items()}


def p_knot(model, nx, nu):
    return nx * nx + nx * nu + nx if model == "lq" else 0


def theta_layout(model, nx, nu, T):
    """[shared | T x per-knot | diag Q (nx) | diag R (nu) | diag Q_T (nx)] -> offsets dict."""
    ps = MODELS[model]["p_shared"]
    pk = p_knot(model, nx, nu)
    o_q = ps + T * pk
    return dict(shared=0, knot=ps, q=o_q, r=o_q + nx, qt=o_q + nx + nu, size=o_q + 2 * nx + nu,
                p_shared=ps, p_knot=pk)


@dataclass
class Workload:
    """A batch of OCPs of one model and horizon, plus solver settings and a loss target."""
    name: str
    model: str
    nx: int
    nu: int
    T: int
    dt: float
    x_s: np.ndarray          # (B, nx) float32
    theta: np.ndarray        # (B, p) float32
    x_ref: np.ndarray        # (B, T+1, nx) float32
    sqp_iters: int = 1
    line_search: bool = False
    pcg_tol: float = 1e-8
    u_target: np.ndarray = None   # (B, nu) float32: loss l = ||u_0 - u_target||^2
    extra: dict = field(default_factory=dict)
    integrator: str = None        # None: the model's own; "trapezoid": implicit trapezoidal rule

    @property
    def B(self):
        return self.x_s.shape[0]

    @property
    def K(self):
        return self.T + 1

    @property
    def n(self):
        return self.K * self.nx + self.T * self.nu

    @property
    def m(self):
        return self.K * self.nx

    @property
    def p(self):
        return self.theta.shape[1]

    def subset(self, idx):
        idx = np.asarray(idx)
        w = Workload(**{**self.__dict__})
        w.x_s, w.theta, w.x_ref = self.x_s[idx], self.theta[idx], self.x_ref[idx]
        if self.u_target is not None:
            w.u_target = self.u_target[idx]
        return w

    def dl_dz(self, z):
        """Gradient of l = sum_b ||u_0 - u_target||^2 with respect to z (float64 numpy)."""
        g = np.zeros_like(np.asarray(z, dtype=np.float64))
        g[:, self.nx:self.nx + self.nu] = 2.0 * (np.asarray(z, np.float64)[:, self.nx:self.nx + self.nu]
                                                  - self.u_target)
        return g


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _cost_weights(rng, B, nx, nu, q_lo=0.1, q_hi=10.0, r_lo=0.01, r_hi=1.0, terminal=10.0):
    q = rng.uniform(q_lo, q_hi, size=(B, nx))
    r = rng.uniform(r_lo, r_hi, size=(B, nu))
    return q, r, terminal * q


def lq_dynamics(rng, B, T, nx, nu, a_scale=0.05, b_var=0.1, rho_max=0.99, c_var=0.0):
    """A_t = I + a_scale M (M ~ N(0,1)), rescaled to spectral radius <= rho_max; B_t ~ N(0, b_var);
    c_t ~ N(0, c_var).  Drawn independently per OCP and knot."""
    M = rng.standard_normal((B, T, nx, nx))
    A = np.eye(nx) + a_scale * M
    rho = np.abs(np.linalg.eigvals(A)).max(axis=-1)
    scale = np.where(rho > rho_max, rho_max / rho, 1.0)
    A = A * scale[..., None, None]
    Bm = np.sqrt(b_var) * rng.standard_normal((B, T, nx, nu))
    c = np.sqrt(c_var) * rng.standard_normal((B, T, nx)) if c_var > 0 else np.zeros((B, T, nx))
    return A, Bm, c


def _pack_theta(model, nx, nu, T, shared, knot, q, r, qt):
    lay = theta_layout(model, nx, nu, T)
    B = q.shape[0]
    th = np.zeros((B, lay["size"]))
    if lay["p_shared"]:
        th[:, :lay["p_shared"]] = shared
    if lay["p_knot"]:
        th[:, lay["knot"]:lay["q"]] = knot.reshape(B, -1)
    th[:, lay["q"]:lay["r"]] = q
    th[:, lay["r"]:lay["qt"]] = r
    th[:, lay["qt"]:lay["size"]] = qt
    return th


def lq_config(B=16, T=20, nx=4, nu=1, seed=0, c_var=0.0):
    """Random LQ OCPs (App. B.1 restated): A_t = I + 0.05 M rescaled to rho <= 0.99, B_t ~ N(0, 0.1),
    diag Q ~ U[0.1, 10], diag R ~ U[0.01, 1], Q_T = 10 Q, x_0 ~ N(0, 1); one SQP step, alpha = 1."""
    rng = np.random.default_rng(seed)
    A, Bm, c = lq_dynamics(rng, B, T, nx, nu, c_var=c_var)
    q, r, qt = _cost_weights(rng, B, nx, nu)
    x_s = rng.standard_normal((B, nx))
    knot = np.concatenate([A.reshape(B, T, -1), Bm.reshape(B, T, -1), c], axis=2)
    th = _pack_theta("lq", nx, nu, T, None, knot, q, r, qt)
    u_t = rng.standard_normal((B, nu))
    return Workload("lq", "lq", nx, nu, T, 1.0, _f32(x_s), _f32(th), _f32(np.zeros((B, T + 1, nx))),
                    sqp_iters=1, line_search=False, pcg_tol=1e-8, u_target=_f32(u_t))


# Closed-loop RL benchmark problems (App. B.1, RL timing table): (nx, nu, MPC horizon T,
# episode length H, batch B).
RL_PROBLEMS = {1: (8, 4, 40, 50, 64), 2: (8, 4, 30, 50, 16), 3: (8, 4, 30, 50, 64), 4: (8, 4, 30, 50, 256),
               5: (16, 8, 30, 50, 16), 6: (16, 8, 30, 50, 64)}


@dataclass
class RLProblem:
    """A batch of random LQ environments x_{h+1} = A x_h + B u_h + b with an MPC policy whose
    cost is x^T diag(q) x + ||u||^2 over horizon T (the learned parameters are q)."""
    nx: int
    nu: int
    T: int
    H: int
    A: np.ndarray       # (B, nx, nx) float32
    Bm: np.ndarray      # (B, nx, nu) float32
    b: np.ndarray       # (B, nx) float32
    x0: np.ndarray      # (B, nx) float32
    q0: np.ndarray      # (B, nx) float32 initial diag(Q)

    @property
    def B(self):
        return self.x0.shape[0]

    def knot_theta(self):
        """Per-knot LQ parameters (A, B, b) of the MPC model, repeated over the horizon."""
        k = np.concatenate([self.A.reshape(self.B, -1), self.Bm.reshape(self.B, -1), self.b], axis=1)
        return _f32(np.repeat(k[:, None, :], self.T, axis=1).reshape(self.B, -1))


def rl_lq_problem(problem=1, seed=0, B=None, H=None, T=None):
    """Random LQ problem of the RL benchmark: A = I + 0.1 dA, vec(dA) ~ N(0, I), eigenvalues
    clipped to modulus <= 0.99 (phases kept); vec(B) ~ N(0, I); b ~ N(0, 1e-4 I); x_0 ~ N(0, 25 I).
    Initial cost weights diag(Q) ~ U[0.5, 2] (the paper does not state them).  B, H, T override
    the table's sizes."""
    nx, nu, T0, H0, B0 = RL_PROBLEMS[problem]
    B, H, T = B or B0, H or H0, T or T0
    rng = np.random.default_rng(seed)
    A = np.eye(nx) + 0.1 * rng.standard_normal((B, nx, nx))
    lam, V = np.linalg.eig(A)
    lam = lam * np.minimum(1.0, 0.99 / np.maximum(np.abs(lam), 1e-300))
    A = np.real(V @ (lam[..., None] * np.linalg.inv(V)))
    Bm = rng.standard_normal((B, nx, nu))
    b = 1e-2 * rng.standard_normal((B, nx))
    x0 = 5.0 * rng.standard_normal((B, nx))
    q0 = rng.uniform(0.5, 2.0, size=(B, nx))
    return RLProblem(nx, nu, T, H, _f32(A), _f32(Bm), _f32(b), _f32(x0), _f32(q0))


def cartpole_config(B=256, T=50, seed=0, sqp_iters=10, pcg_tol=1e-6, dt=0.05, integrator=None):
    """Cart-pole swing-up/balance: m_p ~ U[0.05, 0.2], L ~ U[0.3, 0.7], diag Q ~ U[0.1, 10],
    diag R ~ U[0.01, 1], Q_T = 10 Q; x_0: angle ~ U[-pi, pi], other states ~ N(0, 0.5);
    reference = upright at rest; loss target u_target ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    mp = rng.uniform(0.05, 0.2, size=B)
    L = rng.uniform(0.3, 0.7, size=B)
    q, r, qt = _cost_weights(rng, B, 4, 1)
    x_s = np.sqrt(0.5) * rng.standard_normal((B, 4))
    x_s[:, 2] = rng.uniform(-np.pi, np.pi, size=B)
    th = _pack_theta("cartpole", 4, 1, T, np.stack([mp, L], 1), None, q, r, qt)
    u_t = rng.standard_normal((B, 1))
    return Workload("cartpole" if integrator is None else f"cartpole_{integrator}", "cartpole", 4, 1, T, dt,
                    _f32(x_s), _f32(th), _f32(np.zeros((B, T + 1, 4))), sqp_iters=sqp_iters, line_search=True,
                    pcg_tol=pcg_tol, u_target=_f32(u_t), integrator=integrator)


def pendulum_config(B=64, T=40, seed=0, sqp_iters=10, pcg_tol=1e-6, dt=0.05, integrator=None):
    """Pendulum swing-up/balance: m ~ U[0.5, 2], L ~ U[0.5, 1.5]; angle ~ U[-pi, pi], rate ~ N(0, 0.5)."""
    rng = np.random.default_rng(seed)
    m = rng.uniform(0.5, 2.0, size=B)
    L = rng.uniform(0.5, 1.5, size=B)
    q, r, qt = _cost_weights(rng, B, 2, 1)
    x_s = np.stack([rng.uniform(-np.pi, np.pi, size=B), np.sqrt(0.5) * rng.standard_normal(B)], 1)
    th = _pack_theta("pendulum", 2, 1, T, np.stack([m, L], 1), None, q, r, qt)
    return Workload("pendulum" if integrator is None else f"pendulum_{integrator}", "pendulum", 2, 1, T, dt,
                    _f32(x_s), _f32(th), _f32(np.zeros((B, T + 1, 2))), sqp_iters=sqp_iters, line_search=True,
                    pcg_tol=pcg_tol, u_target=_f32(rng.standard_normal((B, 1))), integrator=integrator)


def bicycle_config(B=64, T=40, seed=0, sqp_iters=10, pcg_tol=1e-6, dt=0.05):
    """Kinematic bicycle keeping a straight lane at speed: wheelbase ~ U[2.5, 3.0]; reference
    x_ref,t = (v_ref t dt, 0, 0, v_ref), v_ref ~ U[3, 8] m/s; x_0: lateral offset ~ U[-1, 1] m,
    heading ~ U[-0.2, 0.2] rad, speed v_ref U[0.8, 1.2]; diag Q ~ U[0.1, 10], Q_T = 10 Q;
    steering weight ~ U[0.5, 5], acceleration weight ~ U[0.01, 1].  (Cheap steering lets the first
    QP step from the cold start command angles past +-pi/2, where tan(delta) has poles.)"""
    rng = np.random.default_rng(seed)
    lwb = rng.uniform(2.5, 3.0, size=B)
    q, r, qt = _cost_weights(rng, B, 4, 2)
    r[:, 0] = rng.uniform(0.5, 5.0, size=B)
    vref = rng.uniform(3.0, 8.0, size=B)
    x_s = np.stack([np.zeros(B), rng.uniform(-1, 1, B), rng.uniform(-0.2, 0.2, B),
                    vref * rng.uniform(0.8, 1.2, B)], 1)
    tt = np.arange(T + 1) * dt
    x_ref = np.zeros((B, T + 1, 4))
    x_ref[:, :, 0] = vref[:, None] * tt[None, :]
    x_ref[:, :, 3] = vref[:, None]
    th = _pack_theta("kin_bicycle", 4, 2, T, lwb[:, None], None, q, r, qt)
    return Workload("kin_bicycle", "kin_bicycle", 4, 2, T, dt, _f32(x_s), _f32(th), _f32(x_ref),
                    sqp_iters=sqp_iters, line_search=True, pcg_tol=pcg_tol,
                    u_target=_f32(rng.standard_normal((B, 2))))


def sinusoid_reference(rng, B, T, dt, speed):
    """Reference states along a path of sinusoidal curvature kappa(s) = k0 sin(2 pi s / wl + ph),
    driven at constant speed: (px, py, psi, r = V kappa, Vy = 0, Vx = V).  Euler-integrated
    with 10 sub-steps per knot."""
    k0 = rng.uniform(0.01, 0.05, size=B)
    wl = rng.uniform(20.0, 60.0, size=B)
    ph = rng.uniform(0, 2 * np.pi, size=B)
    ref = np.zeros((B, T + 1, 6))
    px = np.zeros(B); py = np.zeros(B); psi = np.zeros(B); s = np.zeros(B)
    sub = 10
    h = dt / sub
    for t in range(T + 1):
        kap = k0 * np.sin(2 * np.pi * s / wl + ph)
        ref[:, t] = np.stack([px, py, psi, speed * kap, np.zeros(B), speed], 1)
        for _ in range(sub):
            kap = k0 * np.sin(2 * np.pi * s / wl + ph)
            px = px + h * speed * np.cos(psi)
            py = py + h * speed * np.sin(psi)
            psi = psi + h * speed * kap
            s = s + h * speed
    return ref


def vehicle_config(B=1024, T=100, seed=0, sqp_iters=10, pcg_tol=1e-6, dt=0.02, weights=None):
    """Dynamic single-track vehicle with Fiala tyres tracking a sinusoidal-curvature path:
    mu ~ U[0.3, 1.1], C_alpha ~ U[5e4, 1.5e5] N/rad; speed ~ U[8, 15] m/s; x_0 = reference
    start perturbed (lateral N(0, 0.25), heading N(0, 0.01), yaw rate N(0, 0.01), Vy N(0, 0.01)).
    Cost weights: `weights` = (q (B,6), r (B,2)) from a learned map, else drawn log-uniformly
    around a nominal tracking tune.  Features: 16-dim N(0, 1) per OCP (extra['features'])."""
    rng = np.random.default_rng(seed)
    mu = rng.uniform(0.3, 1.1, size=B)
    ca = rng.uniform(5e4, 1.5e5, size=B)
    speed = rng.uniform(8.0, 15.0, size=B)
    ref = sinusoid_reference(rng, B, T, dt, speed)
    x_s = ref[:, 0].copy()
    x_s[:, 1] += np.sqrt(0.25) * rng.standard_normal(B)
    x_s[:, 2] += np.sqrt(0.01) * rng.standard_normal(B)
    x_s[:, 3] += np.sqrt(0.01) * rng.standard_normal(B)
    x_s[:, 4] += np.sqrt(0.01) * rng.standard_normal(B)
    feats = rng.standard_normal((B, 16))
    if weights is None:
        nominal_q = np.array([1.0, 1.0, 10.0, 1.0, 1.0, 1.0])
        nominal_r = np.array([10.0, 1e-6])
        q = nominal_q * np.exp(rng.uniform(-1, 1, size=(B, 6)))
        r = nominal_r * np.exp(rng.uniform(-1, 1, size=(B, 2)))
    else:
        q, r = weights
    th = _pack_theta("single_track", 6, 2, T, np.stack([mu, ca], 1), None, q, r, 10.0 * q)
    return Workload("vehicle", "single_track", 6, 2, T, dt, _f32(x_s), _f32(th), _f32(ref),
                    sqp_iters=sqp_iters, line_search=True, pcg_tol=pcg_tol,
                    u_target=_f32(np.zeros((B, 2))), extra=dict(features=_f32(feats)))


def vehicle_rate_config(B=64, T=50, seed=0, sqp_iters=10, pcg_tol=1e-6, dt=0.02):
    """The single-track vehicle with control-rate augmentation (App. B.3): state (px, py, psi, r,
    Vy, Vx, delta, Fx), input (delta rate, Fx rate).  Inputs as in vehicle_config; the initial
    steer and drive force are 0 and the reference holds them at 0.  Weights: state as the
    vehicle's tracking tune, the inputs themselves U-log around (1, 1e-6), their rates around
    (0.1, 1e-8) (the drive force changes by thousands of newtons per second)."""
    base = vehicle_config(B=B, T=T, seed=seed, sqp_iters=sqp_iters, pcg_tol=pcg_tol, dt=dt)
    rng = np.random.default_rng(seed + 7919)
    x_s = np.concatenate([base.x_s, np.zeros((B, 2))], 1)
    x_ref = np.concatenate([base.x_ref, np.zeros((B, T + 1, 2))], 2)
    lay = theta_layout("single_track", 6, 2, T)
    q_x = base.theta[:, lay["q"]:lay["q"] + 6].astype(np.float64)
    q_u = np.array([1.0, 1e-6]) * np.exp(rng.uniform(-1, 1, size=(B, 2)))
    r = np.array([0.1, 1e-8]) * np.exp(rng.uniform(-1, 1, size=(B, 2)))
    q = np.concatenate([q_x, q_u], 1)
    th = _pack_theta("single_track_rate", 8, 2, T, base.theta[:, :2].astype(np.float64), None, q, r, 10.0 * q)
    return Workload("vehicle_rate", "single_track_rate", 8, 2, T, dt, _f32(x_s), _f32(th), _f32(x_ref),
                    sqp_iters=sqp_iters, line_search=True, pcg_tol=pcg_tol,
                    u_target=_f32(np.zeros((B, 2))), extra=dict(features=base.extra["features"]))


def rigid_body_config(B=16, T=64, seed=0, sqp_iters=5, pcg_tol=1e-6, dt=0.02):
    """Quadrotor-like rigid body returning to hover at the origin: m ~ U[0.5, 1.5],
    J_i ~ U[0.005, 0.02]; x_0: position ~ N(0, 1), velocity ~ N(0, 0.25), angles ~ U[-0.3, 0.3],
    rates ~ N(0, 0.25)."""
    rng = np.random.default_rng(seed)
    m = rng.uniform(0.5, 1.5, size=B)
    J = rng.uniform(0.005, 0.02, size=(B, 3))
    q, r, qt = _cost_weights(rng, B, 12, 4)
    x_s = np.concatenate([rng.standard_normal((B, 3)), 0.5 * rng.standard_normal((B, 3)),
                          rng.uniform(-0.3, 0.3, size=(B, 3)), 0.5 * rng.standard_normal((B, 3))], 1)
    th = _pack_theta("rigid_body12", 12, 4, T, np.concatenate([m[:, None], J], 1), None, q, r, qt)
    return Workload("rigid_body12", "rigid_body12", 12, 4, T, dt, _f32(x_s), _f32(th),
                    _f32(np.zeros((B, T + 1, 12))), sqp_iters=sqp_iters, line_search=True,
                    pcg_tol=pcg_tol, u_target=_f32(rng.standard_normal((B, 4))))


def attitude_config(B=16, T=25, seed=0, sqp_iters=5, pcg_tol=1e-8, dt=0.1):
    """Attitude-rate stabilisation (App. B.1): diag J ~ U[0.1, 10]^3, w_0 ~ U[-1, 1]^3,
    Q = R = I nominal, terminal Q_T = Q; forward Euler dt = 0.1, T = 25."""
    rng = np.random.default_rng(seed)
    J = rng.uniform(0.1, 10.0, size=(B, 3))
    x_s = rng.uniform(-1, 1, size=(B, 3))
    q = np.ones((B, 3)); r = np.ones((B, 3))
    th = _pack_theta("attitude", 3, 3, T, J, None, q, r, q.copy())
    return Workload("attitude", "attitude", 3, 3, T, dt, _f32(x_s), _f32(th),
                    _f32(np.zeros((B, T + 1, 3))), sqp_iters=sqp_iters, line_search=True,
                    pcg_tol=pcg_tol, u_target=_f32(rng.standard_normal((B, 3))))


def uneven_mix(n_ocps=4096, T_lo=16, T_hi=128, seed=0, sqp_iters=10, pcg_tol=1e-6):
    """Mixed batch: one third each pendulum (2,1), cart-pole (4,1), kinematic bicycle (4,2),
    horizons T ~ U{T_lo..T_hi}.  Returns a list of single-OCP Workloads in submission order."""
    rng = np.random.default_rng(seed)
    kinds = rng.permutation(np.arange(n_ocps) % 3)
    Ts = rng.integers(T_lo, T_hi + 1, size=n_ocps)
    makers = [pendulum_config, cartpole_config, bicycle_config]
    out = []
    for i in range(n_ocps):
        w = makers[kinds[i]](B=1, T=int(Ts[i]), seed=int(rng.integers(1 << 31)),
                             sqp_iters=sqp_iters, pcg_tol=pcg_tol)
        out.append(w)
    return out


# ----------------------------------------------------------------------------------------
# Serving workload: Poisson arrivals of single-OCP requests of mixed state dimension and horizon.
SERVING_SHAPES = (("pendulum", 2, 1, 0.05), ("cartpole", 4, 1, 0.05), ("single_track", 6, 2, 0.02),
                  ("rigid_body12", 12, 4, 0.02))
_SINGLE = {"pendulum": pendulum_config, "cartpole": cartpole_config, "single_track": vehicle_config,
           "rigid_body12": rigid_body_config}


def serving_trace(rate, duration, seed=0, T_lo=16, T_hi=256, shapes=SERVING_SHAPES):
    """Requests arriving as a Poisson process of `rate` per second over `duration` seconds; each
    draws its model uniformly from `shapes` (nx 2, 4, 6, 12) and its horizon log-uniformly in
    [T_lo, T_hi].  Returns a list of dicts (arrival, model, nx, nu, T, dt, x_s, theta, x_ref)."""
    rng = np.random.default_rng(seed)
    n = int(rng.poisson(rate * duration))
    arrivals = np.sort(rng.uniform(0.0, duration, size=n))
    kinds = rng.integers(0, len(shapes), size=n)
    Ts = np.exp(rng.uniform(np.log(T_lo), np.log(T_hi + 1), size=n)).astype(int).clip(T_lo, T_hi)
    seeds = rng.integers(0, 1 << 31, size=n)
    out = [None] * n
    # draw all requests of one (model, horizon) together
    groups = {}
    for i in range(n):
        groups.setdefault((int(kinds[i]), int(Ts[i])), []).append(i)
    for (kind, T), idx in groups.items():
        model, nx, nu, dt = shapes[kind]
        w = _SINGLE[model](B=len(idx), T=T, seed=int(seeds[idx[0]]), dt=dt)
        for j, i in enumerate(idx):
            out[i] = dict(arrival=float(arrivals[i]), model=model, nx=nx, nu=nu, T=T, dt=dt,
                          x_s=w.x_s[j], theta=w.theta[j], x_ref=w.x_ref[j])
    return out
