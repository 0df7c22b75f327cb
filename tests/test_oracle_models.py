"""Pins of the oracle's derivative machinery and dynamics models against things other than
the oracle: complex-step and central differences, closed-form linearisations, conserved
quantities of the equations of motion, and textbook tyre-curve properties."""
import numpy as np
import pytest

from oracle import jet
from oracle.jet import Jet
from oracle.models import (make_model, CartPole, Pendulum, RigidBody12, Attitude,
                           KinematicBicycle, SingleTrackFiala, fiala_lateral_force, GRAVITY)

RNG = np.random.default_rng(1234)


def _random_state(model, n):
    if model.name == "single_track":
        x = np.stack([RNG.normal(0, 5, n), RNG.normal(0, 5, n), RNG.uniform(-1, 1, n),
                      RNG.normal(0, 0.2, n), RNG.normal(0, 0.3, n), RNG.uniform(8, 15, n)], 1)
        u = np.stack([RNG.normal(0, 0.02, n), RNG.normal(0, 500, n)], 1)
        th = np.stack([RNG.uniform(0.3, 1.1, n), RNG.uniform(5e4, 1.5e5, n)], 1)
        return x, u, th
    x = RNG.normal(0, 0.7, (n, model.nx))
    u = RNG.normal(0, 0.7, (n, model.nu))
    th = {"pendulum": lambda: np.stack([RNG.uniform(0.5, 2, n), RNG.uniform(0.5, 1.5, n)], 1),
          "cartpole": lambda: np.stack([RNG.uniform(0.05, 0.2, n), RNG.uniform(0.3, 0.7, n)], 1),
          "kin_bicycle": lambda: RNG.uniform(2.5, 3.0, (n, 1)),
          "rigid_body12": lambda: np.concatenate([RNG.uniform(0.5, 1.5, (n, 1)),
                                                  RNG.uniform(0.005, 0.02, (n, 3))], 1),
          "attitude": lambda: RNG.uniform(0.1, 10, (n, 3))}[model.name]()
    if model.name == "kin_bicycle":
        u[:, 0] = RNG.uniform(-0.4, 0.4, n)
    if model.name == "rigid_body12":
        x[:, 6:9] = RNG.uniform(-0.5, 0.5, (n, 3))
    return x, u, th


def _step_plain(model, x, u, th):
    out = model.step([x[:, i] for i in range(model.nx)], [u[:, i] for i in range(model.nu)],
                     [th[:, i] for i in range(model.p_shared)], [])
    return np.stack([np.broadcast_to(o, x.shape[:1]) for o in out], 1)


def _step_jet(model, x, u, th):
    k = model.nx + model.nu + model.p_shared
    xs = [Jet.seed(x[:, i], i, k) for i in range(model.nx)]
    us = [Jet.seed(u[:, i], model.nx + i, k) for i in range(model.nu)]
    ts = [Jet.seed(th[:, i], model.nx + model.nu + i, k) for i in range(model.p_shared)]
    return model.step(xs, us, ts, [])


ANALYTIC = ["pendulum", "cartpole", "kin_bicycle", "rigid_body12", "attitude"]


@pytest.mark.parametrize("name", ANALYTIC)
def test_jet_jacobian_matches_complex_step(name):
    """First derivatives of Phi (the A_t, B_t of Eq. 4 and dPhi/dtheta) vs complex step."""
    model = make_model(name, dt=0.05)
    x, u, th = _random_state(model, 16)
    out = _step_jet(model, x, u, th)
    J = np.stack([o.g for o in out], 1)      # (n, nx, k)
    v = np.concatenate([x, u, th], 1)
    h = 1e-30
    for j in range(v.shape[1]):
        vc = v.astype(complex)
        vc[:, j] += 1j * h
        xc, uc, tc = vc[:, :model.nx], vc[:, model.nx:model.nx + model.nu], vc[:, model.nx + model.nu:]
        Jcs = _step_plain(model, xc, uc, tc).imag / h
        np.testing.assert_allclose(J[:, :, j], Jcs, rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("name", ANALYTIC + ["single_track"])
def test_jet_hessian_matches_differenced_jacobian(name):
    """Second derivatives (used by dF/dtheta and the exact Hessian) vs central differences
    of the complex-step / jet Jacobian."""
    model = make_model(name, dt=0.05 if name != "single_track" else 0.02)
    x, u, th = _random_state(model, 8)
    out = _step_jet(model, x, u, th)
    H = np.stack([o.h for o in out], 1)       # (n, nx, k, k)
    v = np.concatenate([x, u, th], 1)
    k = v.shape[1]
    for j in range(k):
        step = 1e-5 * max(1.0, np.abs(v[:, j]).max())
        vp, vm = v.copy(), v.copy()
        vp[:, j] += step
        vm[:, j] -= step
        sp = lambda vv: _step_jet(model, vv[:, :model.nx], vv[:, model.nx:model.nx + model.nu],
                                   vv[:, model.nx + model.nu:])
        Jp = np.stack([o.g for o in sp(vp)], 1)
        Jm = np.stack([o.g for o in sp(vm)], 1)
        Hfd = (Jp - Jm) / (2 * step)
        scale = np.abs(H[:, :, :, j]).max() + 1e-12
        assert np.abs(H[:, :, :, j] - Hfd).max() <= 1e-5 * scale + 1e-9


def test_jet_elementary_rules():
    """Closed forms: d/dx [sin(x) x^2] and second derivative; d/dx atan(x); 1/x."""
    xv = np.array([0.3, -1.2, 2.0])
    x = Jet.seed(xv, 0, 1)
    y = jet.sin(x) * x * x
    np.testing.assert_allclose(y.g[:, 0], np.cos(xv) * xv**2 + 2 * xv * np.sin(xv), rtol=1e-14)
    np.testing.assert_allclose(y.h[:, 0, 0], -np.sin(xv) * xv**2 + 4 * xv * np.cos(xv) + 2 * np.sin(xv),
                               rtol=1e-13)
    z = jet.atan(x)
    np.testing.assert_allclose(z.h[:, 0, 0], -2 * xv / (1 + xv**2) ** 2, rtol=1e-14)
    w = 1.0 / x
    np.testing.assert_allclose(w.h[:, 0, 0], 2 / xv**3, rtol=1e-14)


def test_cartpole_upright_linearisation_textbook():
    """Upright (phi = 0) linearisation of the cart-pole: p'' = (u - m_p g phi)/m_c,
    phi'' = ((m_c + m_p) g phi - u)/(L m_c)."""
    model = CartPole(0.05)
    mp, L = 0.1, 0.5
    k = 5
    xs = [Jet.seed(np.zeros(1), i, k) for i in range(4)]
    us = [Jet.seed(np.zeros(1), 4, k)]
    f = model.fc(xs, us, [mp, L])
    J = np.stack([fi.g[0] for fi in f])
    expect = np.array([[0, 1, 0, 0, 0],
                       [0, 0, -mp * GRAVITY / 1.0, 0, 1.0 / 1.0],
                       [0, 0, 0, 1, 0],
                       [0, 0, (1.0 + mp) * GRAVITY / (L * 1.0), 0, -1.0 / (L * 1.0)]])
    np.testing.assert_allclose(J, expect, atol=1e-14)


def _energy_rate(model, energy, x, th):
    """dE/dt = grad E . f(x, 0): zero for conservative, unforced dynamics."""
    k = model.nx
    xs = [Jet.seed(x[:, i], i, k) for i in range(model.nx)]
    E = energy(xs, th)
    f = model.fc([x[:, i] for i in range(model.nx)], [np.zeros(len(x))] * model.nu,
                 [th[:, i] for i in range(th.shape[1])])
    return np.einsum("bi,ib->b", E.g, np.stack([np.broadcast_to(fi, x.shape[:1]) for fi in f]))


def test_cartpole_conserves_energy_unforced():
    model = CartPole(0.05)
    x, _, th = _random_state(model, 32)
    mc = model.m_c

    def energy(xs, th):
        p, v, phi, w = xs
        mp, L = th[:, 0], th[:, 1]
        return (0.5 * (mc + mp) * v * v + mp * L * jet.cos(phi) * v * w + 0.5 * mp * L * L * w * w
                + mp * GRAVITY * L * jet.cos(phi))
    rate = _energy_rate(model, energy, x, th)
    assert np.abs(rate).max() < 1e-12


def test_pendulum_conserves_energy_unforced():
    model = Pendulum(0.05)
    x, _, th = _random_state(model, 32)

    def energy(xs, th):
        phi, w = xs
        m, L = th[:, 0], th[:, 1]
        return 0.5 * m * L * L * w * w + m * GRAVITY * L * jet.cos(phi)
    assert np.abs(_energy_rate(model, energy, x, th)).max() < 1e-12


@pytest.mark.parametrize("cls", [RigidBody12, Attitude])
def test_rigid_body_rotational_energy_conserved(cls):
    """Torque-free Euler equations conserve 1/2 w^T J w."""
    model = cls(0.05)
    x, _, th = _random_state(model, 32)
    off = 9 if cls is RigidBody12 else 0
    jo = 1 if cls is RigidBody12 else 0

    def energy(xs, th):
        w = xs[off:off + 3]
        return 0.5 * sum(th[:, jo + i] * w[i] * w[i] for i in range(3))
    rate = _energy_rate(model, energy, x, th)
    assert np.abs(rate).max() < 1e-12


def test_rigid_body_hover_is_equilibrium():
    model = RigidBody12(0.02)
    x = np.zeros((1, 12)); u = np.zeros((1, 4)); th = np.array([[1.2, 0.01, 0.01, 0.02]])
    np.testing.assert_allclose(_step_plain(model, x, u, th), 0.0, atol=1e-14)


def test_kinematic_bicycle_circle():
    """Constant steer and speed: the rear axle follows a circle of radius l_wb / tan(delta)."""
    model = KinematicBicycle(0.01)
    lwb, delta, v = 2.7, 0.2, 3.0
    x = np.array([[0.0, 0.0, 0.0, v]]); u = np.array([[delta, 0.0]]); th = np.array([[lwb]])
    R = lwb / np.tan(delta)
    for _ in range(300):
        x = _step_plain(model, x, u, th)
        assert abs(np.hypot(x[0, 0], x[0, 1] - R) - R) < 1e-9
    assert abs(x[0, 3] - v) < 1e-14


def test_fiala_curve_properties():
    """Fiala brush model: slope -C at alpha = 0, saturation -mu Fz sign(alpha) beyond alpha_sl,
    value and slope continuous at alpha_sl."""
    mu, C, Fz = 0.9, 8e4, 7000.0
    a = Jet.seed(np.array([0.0]), 0, 1)
    F = fiala_lateral_force(a, mu, C, Fz)
    assert abs(F.g[0, 0] + C) < 1e-9
    a_sl = np.arctan(3 * mu * Fz / C)
    for s in (1.0, -1.0):
        lo = fiala_lateral_force(Jet.seed(np.array([s * a_sl * (1 - 1e-9)]), 0, 1), mu, C, Fz)
        hi = fiala_lateral_force(Jet.seed(np.array([s * a_sl * (1 + 1e-9)]), 0, 1), mu, C, Fz)
        assert abs(lo.v[0] - hi.v[0]) < 1e-3
        assert abs(hi.v[0] + s * mu * Fz) < 1e-9
        assert abs(lo.g[0, 0]) < 1e-2 * C and hi.g[0, 0] == 0.0
    big = fiala_lateral_force(np.array([0.5, -0.5]), mu, C, Fz)
    np.testing.assert_allclose(big, [-mu * Fz, mu * Fz])


def test_single_track_straight_line():
    """No steer, no yaw, no lateral speed: no tyre lateral force, Vx' = Fx/m."""
    model = SingleTrackFiala(0.02)
    x = np.array([[0.0, 0.0, 0.0, 0.0, 0.0, 10.0]])
    u = np.array([[0.0, 1476.0]])
    th = np.array([[0.9, 8e4]])
    f = model.fc([x[:, i] for i in range(6)], [u[:, i] for i in range(2)], [th[:, 0], th[:, 1]])
    np.testing.assert_allclose(np.array([np.broadcast_to(fi, (1,))[0] for fi in f]),
                               [10.0, 0.0, 0.0, 0.0, 0.0, 1.0], atol=1e-12)


def test_rk4_order_on_linear_system():
    """RK4 of x' = a x matches exp(a dt) to O(dt^5) per step (textbook property)."""
    from oracle.models import rk4
    a = -1.3
    for dt in (0.1, 0.05):
        out = rk4(lambda x, u, th: [a * x[0]], [np.array([1.0])], [], [], dt)[0][0]
        series = 1 + a * dt + (a * dt) ** 2 / 2 + (a * dt) ** 3 / 6 + (a * dt) ** 4 / 24
        assert abs(out - series) < 1e-15
        assert abs(out - np.exp(a * dt)) < (abs(a) * dt) ** 5 / 100


def test_single_track_linear_lateral_dynamics_textbook():
    """Straight running (Vy = r = delta = 0, Vx = V): the Jacobian of the lateral states is the
    textbook linear single-track model with axle cornering stiffness C (the Fiala slope at zero
    slip): dr'/d(Vy, r, delta) = (-C (a - b)/(V Iz), -C (a^2 + b^2)/(V Iz), C a / Iz),
    dVy'/d(Vy, r, delta) = (-2C/(m V), -C (a - b)/(m V) - V, C / m)."""
    model = SingleTrackFiala(0.02)
    V, C, mu = 12.0, 8e4, 0.9
    a, b, m, Iz = model.a, model.b, model.m, model.Iz
    k = 8
    vals = [0.0, 0.0, 0.3, 0.0, 0.0, V]
    xs = [Jet.seed(np.array([vals[i]]), i, k) for i in range(6)]
    us = [Jet.seed(np.array([0.0]), 6, k), Jet.seed(np.array([0.0]), 7, k)]
    f = model.fc(xs, us, [mu, C])
    d_r = f[3].g[0][[4, 3, 6]]
    d_vy = f[4].g[0][[4, 3, 6]]
    np.testing.assert_allclose(d_r, [-C * (a - b) / (V * Iz), -C * (a * a + b * b) / (V * Iz), C * a / Iz],
                               rtol=1e-12)
    np.testing.assert_allclose(d_vy, [-2 * C / (m * V), -C * (a - b) / (m * V) - V, C / m], rtol=1e-12)


@pytest.mark.parametrize("cls", [RigidBody12, Attitude])
def test_body_rates_respond_to_torque_at_rest(cls):
    """At zero body rates (and level attitude) the Euler equations reduce to w' = tau / J."""
    model = cls(0.05)
    rng = np.random.default_rng(4)
    tau = rng.standard_normal(3)
    if cls is RigidBody12:
        th = [1.2, 0.01, 0.02, 0.03]
        J = np.array(th[1:])
        f = model.fc([np.zeros(1)] * 12, [np.zeros(1)] + [np.array([t]) for t in tau], [np.array([v]) for v in th])
        wdot = np.array([np.broadcast_to(fi, (1,))[0] for fi in f[9:12]])
    else:
        th = [0.5, 0.7, 0.9]
        J = np.array(th)
        f = model.fc([np.zeros(1)] * 3, [np.array([t]) for t in tau], [np.array([v]) for v in th])
        wdot = np.array([np.broadcast_to(fi, (1,))[0] for fi in f])
    np.testing.assert_allclose(wdot, tau / J, rtol=1e-14)


def _rot_zyx(ro, pi, ya):
    """Textbook ZYX rotation body -> world: Rz(yaw) Ry(pitch) Rx(roll)."""
    cr, sr, cp, sp, cy, sy = np.cos(ro), np.sin(ro), np.cos(pi), np.sin(pi), np.cos(ya), np.sin(ya)
    Rz = np.array([[cy, -sy, 0], [sy, cy, 0], [0, 0, 1]])
    Ry = np.array([[cp, 0, sp], [0, 1, 0], [-sp, 0, cp]])
    Rx = np.array([[1, 0, 0], [0, cr, -sr], [0, sr, cr]])
    return Rz @ Ry @ Rx


def test_rigid_body_kinematics_match_rotation_matrix():
    """Thrust acts along the body z axis, R e3, and the Euler-angle rates reproduce the body
    rates: dR/dt (along the oracle's angle rates) = R [w]x."""
    model = RigidBody12(0.02)
    rng = np.random.default_rng(7)
    for _ in range(5):
        ang = rng.uniform(-0.6, 0.6, 3)
        w = rng.standard_normal(3)
        dT = rng.uniform(-2.0, 2.0)
        th = [1.3, 0.011, 0.013, 0.021]
        x = [np.array([v]) for v in np.concatenate([np.zeros(6), ang, w])]
        u = [np.array([dT]), np.zeros(1), np.zeros(1), np.zeros(1)]
        f = np.array([np.broadcast_to(fi, (1,))[0] for fi in model.fc(x, u, [np.array([v]) for v in th])])
        R = _rot_zyx(*ang)
        acc = (th[0] * GRAVITY + dT) / th[0]
        np.testing.assert_allclose(f[3:6] + [0.0, 0.0, GRAVITY], acc * R[:, 2], rtol=1e-12, atol=1e-12)
        h = 1e-6
        dR = (_rot_zyx(*(ang + h * f[6:9])) - _rot_zyx(*(ang - h * f[6:9]))) / (2 * h)
        W = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
        np.testing.assert_allclose(dR, R @ W, atol=1e-8)
