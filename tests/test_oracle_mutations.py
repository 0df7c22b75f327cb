"""The oracle's pins catch plausible mistakes: each case plants one mistake in the oracle (a
transposed block, a flipped sign, a dropped term, a wrong constant), on the CPU and only for
the duration of the test, and checks that the pin written against it now fails.  A pin that
still passed under its mutation would not be pinning anything."""
import dataclasses
import sys

import numpy as np
import pytest

from oracle import backward as BW
from oracle import models as MD
from oracle import ocp as O
from oracle import schur as S
from oracle import sqp as SQ
from tests import test_oracle_cost as COST
from tests import test_oracle_implicit as IMPL
from tests import test_oracle_kkt as KKT
from tests import test_oracle_models as MODELS
from tests import test_oracle_rate as RATE
from tests import test_oracle_sqp as SQP
from tests import test_oracle_vjp as VJP


def _patch_all(monkeypatch, owner, name, new):
    """Replace `owner.name` in every loaded module that holds the same object (the oracle's
    modules import each other's functions by name)."""
    orig = getattr(owner, name)
    for mod in list(sys.modules.values()):
        if mod is not None and getattr(mod, name, None) is orig:
            monkeypatch.setattr(mod, name, new)
    return orig


def _schur_offdiag_transposed(mp):
    orig = S.schur_blocks

    def mutant(qp):
        D, Off = orig(qp)
        return D, np.swapaxes(Off, -1, -2)
    _patch_all(mp, S, "schur_blocks", mutant)


def _preconditioner_offdiag_sign(mp):
    orig = S.preconditioner_blocks

    def mutant(D, Off):
        Dinv, P = orig(D, Off)
        return Dinv, -P
    _patch_all(mp, S, "preconditioner_blocks", mutant)


def _gamma_drops_next_knot_term(mp):
    orig = S.gamma_spd

    def mutant(qp, q=None, r=None, d=None):
        g = orig(qp, q, r, d).copy()
        qq = qp.q if q is None else q
        g[:, 1:] += np.einsum("btij,btj->bti", qp.Ap, qq[:, 1:] / qp.Q[:, 1:])
        return g
    _patch_all(mp, S, "gamma_spd", mutant)


def _recovery_sign(mp):
    orig = S.recover_primal

    def mutant(qp, lam, q=None, r=None):
        x, u = orig(qp, lam, q, r)
        return -x, -u
    _patch_all(mp, S, "recover_primal", mutant)


def _linearise_drops_delta_form(mp):
    orig = O.linearise

    def mutant(ocp, z):
        qp = orig(ocp, z)
        x, _ = O.split_z(ocp, z)
        return dataclasses.replace(qp, q=qp.q + qp.Q * x)
    _patch_all(mp, O, "linearise", mutant)


def _kkt_rhs_constraint_sign(mp):
    orig = O.kkt_rhs

    def mutant(qp, b):
        mb, d = orig(qp, b)
        return mb, -d
    _patch_all(mp, O, "kkt_rhs", mutant)


def _merit_constraint_norm_doubled(mp):
    orig = SQ.merit_parts

    def mutant(ocp, z):
        c, g = orig(ocp, z)
        return c, 2.0 * g
    _patch_all(mp, SQ, "merit_parts", mutant)


def _rk4_weights(mp):
    def mutant(fc, x, u, ths, dt):
        k1 = fc(x, u, ths)
        k2 = fc([xi + 0.5 * dt * ki for xi, ki in zip(x, k1)], u, ths)
        k3 = fc([xi + 0.5 * dt * ki for xi, ki in zip(x, k2)], u, ths)
        k4 = fc([xi + dt * ki for xi, ki in zip(x, k3)], u, ths)
        return [xi + (dt / 4.0) * (a + b + c + d) for xi, a, b, c, d in zip(x, k1, k2, k3, k4)]
    _patch_all(mp, MD, "rk4", mutant)


def _cartpole_gravity_sign(mp):
    def mutant(self, x, u, ths):
        p, v, phi, w = x
        m_p, L = ths
        s, c = MD.sin(phi), MD.cos(phi)
        den = self.m_c + m_p * s * s
        pdd = (u[0] + m_p * s * (L * w * w - MD.GRAVITY * c)) / den
        wdd = (-(self.m_c + m_p) * MD.GRAVITY * s - u[0] * c - m_p * L * w * w * s * c) / (L * den)
        return [v, pdd, w, wdd]
    mp.setattr(MD.CartPole, "fc", mutant)


def _backward_drops_mixed_term(mp):
    orig = BW._phi_jets

    def mutant(ocp, z):
        g, h = orig(ocp, z)
        return g, np.zeros_like(h)
    _patch_all(mp, BW, "_phi_jets", mutant)


def _exact_hessian_curvature_sign(mp):
    def mutant(ocp, z, lam, b, h=None):
        nx, nu, T = ocp.nx, ocp.nu, ocp.T
        _, _, qd, rd, qtd = O.split_theta(ocp.one(b))
        if h is None:
            _, h = BW._phi_jets(ocp.one(b), z[b:b + 1])
            bb = 0
        else:
            bb = b
        L = lam[b].reshape(T + 1, nx)
        blocks = [np.diag(np.concatenate([qd[0], rd[0]]))
                  + np.einsum("i,ijk->jk", L[t + 1], h[bb, t][:, :nx + nu, :nx + nu]) for t in range(T)]
        return blocks + [np.diag(qtd[0])]
    _patch_all(mp, BW, "exact_hessian_blocks", mutant)


def _trapezoid_one_sided(mp):
    orig = MD.Model.residual

    def mutant(self, x, u, xn, ths, thk):
        if not self.implicit:
            return orig(self, x, u, xn, ths, thk)
        fa = self.fc(x, u, ths)
        return [xn[i] - x[i] - self.dt * fa[i] for i in range(self.nx)]
    mp.setattr(MD.Model, "residual", mutant)


def _pcg_beta_inverted(mp):
    def mutant(D, Off, Pd, Po, gamma, lam0, rel_tol, max_iter):
        mv = S.block_tridiag_matvec
        lam = lam0.copy()
        r = gamma - mv(D, Off, lam)
        rt = mv(Pd, Po, r)
        p = rt.copy()
        eta = np.einsum("bti,bti->b", r, rt)
        eta0 = np.einsum("bti,bti->b", gamma, mv(Pd, Po, gamma))
        iters = np.zeros(lam.shape[0], dtype=np.int64)
        for _ in range(max_iter):
            y = mv(D, Off, p)
            alpha = eta / np.einsum("bti,bti->b", p, y)
            lam += alpha[:, None, None] * p
            r -= alpha[:, None, None] * y
            rt = mv(Pd, Po, r)
            eta_new = np.einsum("bti,bti->b", r, rt)
            p = rt + (eta / eta_new)[:, None, None] * p      # planted: beta inverted
            eta = eta_new
            iters += 1
            if (eta <= rel_tol * eta0).all():
                break
        return lam, iters, eta, eta0
    _patch_all(mp, S, "pcg", mutant)


def _preconditioner_diagonal_not_inverted(mp):
    orig = S.preconditioner_blocks

    def mutant(D, Off):
        _, P = orig(D, Off)
        return D.copy(), P
    _patch_all(mp, S, "preconditioner_blocks", mutant)


def _fiala_cubic_sign(mp):
    def mutant(alpha, mu, c_alpha, fz):
        t = MD.tan(alpha)
        sat = 3.0 * mu * fz / c_alpha
        lin = (-1.0 * c_alpha * t + (c_alpha * c_alpha / (3.0 * mu * fz)) * MD.absval(t) * t
               + (c_alpha * c_alpha * c_alpha / (27.0 * mu * mu * fz * fz)) * t * t * t)  # planted sign
        slide = -1.0 * mu * fz * np.sign(MD.value(t))
        return MD.where(np.abs(MD.value(t)) < np.abs(MD.value(sat)), lin, slide)
    _patch_all(mp, MD, "fiala_lateral_force", mutant)


def _rigid_body_gyroscopic_sign(mp):
    orig = MD.RigidBody12.fc

    def mutant(self, x, u, ths):
        out = list(orig(self, x, u, ths))
        wx, wy, wz = x[9:12]
        m, jx, jy, jz = ths
        out[9] = out[9] + 2.0 * (wy * (jz * wz) - wz * (jy * wy)) / jx   # w x (J w) sign flipped in x
        return out
    mp.setattr(MD.RigidBody12, "fc", mutant)


def _cost_gradient_without_reference(mp):
    def mutant(ocp, z):
        _, _, qd, rd, qtd = O.split_theta(ocp)
        x, u = O.split_z(ocp, z)
        gx = x * qd[:, None, :]            # planted: x_ref left out
        gx[:, -1] = x[:, -1] * qtd
        return O.join_z(gx, u * rd[:, None, :])
    _patch_all(mp, O, "cost_gradient", mutant)


def _cost_value_terminal_factor(mp):
    orig = O.cost_value

    def mutant(ocp, z):
        _, _, _, _, qtd = O.split_theta(ocp)
        x, _ = O.split_z(ocp, z)
        dT = x[:, -1] - ocp.x_ref[:, -1]
        return orig(ocp, z) + 0.5 * np.einsum("bn,bn->b", dT ** 2, qtd)   # planted: no 1/2 at t = T
    _patch_all(mp, O, "cost_value", mutant)


def _lq_transition_transposed(mp):
    def mutant(self, x, u, ths, thk):
        nx, nu = self.nx, self.nu
        out = []
        for i in range(nx):
            acc = thk[nx * nx + nx * nu + i]
            for j in range(nx):
                acc = acc + thk[j * nx + i] * x[j]          # planted: Abar^T
            for j in range(nu):
                acc = acc + thk[nx * nx + i * nu + j] * u[j]
            out.append(acc)
        return out
    mp.setattr(MD.LQ, "step", mutant)


def _pendulum_gravity_sign(mp):
    def mutant(self, x, u, ths):
        phi, w = x
        m, L = ths
        return [w, -(MD.GRAVITY / L) * MD.sin(phi) + u[0] / (m * L * L)]
    mp.setattr(MD.Pendulum, "fc", mutant)


def _bicycle_sin_for_tan(mp):
    def mutant(self, x, u, ths):
        px, py, psi, v = x
        delta, a = u
        (lwb,) = ths
        return [v * MD.cos(psi), v * MD.sin(psi), v * MD.sin(delta) / lwb, a]
    mp.setattr(MD.KinematicBicycle, "fc", mutant)


def _banded_solve_swapped_entries(mp):
    orig = O.solve_kkt_banded

    def mutant(trip, rhs, nx, nu, T):
        sol = orig(trip, rhs, nx, nu, T).copy()
        sol[[0, 1]] = sol[[1, 0]]                        # planted: two unknowns swapped
        return sol
    _patch_all(mp, O, "solve_kkt_banded", mutant)


def _single_track_axles_swapped(mp):
    orig = MD.SingleTrackFiala.fc

    def mutant(self, x, u, ths):
        out = list(orig(self, x, u, ths))
        px, py, psi, r, vy, vx = x
        delta, fx = u
        mu, ca = ths
        a, b, m = self.a, self.b, self.m
        fyf = MD.fiala_lateral_force(MD.atan((vy + a * r) / vx) - delta, mu, ca, m * MD.GRAVITY * b / (a + b))
        fyr = MD.fiala_lateral_force(MD.atan((vy - b * r) / vx), mu, ca, m * MD.GRAVITY * a / (a + b))
        out[3] = (b * fyf * MD.cos(delta) - a * fyr) / self.Iz       # planted: lever arms swapped
        return out
    mp.setattr(MD.SingleTrackFiala, "fc", mutant)


def _attitude_torque_inertia(mp):
    orig = MD.Attitude.fc

    def mutant(self, x, u, ths):
        out = list(orig(self, x, u, ths))
        j1, j2, j3 = ths
        out[0] = out[0] - u[0] / j1 + u[0] / j2                        # planted: tau_1 / J_2
        return out
    mp.setattr(MD.Attitude, "fc", mutant)


def _rigid_body_euler_rate_sign(mp):
    orig = MD.RigidBody12.fc

    def mutant(self, x, u, ths):
        out = list(orig(self, x, u, ths))
        ro, pi = x[6], x[7]
        wy = x[10]
        out[6] = out[6] - 2.0 * MD.sin(ro) * (MD.sin(pi) / MD.cos(pi)) * wy     # planted: sign of a roll-rate term
        return out
    mp.setattr(MD.RigidBody12, "fc", mutant)


def _line_search_eta(mp):
    orig = SQ.line_search

    def mutant(ocp, z, z_plus, alphas=SQ.LS_ALPHAS, eta=SQ.LS_ETA):
        return orig(ocp, z, z_plus, alphas, 0.5)                     # planted: eta = 0.5
    _patch_all(mp, SQ, "line_search", mutant)


def _line_search_takes_last_passing_step(mp):
    orig = SQ.line_search

    def mutant(ocp, z, z_plus, alphas=SQ.LS_ALPHAS, eta=SQ.LS_ETA):
        alpha, diag = orig(ocp, z, z_plus, alphas, eta)
        for b in range(ocp.B):
            ok = np.where(diag["delta"][b] < 0.0)[0]
            if ok.size:
                alpha[b] = alphas[ok[-1]]                             # planted: last passing alpha
        return alpha, diag
    _patch_all(mp, SQ, "line_search", mutant)


def _dF_dtheta_cost_rows_without_reference(mp):
    orig = BW.dF_dtheta

    def mutant(ocp, z, lam, b, g=None, h=None):
        M = orig(ocp, z, lam, b, g, h)
        nx, nu, T = ocp.nx, ocp.nu, ocp.T
        _, _, o_q, _, o_qt, _ = O.theta_offsets(ocp.model, T)
        for t in range(T):
            M[O.x_index(nx, nu, t), o_q + np.arange(nx)] += ocp.x_ref[b, t]    # planted: x for x - x_ref
        M[O.x_index(nx, nu, T), o_qt + np.arange(nx)] += ocp.x_ref[b, T]
        return M
    _patch_all(mp, BW, "dF_dtheta", mutant)


def _dF_dtheta_fiala_columns_swapped(mp):
    orig = BW.dF_dtheta

    def mutant(ocp, z, lam, b, g=None, h=None):
        M = orig(ocp, z, lam, b, g, h)
        if ocp.model.name == "single_track":
            M[:, [0, 1]] = M[:, [1, 0]]                                  # planted: mu <-> C_alpha
        return M
    _patch_all(mp, BW, "dF_dtheta", mutant)


def _control_rate_without_dt(mp):
    def mutant(self, x, u, ths, thk):
        nb = self.base.nx
        xb, ub = list(x[:nb]), list(x[nb:])
        return list(self.base.step(xb, ub, ths, thk)) + [ub[i] + u[i] for i in range(self.nu)]   # planted: no dt
    mp.setattr(MD.ControlRate, "step", mutant)


def _implicit_a_plus_transposed(mp):
    orig = O.linearise

    def mutant(ocp, z):
        qp = orig(ocp, z)
        if not ocp.model.implicit:
            return qp
        return dataclasses.replace(qp, Ap=np.swapaxes(qp.Ap, -1, -2))   # planted: A^+ transposed
    _patch_all(mp, O, "linearise", mutant)


def _pd_floor_without_unit_bound(mp):
    def mutant(d):
        return np.maximum(d, O.PD_EPS * d.max(axis=-1, keepdims=True))   # planted: no max(1, .)
    _patch_all(mp, O, "pd_project_diag", mutant)


CASES = {
    "Schur off-diagonal block transposed (Eq. 10)": (_schur_offdiag_transposed,
                                                     lambda: KKT.test_schur_blocks_match_dense("lq")),
    "preconditioner off-diagonal sign (Eq. 10)": (_preconditioner_offdiag_sign,
                                                  KKT.test_preconditioner_matches_displayed_blocks),
    # the bicycle tracks a moving reference, so its Delta-form q_t is nonzero
    "gamma without the A^+ Q^-1 q_{t+1} term (App. A.2)": (_gamma_drops_next_knot_term,
                                                           lambda: KKT.test_schur_blocks_match_dense("kin_bicycle")),
    "recovery sign (Eq. 11)": (_recovery_sign, lambda: KKT.test_pcg_and_recovery_match_direct_kkt("cartpole")),
    "linear cost term without the Delta-form shift (Eq. 4)": (_linearise_drops_delta_form,
                                                              SQP.test_sqp_converges_to_kkt_point_cartpole),
    "constraint right-hand side sign (Eq. 6)": (_kkt_rhs_constraint_sign,
                                                lambda: KKT.test_lq_kkt_matches_riccati(0.01)),
    "merit constraint norm scaled (Algorithm 5)": (_merit_constraint_norm_doubled,
                                                   SQP.test_line_search_penalty_formula_on_infeasible_start),
    "RK4 stage weights": (_rk4_weights, MODELS.test_rk4_order_on_linear_system),
    "cart-pole gravity sign (App. B.2)": (_cartpole_gravity_sign, MODELS.test_cartpole_upright_linearisation_textbook),
    "backward without the mixed term d_theta(grad_z f^T lambda) (Eq. 3)": (_backward_drops_mixed_term,
                                                                           VJP.test_vjp_matches_fd_lq_all_parameters),
    "exact Hessian with the curvature sign flipped (Sec. 3.4)": (_exact_hessian_curvature_sign,
                                                                 VJP.test_vjp_exact_hessian_matches_fd_cartpole),
    "trapezoidal residual with one endpoint only": (_trapezoid_one_sided, IMPL.test_trapezoid_rule_is_second_order),
    "PCG beta inverted (Algorithm 4)": (_pcg_beta_inverted, lambda: KKT.test_pcg_and_recovery_match_direct_kkt("lq")),
    "preconditioner diagonal blocks not inverted (Eq. 10)": (_preconditioner_diagonal_not_inverted,
                                                             KKT.test_preconditioner_matches_displayed_blocks),
    "Fiala cubic term sign": (_fiala_cubic_sign, MODELS.test_fiala_curve_properties),
    "rigid-body gyroscopic term sign": (_rigid_body_gyroscopic_sign,
                                        lambda: MODELS.test_rigid_body_rotational_energy_conserved(MD.RigidBody12)),
    "cost gradient without the reference": (_cost_gradient_without_reference,
                                            COST.test_cost_gradient_matches_differences_with_reference),
    "terminal cost without its 1/2": (_cost_value_terminal_factor, COST.test_cost_value_hand_computed),
    "PD-projection floor without its unit bound (Sec. 3.1)": (_pd_floor_without_unit_bound,
                                                              COST.test_pd_projection_reading),
    "LQ transition matrix transposed (App. B.1)": (_lq_transition_transposed,
                                                  lambda: KKT.test_lq_kkt_matches_riccati(0.0)),
    "pendulum gravity sign": (_pendulum_gravity_sign, MODELS.test_pendulum_conserves_energy_unforced),
    "bicycle yaw rate with sin(delta) for tan(delta)": (_bicycle_sin_for_tan, MODELS.test_kinematic_bicycle_circle),
    "banded KKT solve with two unknowns swapped": (_banded_solve_swapped_entries,
                                                   lambda: KKT.test_banded_solve_matches_dense_lu("cartpole")),
    "single-track lever arms swapped in the yaw equation": (_single_track_axles_swapped,
                                                            MODELS.test_single_track_linear_lateral_dynamics_textbook),
    "attitude torque divided by the wrong inertia (App. B.1)": (
        _attitude_torque_inertia, lambda: MODELS.test_body_rates_respond_to_torque_at_rest(MD.Attitude)),
    "rigid-body Euler-rate term sign": (_rigid_body_euler_rate_sign,
                                        MODELS.test_rigid_body_kinematics_match_rotation_matrix),
    "decrease-test constant 0.5 for 0.4 (Algorithm 5)": (_line_search_eta,
                                                         SQP.test_line_search_closed_form_on_feasible_lq),
    "line search keeps the last passing step (Algorithm 5)": (_line_search_takes_last_passing_step,
                                                              SQP.test_line_search_closed_form_on_feasible_lq),
    "dF/dtheta cost-weight columns without the reference (Eq. 3)": (
        _dF_dtheta_cost_rows_without_reference, lambda: VJP.test_dF_dtheta_matches_differenced_residual("kin_bicycle")),
    "dF/dtheta friction and cornering-stiffness columns swapped (vehicle, Eq. 3)": (
        _dF_dtheta_fiala_columns_swapped, lambda: VJP.test_dF_dtheta_matches_differenced_residual("single_track")),
    "control-rate augmentation integrating the rate without dt (App. B.3)": (
        _control_rate_without_dt, RATE.test_augmented_step_reproduces_the_base_trajectory),
    "implicit integrator's A^+ transposed (Eq. 4)": (
        _implicit_a_plus_transposed,
        lambda: IMPL.test_implicit_linearisation_matches_differences(IMPL.workloads.cartpole_config)),
}


@pytest.mark.parametrize("case", list(CASES))
def test_pin_fails_under_planted_mistake(case, monkeypatch):
    plant, pin = CASES[case]
    plant(monkeypatch)
    with pytest.raises(AssertionError):
        pin()
