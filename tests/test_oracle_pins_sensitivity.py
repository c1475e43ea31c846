"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin catches each.

Each mutation is applied with monkeypatch to a copy of one oracle function; the
corresponding pin from the other oracle tests must then fail.
"""

import numpy as np
import pytest

from oracle import dirac, force, evenodd, cloverdet, md, measure
import test_oracle_operator as t_op
import test_oracle_md as t_md
import test_oracle_cloverdet as t_cd
import test_oracle_clover as t_cl
import test_oracle_force as t_fo
import test_oracle_measure as t_me


def _fails(fn, *args):
    try:
        fn(*args)
    except AssertionError:
        return True
    return False


def test_backward_hop_without_dagger_is_caught(monkeypatch):
    orig_dagger = dirac.dagger

    def hopping_nodag(U, psi, t_bc):
        dims = psi.shape[3], psi.shape[2], psi.shape[1], psi.shape[0]
        s = dirac.boundary_sign(dims, t_bc)
        out = np.zeros_like(psi, dtype=complex)
        for mu in range(4):
            Umu = U[..., mu, :, :] * s[..., mu, None, None]
            out += dirac.spin_mul(dirac.ONE4 - dirac.GAMMA[mu], dirac.colour_mul(Umu, dirac.shift(psi, mu, 1)))
            out += dirac.spin_mul(dirac.ONE4 + dirac.GAMMA[mu],
                                  dirac.colour_mul(dirac.shift(Umu, mu, -1), dirac.shift(psi, mu, -1)))
        return out
    monkeypatch.setattr(dirac, "hopping", hopping_nodag)
    assert _fails(t_op.test_gamma5_hermiticity_and_adjoint, (4, 2, 6, 4), 1)
    assert orig_dagger is dirac.dagger


def test_wrong_projector_sign_is_caught(monkeypatch):
    orig = dirac.hopping

    def hopping_swapped(U, psi, t_bc):
        # (1 + g) forward and (1 - g) backward
        g5 = dirac.GAMMA.copy()
        monkeypatch.setattr(dirac, "GAMMA", -g5)
        try:
            return orig(U, psi, t_bc)
        finally:
            monkeypatch.setattr(dirac, "GAMMA", g5)
    monkeypatch.setattr(dirac, "hopping", hopping_swapped)
    assert _fails(t_op.test_free_field_plane_wave, (4, 6, 2, 8))


def test_field_strength_normalisation_is_caught(monkeypatch):
    orig = dirac.field_strength
    monkeypatch.setattr(dirac, "field_strength", lambda U, mu, nu: 2.0 * orig(U, mu, nu))
    assert _fails(t_cl.test_uniform_abelian_flux_closed_form)


def test_misplaced_leaf_is_caught(monkeypatch):
    orig = dirac.leaf_paths

    def leaves_wrong(mu, nu):
        p = orig(mu, nu)
        # replace the third leaf by a copy of the first: the sum of four leaves is wrong
        return [p[0], p[1], p[0], p[3]]
    monkeypatch.setattr(dirac, "leaf_paths", leaves_wrong)
    assert _fails(t_cl.test_random_abelian_field_strength_from_plaquette_angles)


def test_missing_kappa2_on_odd_clover_force_is_caught(monkeypatch):
    orig = force.solution_fields

    def fields_wrong(op, X_e):
        X, Y, W = orig(op, X_e)
        return X, Y, Y  # W should carry kappa^2 on the odd sites
    monkeypatch.setattr(force, "solution_fields", fields_wrong)
    assert _fails(t_fo.test_force_against_finite_differences, 1.0)


def test_transposed_insertion_is_caught(monkeypatch):
    orig = force.insert

    def insert_transposed(G, U, path, C):
        orig(G, U, path, np.swapaxes(C, -1, -2))
    monkeypatch.setattr(force, "insert", insert_transposed)
    assert _fails(t_fo.test_force_against_finite_differences, 0.0)


def test_schur_sign_is_caught(monkeypatch):
    def mhat_plus(self, x_e):
        t_o = self.site(self.A_oo_inv, self.D_oe(x_e))
        return self.site(self.A_ee, x_e) + self.kappa ** 2 * self.D_eo(t_o)
    monkeypatch.setattr(evenodd.SchurOperator, "Mhat", mhat_plus)
    import test_oracle_solve as t_so
    assert _fails(t_so.test_schur_complement_matches_dense_full_solve, (2, 2, 2, 2), 0.5, 1)


def test_determinant_coefficient_without_traceless_part_is_caught(monkeypatch):
    orig = cloverdet.coefficients

    def coeffs_with_trace(op):
        C = orig(op)
        odd = np.broadcast_to((np.indices(op.U.shape[:4]).sum(axis=0) % 2 == 1)[..., None, None], C.shape[1:])
        return C + 0.01j * np.where(odd, np.eye(3), 0.0)[None]
    monkeypatch.setattr(cloverdet, "coefficients", coeffs_with_trace)
    assert _fails(t_cd.test_force_against_finite_differences)


def test_determinant_of_even_sites_is_caught(monkeypatch):
    monkeypatch.setattr(cloverdet, "action", lambda op: -2.0 * cloverdet.logdet(op)[0])
    assert _fails(t_cd.test_small_csw_second_order_closed_form)


def test_reconstruction_sign_is_caught(monkeypatch):
    monkeypatch.setattr(cloverdet, "reconstruct_odd",
                        lambda op, x_e, b_o: evenodd.SchurOperator.site(op.A_oo_inv, b_o - op.kappa * op.D_oe(x_e)))
    assert _fails(t_cd.test_full_solve_with_both_parities_matches_dense, (2, 2, 2, 2), 24)


def test_gauge_force_factor_is_caught(monkeypatch):
    orig = md.gauge_force
    monkeypatch.setattr(md, "gauge_force", lambda U, beta: 0.5 * orig(U, beta))
    assert _fails(t_md.test_leapfrog_energy_error_is_second_order_and_reversible)


def test_noise_drawn_before_the_half_step_is_caught(monkeypatch):
    def r_step_early(U, P, eta, eps, beta, kappa, csw, with_det=True):
        op = evenodd.SchurOperator(U, kappa, csw)
        phis = [op.Mhat_dag(e) for e in eta]
        Uh = md.update_links(U, P, eps / 2.0)
        P = P - eps * md.total_force(Uh, beta, kappa, csw, phis, with_det)
        return md.update_links(Uh, P, eps / 2.0), P
    monkeypatch.setattr(md, "r_step", r_step_early)
    assert _fails(t_md.test_r_step_is_reversible_for_fixed_noise)


def test_polyakov_along_the_wrong_direction_is_caught(monkeypatch):
    def along_z(U):
        Z = U.shape[1]
        prod = U[:, 0, ..., 2, :, :]
        for z in range(1, Z):
            prod = prod @ U[:, z, ..., 2, :, :]
        return complex(np.mean(np.trace(prod, axis1=-2, axis2=-1)) / 3.0)
    monkeypatch.setattr(measure, "polyakov_loop", along_z)
    assert _fails(t_me.test_polyakov_unit_and_closed_form)


def test_polyakov_product_in_reverse_order_is_caught(monkeypatch):
    def reversed_product(U):
        T = U.shape[0]
        prod = U[T - 1, ..., 3, :, :]
        for t in range(T - 2, -1, -1):
            prod = prod @ U[t, ..., 3, :, :]
        return complex(np.mean(np.trace(prod, axis1=-2, axis2=-1)) / 3.0)
    monkeypatch.setattr(measure, "polyakov_loop", reversed_product)
    assert _fails(t_me.test_polyakov_centre_and_gauge_transformations)


def test_pbp_without_the_odd_sites_is_caught(monkeypatch):
    def even_only(op, eta_e, eta_o, tol=1e-12):
        x_e, _ = measure.solve_full(op, eta_e, eta_o, tol)
        return float(np.vdot(eta_e.reshape(-1), x_e.reshape(-1)).real / (4.0 * eta_e.shape[0]))
    monkeypatch.setattr(measure, "pbp", even_only)
    assert _fails(t_me.test_pbp_estimator_against_dense_inverse)


def test_link_update_with_the_wrong_sign_is_caught(monkeypatch):
    orig = md.update_links
    monkeypatch.setattr(md, "update_links", lambda U, P, eps: orig(U, P, -eps))
    assert _fails(t_md.test_link_update_special_cases)


def test_reunitarisation_without_conjugate_is_caught(monkeypatch):
    def reunit_noconj(U):
        r0 = U[..., 0, :] / np.linalg.norm(U[..., 0, :], axis=-1, keepdims=True)
        r1 = U[..., 1, :] - np.sum(np.conj(r0) * U[..., 1, :], axis=-1, keepdims=True) * r0
        r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
        return np.stack([r0, r1, np.cross(r0, r1)], axis=-2)
    monkeypatch.setattr(md, "reunitarise", reunit_noconj)
    assert _fails(t_md.test_link_update_special_cases)
