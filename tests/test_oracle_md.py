"""Pins of the oracle's molecular-dynamics pieces (gauge action and force, link update, leapfrog,
R-algorithm step).

* unit links: S_g = 0, mean plaquette 1, no gauge force; S_g is gauge invariant;
* the gauge gradient and force against central differences of S_g;
* exp(eps P) U with P = 0 returns U, and with diagonal P the diagonal phases exp(i eps theta);
* leapfrog with gauge, pseudofermion and determinant forces: Delta H falls as eps^2 (halving eps
  divides it by about 4) and the trajectory is reversible;
* the R-algorithm step is reversible for fixed noise (its pseudofermion is drawn at the half step,
  which the forward and the reversed step share).
"""

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import dirac, lattice, evenodd, force, md
from paper_0910_0262_gb300 import synth
from helpers import rel_l2, lattice_shape

KAPPA, CSW, BETA = 0.12, 1.0, 5.6


def random_momenta(shape, rng):
    p = rng.standard_normal(tuple(shape) + (8,))
    return np.einsum('...a,aij->...ij', 1j * p, synth.T_GEN)


def test_unit_links():
    dims = (4, 2, 2, 4)
    U = np.broadcast_to(np.eye(3, dtype=complex), lattice_shape(dims) + (4, 3, 3)).copy()
    assert abs(md.gauge_action(U, BETA)) < 1e-12
    assert abs(md.mean_plaquette(U) - 1.0) < 1e-15
    assert np.max(np.abs(md.gauge_force(U, BETA))) < 1e-14


def test_gauge_action_is_gauge_invariant():
    dims = (4, 2, 4, 2)
    U, _ = synth.make_problem(dims, 0.5, 51)
    rng = np.random.default_rng(3)
    Om = synth.random_su3_field(lattice_shape(dims), rng)
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[..., mu, :, :] = Om @ U[..., mu, :, :] @ dirac.dagger(lattice.shift(Om, mu, +1))
    S = md.gauge_action(U, BETA)
    assert S > 1.0
    assert abs(md.gauge_action(Ug, BETA) - S) <= 1e-12 * S


def test_gauge_force_against_finite_differences():
    dims = (4, 2, 2, 4)
    U, _ = synth.make_problem(dims, 0.5, 52)
    G = md.gauge_gradient(U, BETA)
    F = md.gauge_force(U, BETA)
    rng = np.random.default_rng(7)
    h = 1e-5
    for _ in range(4):
        site = tuple(int(rng.integers(0, n)) for n in U.shape[:4])
        mu = int(rng.integers(0, 4))
        D = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
        Up, Um = U.copy(), U.copy()
        Up[site + (mu,)] += h * D
        Um[site + (mu,)] -= h * D
        fd = (md.gauge_action(Up, BETA) - md.gauge_action(Um, BETA)) / (2 * h)
        an = float(np.real(np.sum(np.conj(G[site + (mu,)]) * D)))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))
        a = int(rng.integers(0, 8))
        Up, Um = U.copy(), U.copy()
        Up[site + (mu,)] = expm(1j * h * synth.T_GEN[a]) @ U[site + (mu,)]
        Um[site + (mu,)] = expm(-1j * h * synth.T_GEN[a]) @ U[site + (mu,)]
        fd = (md.gauge_action(Up, BETA) - md.gauge_action(Um, BETA)) / (2 * h)
        an = 2.0 * np.imag(np.trace(F[site + (mu,)] @ synth.T_GEN[a]))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


def test_link_update_special_cases():
    dims = (2, 2, 2, 2)
    U, _ = synth.make_problem(dims, 0.5, 53)
    assert rel_l2(md.update_links(U, np.zeros_like(U), 0.1), U) < 1e-14
    rng = np.random.default_rng(9)
    th = rng.standard_normal(U.shape[:5] + (3,))
    th -= th.mean(axis=-1, keepdims=True)
    P = np.zeros_like(U)
    for k in range(3):
        P[..., k, k] = 1j * th[..., k]
    want = np.exp(0.3j * th)[..., :, None] * U
    assert rel_l2(md.update_links(U, P, 0.3), want) < 1e-14


def _setup(dims, seed):
    U, eta = synth.make_problem(dims, 0.3, seed, nrhs=2)
    rng = np.random.default_rng(seed)
    P = random_momenta(U.shape[:5], rng)
    op = evenodd.SchurOperator(U, KAPPA, CSW)
    phis = [op.Mhat_dag(e) for e in eta]
    return U, P, eta, phis


def test_leapfrog_energy_error_is_second_order_and_reversible():
    dims = (2, 2, 2, 4)
    U, P, eta, phis = _setup(dims, 54)
    H0 = md.hamiltonian(U, P, BETA, KAPPA, CSW, phis, True)
    dH = []
    for n in (4, 8):
        U1, P1 = md.leapfrog(U, P, 0.2 / n, n, BETA, KAPPA, CSW, phis, True)
        dH.append(abs(md.hamiltonian(U1, P1, BETA, KAPPA, CSW, phis, True) - H0))
    assert dH[0] > 1e-8
    assert 3.0 < dH[0] / dH[1] < 5.5, dH
    U1, P1 = md.leapfrog(U, P, 0.05, 4, BETA, KAPPA, CSW, phis, True)
    U2, P2 = md.leapfrog(U1, -P1, 0.05, 4, BETA, KAPPA, CSW, phis, True)
    assert rel_l2(U2, U) < 1e-10 and rel_l2(-P2, P) < 1e-9


def test_r_step_is_reversible_for_fixed_noise():
    dims = (2, 2, 2, 4)
    U, P, eta, _ = _setup(dims, 55)
    U1, P1 = md.r_step(U, P, eta, 0.05, BETA, KAPPA, CSW)
    assert rel_l2(U1, U) > 1e-4
    U2, P2 = md.r_step(U1, -P1, eta, 0.05, BETA, KAPPA, CSW)
    assert rel_l2(U2, U) < 1e-10 and rel_l2(-P2, P) < 1e-9
