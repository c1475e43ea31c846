"""Pins of the oracle's fermion force against finite differences and symmetries.

* G (Wirtinger gradient) against central differences of S along random complex
  directions of single links (S from dense solves, no CG);
* F (Lie-algebra force) against central differences along U -> exp(+-i eps T_a) U;
* operator-level difference: dS = -2 Re <Y, dMhat X> with no solve;
* F is traceless and anti-Hermitian, and gauge covariant: F -> Om F Om^dag;
* c_sw = 0 leaves only the hopping force (also checked by differences).
"""

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import dirac, lattice, evenodd, force
from paper_0910_0262_gb300 import synth
from helpers import lattice_shape


def dense_action(U, kappa, csw, phi):
    op = evenodd.SchurOperator(U, kappa, csw)
    n = phi.size
    cols = []
    for j in range(n):
        e = np.zeros(n, dtype=complex)
        e[j] = 1.0
        cols.append(op.Mhat(e.reshape(phi.shape)).reshape(-1))
    Mh = np.stack(cols, axis=1)
    K = Mh.conj().T @ Mh
    x = np.linalg.solve(K, phi.reshape(-1))
    return float(np.vdot(phi.reshape(-1), x).real), op, x.reshape(phi.shape)


@pytest.mark.parametrize("csw", [1.0, 0.0])
def test_force_against_finite_differences(csw):
    dims = (4, 2, 2, 4)
    kappa = 0.12
    U, eta = synth.make_problem(dims, 0.3, 8)
    op0 = evenodd.SchurOperator(U, kappa, csw)
    phi = op0.Mhat_dag(eta[0])
    S0, op, X = dense_action(U, kappa, csw, phi)
    assert abs(S0 - force.action(phi, X)) < 1e-10 * abs(S0)
    G = force.gradient(op, X)
    F = force.lie_force(U, G)
    rng = np.random.default_rng(17)
    h = 1e-5
    for _ in range(3):
        site = tuple(int(rng.integers(0, n)) for n in U.shape[:4])
        mu = int(rng.integers(0, 4))
        D = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
        Up = U.copy()
        Up[site + (mu,)] += h * D
        Um = U.copy()
        Um[site + (mu,)] -= h * D
        fd = (dense_action(Up, kappa, csw, phi)[0] - dense_action(Um, kappa, csw, phi)[0]) / (2 * h)
        an = float(np.real(np.sum(np.conj(G[site + (mu,)]) * D)))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))
        a = int(rng.integers(0, 8))
        Up = U.copy()
        Up[site + (mu,)] = expm(1j * h * synth.T_GEN[a]) @ U[site + (mu,)]
        Um = U.copy()
        Um[site + (mu,)] = expm(-1j * h * synth.T_GEN[a]) @ U[site + (mu,)]
        fd = (dense_action(Up, kappa, csw, phi)[0] - dense_action(Um, kappa, csw, phi)[0]) / (2 * h)
        an = 2.0 * np.imag(np.trace(F[site + (mu,)] @ synth.T_GEN[a]))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


def test_operator_level_difference():
    dims = (4, 2, 2, 4)
    kappa, csw = 0.12, 1.0
    U, eta = synth.make_problem(dims, 0.3, 9)
    op = evenodd.SchurOperator(U, kappa, csw)
    rng = np.random.default_rng(3)
    X = eta[0]
    Y = op.Mhat(X)
    G = force.gradient(op, X)
    h = 1e-6
    for _ in range(3):
        site = tuple(int(rng.integers(0, n)) for n in U.shape[:4])
        mu = int(rng.integers(0, 4))
        D = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
        Up = U.copy()
        Up[site + (mu,)] += h * D
        Um = U.copy()
        Um[site + (mu,)] -= h * D
        dM = (evenodd.SchurOperator(Up, kappa, csw).Mhat(X) - evenodd.SchurOperator(Um, kappa, csw).Mhat(X)) / (2 * h)
        dS = -2.0 * np.vdot(Y.reshape(-1), dM.reshape(-1)).real
        an = float(np.real(np.sum(np.conj(G[site + (mu,)]) * D)))
        assert abs(dS - an) <= 1e-7 * max(1.0, abs(an))


def test_force_algebra_and_gauge_covariance():
    dims = (4, 2, 2, 4)
    kappa, csw = 0.12, 1.0
    U, eta = synth.make_problem(dims, 0.3, 10)
    op = evenodd.SchurOperator(U, kappa, csw)
    X = eta[0]
    F = force.lie_force(U, force.gradient(op, X))
    assert np.max(np.abs(F + dirac.dagger(F))) < 1e-14
    assert np.max(np.abs(np.trace(F, axis1=-2, axis2=-1))) < 1e-13
    rng = np.random.Generator(np.random.PCG64(12))
    Om = synth.random_su3_field(lattice_shape(dims), rng)
    UO = np.empty_like(U)
    for mu in range(4):
        UO[..., mu, :, :] = Om @ U[..., mu, :, :] @ dirac.dagger(lattice.shift(Om, mu, +1))
    Om_e, _ = lattice.split_eo(Om, dims)
    XO = np.einsum('nab,nsb->nsa', Om_e, X)
    opO = evenodd.SchurOperator(UO, kappa, csw)
    FO = force.lie_force(UO, force.gradient(opO, XO))
    expect = Om[..., None, :, :] @ F @ dirac.dagger(Om)[..., None, :, :]
    assert np.max(np.abs(FO - expect)) < 1e-12


def test_multi_rhs_force_is_sum():
    dims = (2, 2, 2, 4)
    U, eta = synth.make_problem(dims, 0.3, 11, nrhs=2)
    op = evenodd.SchurOperator(U, 0.12, 1.0)
    G2 = force.gradient(op, eta)
    G = force.gradient(op, eta[0]) + force.gradient(op, eta[1])
    assert np.max(np.abs(G2 - G)) < 1e-13
