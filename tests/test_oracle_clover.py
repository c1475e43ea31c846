"""Pins of the oracle's clover term.

* unit links and pure-gauge links give F = 0, A = 1;
* a uniform abelian flux (twisted so every xy plaquette equals exp(i q phi))
  gives F_xy = diag(sin phi, -sin phi, 0) exactly, other planes zero;
* random abelian (diagonal) links: F_{mu nu}(x) is one quarter of the sum of sin of
  the plaquette angles of the four plaquettes touching x -- computed here from the
  link phases, not from matrix products, so it pins the set of leaves;
* A is Hermitian, commutes with gamma_5, and A A^-1 = 1 for the inverse used.
"""

import numpy as np

from oracle import dirac, lattice, evenodd
from paper_0910_0262_gb300 import synth
from helpers import lattice_shape


def unit_links(dims):
    return np.broadcast_to(np.eye(3, dtype=complex), lattice_shape(dims) + (4, 3, 3)).copy()


def test_unit_and_pure_gauge_links():
    dims = (4, 2, 2, 6)
    U = unit_links(dims)
    assert np.allclose(dirac.clover_term(U, 0.12, 1.0), np.eye(12), atol=0)
    rng = np.random.Generator(np.random.PCG64(5))
    Om = synth.random_su3_field(lattice_shape(dims), rng)
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[..., mu, :, :] = Om @ dirac.dagger(lattice.shift(Om, mu, +1))
    for mu, nu in dirac.PLANES:
        assert np.max(np.abs(dirac.field_strength(Ug, mu, nu))) < 1e-14
    assert np.max(np.abs(dirac.clover_term(Ug, 0.12, 1.0) - np.eye(12))) < 1e-14


def abelian_flux_links(dims, n_flux, charges):
    """U_y(x, y) = exp(i q phi x); U_x = 1 except U_x(X-1, y) = exp(-i q phi X y); phi = 2 pi n/(X Y)."""
    X, Y, Z, T = dims
    phi = 2 * np.pi * n_flux / (X * Y)
    x, y, z, t = lattice.coords(dims)
    U = unit_links(dims)
    for c, q in enumerate(charges):
        U[..., 1, c, c] = np.exp(1j * q * phi * x)
        ux = np.where(x == X - 1, np.exp(-1j * q * phi * X * y), 1.0)
        U[..., 0, c, c] = ux
    return U, phi


def test_uniform_abelian_flux_closed_form():
    dims = (4, 6, 2, 4)
    U, phi = abelian_flux_links(dims, 1, (1, -1, 0))
    assert np.allclose(np.linalg.det(U), 1.0)
    Fxy = dirac.field_strength(U, 0, 1)
    expect = np.diag([np.sin(phi), -np.sin(phi), 0.0])
    assert np.max(np.abs(Fxy - expect)) < 1e-14
    for mu, nu in dirac.PLANES:
        if (mu, nu) != (0, 1):
            assert np.max(np.abs(dirac.field_strength(U, mu, nu))) < 1e-14
    kappa, csw = 0.12, 1.0
    A = dirac.clover_term(U, kappa, csw)
    A_expect = np.eye(12) - kappa * csw * np.kron(dirac.sigma(0, 1), expect)
    assert np.max(np.abs(A - A_expect)) < 1e-14


def test_random_abelian_field_strength_from_plaquette_angles():
    dims = (4, 2, 6, 4)
    rng = np.random.default_rng(21)
    ph = rng.uniform(-np.pi, np.pi, lattice_shape(dims) + (4, 2))
    phases = np.concatenate([ph, -ph.sum(axis=-1, keepdims=True)], axis=-1)  # det = 1
    U = np.zeros(lattice_shape(dims) + (4, 3, 3), dtype=complex)
    for c in range(3):
        U[..., c, c] = np.exp(1j * phases[..., c])
    for mu, nu in dirac.PLANES:
        a_mu = phases[..., mu, :]
        a_nu = phases[..., nu, :]
        # plaquette angle with lower-left corner z, colour by colour
        theta = a_mu + lattice.shift(a_nu, mu, 1) - lattice.shift(a_mu, nu, 1) - a_nu
        corners = (theta + lattice.shift(theta, mu, -1) + lattice.shift(theta, nu, -1)
                   + lattice.shift(lattice.shift(theta, mu, -1), nu, -1))
        s = (np.sin(theta) + np.sin(lattice.shift(theta, mu, -1)) + np.sin(lattice.shift(theta, nu, -1))
             + np.sin(lattice.shift(lattice.shift(theta, mu, -1), nu, -1))) / 4.0
        s = s - s.sum(axis=-1, keepdims=True) / 3.0
        F = dirac.field_strength(U, mu, nu)
        assert np.max(np.abs(F - np.einsum('...c,cd->...cd', s, np.eye(3)))) < 1e-14
        del corners


def test_clover_hermitian_chiral_blocks_and_inverse():
    dims = (4, 4, 2, 4)
    U, _ = synth.make_problem(dims, 0.2, 1)
    A = dirac.clover_term(U, 0.12, 1.0)
    assert np.max(np.abs(A - dirac.dagger(A))) < 1e-15
    G5 = np.kron(dirac.GAMMA5, np.eye(3))
    assert np.max(np.abs(A @ G5 - G5 @ A)) < 1e-15
    op = evenodd.SchurOperator(U, 0.12, 1.0)
    eye = np.eye(12)
    assert np.max(np.abs(op.A_oo @ op.A_oo_inv - eye)) < 1e-14
    assert np.max(np.abs(op.A_oo_inv @ op.A_oo - eye)) < 1e-14
    # near-unit links: the blocks are positive definite (needed by the GPU Cholesky)
    w = np.linalg.eigvalsh(A)
    assert w.min() > 0.5
