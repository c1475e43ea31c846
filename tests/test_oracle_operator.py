"""Pins of the oracle's Wilson-clover operator against what the physics fixes.

* gamma algebra of the DeGrand-Rossi basis;
* free field (unit links): plane waves are eigenvectors with the closed-form
  symbol 1 - 2 kappa sum cos p + 2 i kappa sum gamma_mu sin p, antiperiodic in t;
* gamma_5-hermiticity: gamma_5 M gamma_5 equals the explicitly written M^dag, and
  <chi, M psi> = <M^dag chi, psi>;
* gauge covariance under a random SU(3) transformation.
"""

import numpy as np
import pytest

from oracle import dirac, lattice
from paper_0910_0262_gb300 import synth
from helpers import rand_spinor, rel_l2, lattice_shape

KAPPA = 0.12


def test_gamma_algebra():
    g = dirac.GAMMA
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T)
        for nu in range(4):
            anti = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(anti, 2.0 * (mu == nu) * np.eye(4))
    assert np.allclose(dirac.GAMMA5, np.diag([1, 1, -1, -1]))
    for mu, nu in dirac.PLANES:
        s = dirac.sigma(mu, nu)
        assert np.allclose(s, s.conj().T)
        # block diagonal in chirality: the clover term splits into two 6x6 blocks
        assert np.allclose(s[:2, 2:], 0) and np.allclose(s[2:, :2], 0)


@pytest.mark.parametrize("dims", [(4, 6, 2, 8), (6, 4, 4, 4)])
def test_free_field_plane_wave(dims):
    X, Y, Z, T = dims
    U = np.broadcast_to(np.eye(3, dtype=complex), lattice_shape(dims) + (4, 3, 3)).copy()
    A = dirac.clover_term(U, KAPPA, 1.7)
    assert np.allclose(A, np.eye(12))
    x, y, z, t = lattice.coords(dims)
    rng = np.random.default_rng(11)
    for n in [(0, 0, 0, 0), (1, 2, 1, 3), (X - 1, 1, 0, T // 2)]:
        p = [2 * np.pi * n[0] / X, 2 * np.pi * n[1] / Y, 2 * np.pi * n[2] / Z, (2 * n[3] + 1) * np.pi / T]
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        psi = phase[..., None, None] * u
        symbol = (1 - 2 * KAPPA * sum(np.cos(q) for q in p)) * np.eye(4) \
            + 2j * KAPPA * sum(dirac.GAMMA[mu] * np.sin(p[mu]) for mu in range(4))
        expect = phase[..., None, None] * (symbol @ u)
        got = dirac.apply_M(U, A, psi, KAPPA, -1.0)
        assert np.max(np.abs(got - expect)) < 1e-13
        # |eigenvalue|^2 of the symbol: (1 - 2k sum cos)^2 + 4 k^2 sum sin^2
        lam2 = (1 - 2 * KAPPA * sum(np.cos(q) for q in p)) ** 2 + 4 * KAPPA ** 2 * sum(np.sin(q) ** 2 for q in p)
        assert np.allclose(symbol.conj().T @ symbol, lam2 * np.eye(4))


def test_free_field_periodic_time_breaks_with_wrong_momentum():
    """With t_bc = -1 a periodic-in-t plane wave is NOT an eigenvector (the sign is live)."""
    dims = (4, 4, 4, 4)
    U = np.broadcast_to(np.eye(3, dtype=complex), lattice_shape(dims) + (4, 3, 3)).copy()
    A = dirac.clover_term(U, KAPPA, 1.0)
    x, y, z, t = lattice.coords(dims)
    psi = np.exp(1j * 0 * t)[..., None, None] * np.ones((4, 3))
    got = dirac.apply_M(U, A, psi, KAPPA, -1.0)
    symbol = (1 - 2 * KAPPA * 4) * np.ones((4, 3))
    assert np.max(np.abs(got - symbol)) > 0.1
    got_p = dirac.apply_M(U, A, psi, KAPPA, +1.0)
    assert np.max(np.abs(got_p - symbol)) < 1e-13


@pytest.mark.parametrize("dims,seed", [((4, 2, 6, 4), 1), ((2, 4, 4, 6), 5)])
def test_gamma5_hermiticity_and_adjoint(dims, seed):
    U, _ = synth.make_problem(dims, 0.4, seed)
    A = dirac.clover_term(U, KAPPA, 1.0)
    rng = np.random.default_rng(seed)
    psi = rand_spinor(lattice_shape(dims), rng)
    chi = rand_spinor(lattice_shape(dims), rng)
    Mdag_chi = dirac.apply_Mdag(U, A, chi, KAPPA, -1.0)
    g5Mg5 = dirac.gamma5(dirac.apply_M(U, A, dirac.gamma5(chi), KAPPA, -1.0))
    assert rel_l2(g5Mg5, Mdag_chi) < 1e-14
    lhs = np.vdot(chi, dirac.apply_M(U, A, psi, KAPPA, -1.0))
    rhs = np.vdot(Mdag_chi, psi)
    assert abs(lhs - rhs) / abs(lhs) < 1e-14
    # the hopping term alone is gamma5-hermitian too, and the clover term Hermitian
    Dpsi = dirac.hopping(U, psi, -1.0)
    assert abs(np.vdot(chi, Dpsi) - np.vdot(dirac.hopping_dagger(U, chi, -1.0), psi)) / abs(np.vdot(chi, Dpsi)) < 1e-14
    assert np.allclose(A, dirac.dagger(A), atol=1e-15)


def gauge_transform(U, Om):
    """U^Om_mu(x) = Om(x) U_mu(x) Om(x+mu)^dag."""
    out = np.empty_like(U)
    for mu in range(4):
        out[..., mu, :, :] = Om @ U[..., mu, :, :] @ dirac.dagger(lattice.shift(Om, mu, +1))
    return out


@pytest.mark.parametrize("dims", [(4, 2, 6, 4)])
def test_gauge_covariance(dims):
    U, _ = synth.make_problem(dims, 0.4, 3)
    rng = np.random.Generator(np.random.PCG64(99))
    Om = synth.random_su3_field(lattice_shape(dims), rng)
    UO = gauge_transform(U, Om)
    A = dirac.clover_term(U, KAPPA, 1.0)
    AO = dirac.clover_term(UO, KAPPA, 1.0)
    # A[U^Om] = Om A Om^dag (Om acts on colour, identity on spin)
    Om12 = np.einsum('st,...ab->...satb', np.eye(4), Om).reshape(Om.shape[:-2] + (12, 12))
    assert np.max(np.abs(AO - Om12 @ A @ dirac.dagger(Om12))) < 1e-14
    psi = rand_spinor(lattice_shape(dims), np.random.default_rng(4))
    lhs = dirac.apply_M(UO, AO, dirac.colour_mul(Om, psi), KAPPA, -1.0)
    rhs = dirac.colour_mul(Om, dirac.apply_M(U, A, psi, KAPPA, -1.0))
    assert rel_l2(lhs, rhs) < 1e-14


def test_lexicographic_order_and_eo_split():
    dims = (4, 2, 6, 4)
    X, Y, Z, T = dims
    x, y, z, t = lattice.coords(dims)
    idx = (x + X * (y + Y * (z + Z * t))).reshape(-1)
    assert np.array_equal(idx, np.arange(X * Y * Z * T))
    f = idx.reshape(lattice_shape(dims))[..., None, None].astype(complex)
    fe, fo = lattice.split_eo(f, dims)
    assert fe.shape[0] == fo.shape[0] == X * Y * Z * T // 2
    # with X even, the half index of site i is i // 2 on both parities
    assert np.array_equal(fe[:, 0, 0].real.astype(int) // 2, np.arange(fe.shape[0]))
    assert np.array_equal(fo[:, 0, 0].real.astype(int) // 2, np.arange(fo.shape[0]))
    assert np.array_equal(lattice.join_eo(fe, fo, dims), f)
