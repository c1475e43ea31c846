"""Pins of the oracle's clover determinant term and full-lattice even-odd solve.

* unit links: A = 1, so log det A = 0 and the force vanishes;
* small c_sw: -2 log det A_oo = 4 (kappa c_sw)^2 sum_{x odd} sum_{mu<nu} tr F_{mu nu}(x)^2 to
  second order (tr sigma_{mu nu} = 0 and tr sigma_p sigma_q = 4 delta_pq for the six planes), from
  the oracle's field strength, not its determinant;
* gauge invariance of log det A, gauge covariance of its force;
* the Wirtinger gradient and the Lie-algebra force against central differences of S_det;
* source preparation and odd-site reconstruction against a dense solve of the full M with a
  source on both parities.
"""

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import dirac, lattice, evenodd, force, cloverdet
from paper_0910_0262_gb300 import synth
from helpers import rel_l2, lattice_shape

KAPPA = 0.12


def test_unit_links_give_zero_logdet_and_force():
    dims = (4, 2, 2, 4)
    U = np.broadcast_to(np.eye(3, dtype=complex), lattice_shape(dims) + (4, 3, 3)).copy()
    op = evenodd.SchurOperator(U, KAPPA, 1.0)
    le, lo = cloverdet.logdet(op)
    assert abs(le) < 1e-13 and abs(lo) < 1e-13
    assert np.max(np.abs(cloverdet.gradient(op))) < 1e-14


def test_small_csw_second_order_closed_form():
    dims = (4, 6, 4, 4)  # no extent 2: with one, the even and odd sums of tr F^2 nearly coincide
    U, _ = synth.make_problem(dims, 0.4, 21)
    csw = 1e-3
    op = evenodd.SchurOperator(U, KAPPA, csw)
    odd = lattice.parity(dims) == 1
    trF2 = 0.0
    for mu, nu in dirac.PLANES:
        F = dirac.field_strength(U, mu, nu)
        trF2 += float(np.sum(np.trace(F @ F, axis1=-2, axis2=-1).real[odd]))
    want = 4.0 * (KAPPA * csw) ** 2 * trF2
    got = cloverdet.action(op)
    assert want > 0.0
    assert abs(got - want) <= 1e-4 * want  # third-order terms: about 1e-6 relative here


def test_logdet_gauge_invariance_and_force_covariance():
    dims = (4, 2, 4, 2)
    U, _ = synth.make_problem(dims, 0.4, 22)
    op = evenodd.SchurOperator(U, KAPPA, 1.0)
    rng = np.random.default_rng(5)
    Om = synth.random_su3_field(lattice_shape(dims), rng)
    Ug = np.empty_like(U)
    for mu in range(4):
        Om_next = lattice.shift(Om, mu, +1)
        Ug[..., mu, :, :] = Om @ U[..., mu, :, :] @ dirac.dagger(Om_next)
    opg = evenodd.SchurOperator(Ug, KAPPA, 1.0)
    le, lo = cloverdet.logdet(op)
    leg, log = cloverdet.logdet(opg)
    assert abs(le - leg) <= 1e-12 * abs(le) and abs(lo - log) <= 1e-12 * abs(lo)
    F = force.lie_force(U, cloverdet.gradient(op))
    Fg = force.lie_force(Ug, cloverdet.gradient(opg))
    want = Om[..., None, :, :] @ F @ dirac.dagger(Om)[..., None, :, :]
    assert rel_l2(Fg, want) < 1e-12
    assert np.max(np.abs(F + dirac.dagger(F))) < 1e-14
    assert np.max(np.abs(np.trace(F, axis1=-2, axis2=-1))) < 1e-14


def test_force_against_finite_differences():
    dims = (4, 2, 2, 4)
    U, _ = synth.make_problem(dims, 0.3, 23)
    csw = 1.0
    op = evenodd.SchurOperator(U, KAPPA, csw)
    G = cloverdet.gradient(op)
    F = force.lie_force(U, G)
    assert np.max(np.abs(F)) > 1e-4

    def S(Uv):
        return cloverdet.action(evenodd.SchurOperator(Uv, KAPPA, csw))

    rng = np.random.default_rng(31)
    h = 1e-5
    for _ in range(4):
        site = tuple(int(rng.integers(0, n)) for n in U.shape[:4])
        mu = int(rng.integers(0, 4))
        D = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
        Up, Um = U.copy(), U.copy()
        Up[site + (mu,)] += h * D
        Um[site + (mu,)] -= h * D
        fd = (S(Up) - S(Um)) / (2 * h)
        an = float(np.real(np.sum(np.conj(G[site + (mu,)]) * D)))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)
        a = int(rng.integers(0, 8))
        Up, Um = U.copy(), U.copy()
        Up[site + (mu,)] = expm(1j * h * synth.T_GEN[a]) @ U[site + (mu,)]
        Um[site + (mu,)] = expm(-1j * h * synth.T_GEN[a]) @ U[site + (mu,)]
        fd = (S(Up) - S(Um)) / (2 * h)
        an = 2.0 * np.imag(np.trace(F[site + (mu,)] @ synth.T_GEN[a]))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


@pytest.mark.parametrize("dims,seed", [((2, 2, 2, 2), 24), ((2, 4, 2, 2), 25)])
def test_full_solve_with_both_parities_matches_dense(dims, seed):
    U, b = synth.make_problem(dims, 0.4, seed, nrhs=2)
    b_e, b_o = b[0], b[1]
    op = evenodd.SchurOperator(U, KAPPA, 1.0)
    A = dirac.clover_term(U, KAPPA, 1.0)
    full_shape = lattice_shape(dims) + (4, 3)
    n = int(np.prod(full_shape))
    cols = []
    for j in range(n):
        e = np.zeros(n, dtype=complex)
        e[j] = 1.0
        cols.append(dirac.apply_M(U, A, e.reshape(full_shape), KAPPA, -1.0).reshape(-1))
    M = np.stack(cols, axis=1)
    sol = np.linalg.solve(M, lattice.join_eo(b_e, b_o, dims).reshape(-1)).reshape(full_shape)
    sol_e, sol_o = lattice.split_eo(sol, dims)
    m = b_e.size
    cols = []
    for j in range(m):
        e = np.zeros(m, dtype=complex)
        e[j] = 1.0
        cols.append(op.Mhat(e.reshape(b_e.shape)).reshape(-1))
    Mh = np.stack(cols, axis=1)
    x_e = np.linalg.solve(Mh, cloverdet.prepare_source(op, b_e, b_o).reshape(-1)).reshape(b_e.shape)
    assert rel_l2(x_e, sol_e) < 1e-12
    assert rel_l2(cloverdet.reconstruct_odd(op, x_e, b_o), sol_o) < 1e-12
