"""Pins of the oracle's even-odd Schur operator and CG by dense brute force.

The full M is assembled column by column from unit vectors and solved with
numpy.linalg.solve; the even half of M^-1 (b, 0) must equal Mhat^-1 b, the dense
Mhat^dag must be the conjugate transpose of the dense Mhat, and the oracle CG
must reach the dense solution with a true residual <= 1e-8.
"""

import numpy as np
import pytest

from oracle import dirac, lattice, evenodd, cg
from paper_0910_0262_gb300 import synth
from helpers import rel_l2, lattice_shape


def dense(apply, shape):
    n = int(np.prod(shape))
    cols = []
    for j in range(n):
        e = np.zeros(n, dtype=complex)
        e[j] = 1.0
        cols.append(apply(e.reshape(shape)).reshape(-1))
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("dims,eps,seed", [((2, 2, 2, 2), 0.5, 1), ((2, 4, 2, 4), 0.3, 2)])
def test_schur_complement_matches_dense_full_solve(dims, eps, seed):
    kappa, csw = 0.12, 1.0
    U, b = synth.make_problem(dims, eps, seed)
    b = b[0]
    op = evenodd.SchurOperator(U, kappa, csw)
    A = dirac.clover_term(U, kappa, csw)
    full_shape = lattice_shape(dims) + (4, 3)
    M = dense(lambda v: dirac.apply_M(U, A, v, kappa, -1.0), full_shape)
    Mdag = dense(lambda v: dirac.apply_Mdag(U, A, v, kappa, -1.0), full_shape)
    assert np.max(np.abs(Mdag - M.conj().T)) < 1e-14
    rhs = lattice.join_eo(b, np.zeros_like(b), dims).reshape(-1)
    sol = np.linalg.solve(M, rhs).reshape(full_shape)
    sol_e, sol_o = lattice.split_eo(sol, dims)
    Mh = dense(op.Mhat, b.shape)
    Mhd = dense(op.Mhat_dag, b.shape)
    assert np.max(np.abs(Mhd - Mh.conj().T)) < 1e-14
    x_e = np.linalg.solve(Mh, b.reshape(-1)).reshape(b.shape)
    assert rel_l2(x_e, sol_e) < 1e-12
    assert rel_l2(op.odd_solution(x_e), sol_o) < 1e-12


@pytest.mark.parametrize("dims,seed", [((4, 2, 2, 4), 3), ((4, 4, 4, 4), 4)])
def test_cg_reaches_dense_solution(dims, seed):
    kappa, csw = 0.12, 1.0
    U, b = synth.make_problem(dims, 0.2, seed)
    b = b[0]
    op = evenodd.SchurOperator(U, kappa, csw)
    x, iters, res = cg.cg(op.MdagM, b, tol=1e-8)
    assert res <= 1e-8
    assert iters > 5
    true = np.linalg.norm((b - op.MdagM(x)).reshape(-1)) / np.linalg.norm(b.reshape(-1))
    assert true <= 1e-8
    if np.prod(dims) <= 64:
        Mh = dense(op.Mhat, b.shape)
        x_dense = np.linalg.solve(Mh.conj().T @ Mh, b.reshape(-1)).reshape(b.shape)
        cond = np.linalg.cond(Mh.conj().T @ Mh)
        assert rel_l2(x, x_dense) < 10 * cond * 1e-8
