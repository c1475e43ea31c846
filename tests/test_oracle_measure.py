"""Pins of the oracle's measurements (Polyakov loop, psi-bar psi).

* Polyakov loop: unit links give 1; constant diagonal time links give the closed form
  (e^{i T a} + e^{i T b} + e^{-i T (a+b)}) / 3; a centre transformation of the t = 0 slice multiplies
  it by exp(2 pi i / 3); a random gauge transformation leaves it unchanged;
* psi-bar psi: for a fixed noise vector the even-odd route equals eta^dag x / (2V) with x from a
  dense solve of the full M; averaged over 400 noise vectors it reaches Re Tr M^-1 / V of the dense
  inverse within five standard errors.
"""

import numpy as np

from oracle import dirac, lattice, evenodd, measure
from paper_0910_0262_gb300 import synth
from helpers import lattice_shape

KAPPA, CSW = 0.12, 1.0


def test_polyakov_unit_and_closed_form():
    dims = (2, 4, 2, 6)
    U = np.broadcast_to(np.eye(3, dtype=complex), lattice_shape(dims) + (4, 3, 3)).copy()
    assert abs(measure.polyakov_loop(U) - 1.0) < 1e-15
    a, b = 0.3, -0.7
    U[..., 3, :, :] = np.diag([np.exp(1j * a), np.exp(1j * b), np.exp(-1j * (a + b))])
    T = dims[3]
    want = (np.exp(1j * T * a) + np.exp(1j * T * b) + np.exp(-1j * T * (a + b))) / 3.0
    assert abs(measure.polyakov_loop(U) - want) < 1e-14


def test_polyakov_centre_and_gauge_transformations():
    dims = (4, 2, 4, 4)
    U, _ = synth.make_problem(dims, 0.4, 81)
    L = measure.polyakov_loop(U)
    assert abs(L) > 1e-3
    Uc = U.copy()
    Uc[0, ..., 3, :, :] *= np.exp(2j * np.pi / 3)
    assert abs(measure.polyakov_loop(Uc) - np.exp(2j * np.pi / 3) * L) < 1e-14
    Om = synth.random_su3_field(lattice_shape(dims), np.random.default_rng(4))
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[..., mu, :, :] = Om @ U[..., mu, :, :] @ dirac.dagger(lattice.shift(Om, mu, +1))
    assert abs(measure.polyakov_loop(Ug) - L) < 1e-13


def _dense_M(U, dims):
    A = dirac.clover_term(U, KAPPA, CSW)
    shape = lattice_shape(dims) + (4, 3)
    n = int(np.prod(shape))
    cols = []
    for j in range(n):
        e = np.zeros(n, dtype=complex)
        e[j] = 1.0
        cols.append(dirac.apply_M(U, A, e.reshape(shape), KAPPA, -1.0).reshape(-1))
    return np.stack(cols, axis=1), shape


def test_pbp_estimator_against_dense_inverse():
    dims = (2, 2, 2, 2)
    U, _ = synth.make_problem(dims, 0.5, 82)
    op = evenodd.SchurOperator(U, KAPPA, CSW)
    M, shape = _dense_M(U, dims)
    V = int(np.prod(dims))
    rng = np.random.default_rng(5)
    vh = V // 2
    ests = []
    for k in range(400):
        ee = rng.standard_normal((vh, 4, 3)) + 1j * rng.standard_normal((vh, 4, 3))
        eo = rng.standard_normal((vh, 4, 3)) + 1j * rng.standard_normal((vh, 4, 3))
        est = measure.pbp(op, ee, eo)
        if k < 2:
            eta = lattice.join_eo(ee, eo, dims).reshape(-1)
            x = np.linalg.solve(M, eta)
            assert abs(est - np.vdot(eta, x).real / (2 * V)) < 1e-10 * abs(est)
        ests.append(est)
    exact = np.trace(np.linalg.inv(M)).real / V
    err = np.std(ests) / np.sqrt(len(ests))
    assert abs(np.mean(ests) - exact) < 5 * err, (np.mean(ests), exact, err)
    assert err < 0.05 * abs(exact)
