"""GPU parity of the clover determinant term and the full-lattice even-odd solve against the oracle.

* log det A summed per parity (qcd_clover_logdet) against numpy.linalg.slogdet per site;
* the force and the Wirtinger gradient of S_det = -2 log det A_oo (QCD_FORCE_CLOVER_DET with no
  pseudofermion) against the oracle's leaf insertion, element by element, and against central
  differences of the GPU's own log det;
* the pseudofermion force with the flag equals the sum of the two terms;
* source preparation and odd-site reconstruction against the oracle, and a full-lattice solve
  M (x_e, x_o) = (b_e, b_o) whose residual the oracle's unpreconditioned M recomputes;
* on 16^4 (the force workload) the determinant force against the oracle over the whole lattice.
Tolerances: FP64, relative L2 1e-12 (sums of many logarithms and products), 1e-13 per field for the
linear maps.
"""

import numpy as np
import pytest
import torch
from scipy.linalg import expm

from oracle import dirac, lattice, evenodd, force, cloverdet
from paper_0910_0262_gb300 import synth
from gpu_util import require_gpu, to_dev, to_np, rel_l2, rand_eo

pytestmark = pytest.mark.gpu

KAPPA, CSW = 0.12, 1.0


@pytest.fixture(scope="module", params=[(6, 6, 4, 6), (4, 2, 6, 4)], ids=["6x6x4x6", "4x2x6x4"])
def setup(request):
    require_gpu()
    from paper_0910_0262_gb300.qcd import CloverWilson
    dims = request.param
    U, _ = synth.make_problem(dims, 0.3, 41)
    ref = evenodd.SchurOperator(U, KAPPA, CSW, -1.0)
    c = CloverWilson(dims, -1.0)
    c.load_gauge(to_dev(U), recon12=True)
    c.clover_build(KAPPA, CSW)
    yield dims, U, ref, c
    c.close()


def test_logdet_matches_oracle(setup):
    dims, U, ref, c = setup
    le, lo = c.clover_logdet()
    we, wo = cloverdet.logdet(ref)
    assert abs(le - we) <= 1e-12 * abs(we)
    assert abs(lo - wo) <= 1e-12 * abs(wo)


def test_determinant_force_matches_oracle(setup):
    dims, U, ref, c = setup
    G = to_np(c.fermion_force(None, gradient=True, clover_det=True)[0])
    G_ref = cloverdet.gradient(ref)
    assert rel_l2(G, G_ref) <= 1e-12
    F = to_np(c.fermion_force(None, clover_det=True)[0])
    assert rel_l2(F, force.lie_force(U, G_ref)) <= 1e-12


def test_pseudofermion_plus_determinant_is_the_sum(setup):
    dims, U, ref, c = setup
    rng = np.random.default_rng(8)
    X = to_dev(rand_eo(3, ref.A_ee.shape[0], rng))
    both = to_np(c.fermion_force(X, input_is_solution=True, clover_det=True)[0])
    pf = to_np(c.fermion_force(X, input_is_solution=True)[0])
    det = to_np(c.fermion_force(None, clover_det=True)[0])
    assert rel_l2(both, pf + det) <= 1e-13


def test_determinant_force_against_differences_of_gpu_logdet(setup):
    """Central differences (h = 1e-5) of -2 * (odd log det) from rebuilt clover terms, along
    U -> exp(+-i h T_a) U at seeded links, against the GPU force: relative L2 over the sample."""
    from paper_0910_0262_gb300.qcd import CloverWilson
    dims, U, ref, c = setup
    F = to_np(c.fermion_force(None, clover_det=True)[0])
    d = CloverWilson(dims, -1.0)
    h = 1e-5

    def S(Uv):
        d.load_gauge(to_dev(Uv))
        d.clover_build(KAPPA, CSW)
        return -2.0 * d.clover_logdet()[1]

    num = den = 0.0
    for (i, mu) in synth.sample_links(dims, 6, seed=9):
        X, Y, Z, T = dims
        site = (i // (X * Y * Z), (i // (X * Y)) % Z, (i // X) % Y, i % X)
        for a in (0, 3, 7):
            Up, Um = U.copy(), U.copy()
            Up[site + (mu,)] = expm(1j * h * synth.T_GEN[a]) @ U[site + (mu,)]
            Um[site + (mu,)] = expm(-1j * h * synth.T_GEN[a]) @ U[site + (mu,)]
            fd = (S(Up) - S(Um)) / (2 * h)
            an = 2.0 * np.imag(np.trace(F[site + (mu,)] @ synth.T_GEN[a]))
            num += (fd - an) ** 2
            den += an ** 2
    d.close()
    assert den > 0 and np.sqrt(num / den) <= 1e-6


def test_prepare_source_and_reconstruct_match_oracle(setup):
    dims, U, ref, c = setup
    rng = np.random.default_rng(12)
    vh = ref.A_ee.shape[0]
    b_e, b_o, x_e = rand_eo(3, vh, rng), rand_eo(3, vh, rng), rand_eo(3, vh, rng)
    bh = to_np(c.prepare_source(to_dev(b_e), to_dev(b_o)))
    xo = to_np(c.reconstruct_odd(to_dev(x_e), to_dev(b_o)))
    xo0 = to_np(c.reconstruct_odd(to_dev(x_e)))
    for r in range(3):
        assert rel_l2(bh[r], cloverdet.prepare_source(ref, b_e[r], b_o[r])) <= 1e-13
        assert rel_l2(xo[r], cloverdet.reconstruct_odd(ref, x_e[r], b_o[r])) <= 1e-13
        assert rel_l2(xo0[r], cloverdet.reconstruct_odd(ref, x_e[r], np.zeros_like(b_o[r]))) <= 1e-13
    assert np.array_equal(to_np(c.prepare_source(to_dev(b_e))), b_e)


def test_full_lattice_solve_residual(setup):
    """M (x_e, x_o) = (b_e, b_o): Mhat^dag Mhat x_e = Mhat^dag bhat_e on the GPU, x_o reconstructed,
    residual of the whole system recomputed by the oracle's unpreconditioned M."""
    from paper_0910_0262_gb300 import qcd as Q
    dims, U, ref, c = setup
    rng = np.random.default_rng(13)
    vh = ref.A_ee.shape[0]
    b_e, b_o = rand_eo(1, vh, rng), rand_eo(1, vh, rng)
    bh = c.prepare_source(to_dev(b_e), to_dev(b_o))
    rhs = c.dslash(bh, Q.QCD_OP_MHAT, dagger=True)
    x_e, stats, ok = c.cg_solve(rhs, tol=1e-12, inner_prec=64)
    assert ok
    x_o = c.reconstruct_odd(x_e, to_dev(b_o))
    x = lattice.join_eo(to_np(x_e)[0], to_np(x_o)[0], dims)
    b = lattice.join_eo(b_e[0], b_o[0], dims)
    A = dirac.clover_term(U, KAPPA, CSW)
    res = dirac.apply_M(U, A, x, KAPPA, -1.0) - b
    assert np.linalg.norm(res.reshape(-1)) <= 1e-9 * np.linalg.norm(b.reshape(-1))


def test_c2_determinant_force_full_lattice():
    """16^4 links of the force workload (seed 3): the determinant force over all 262144 links."""
    require_gpu()
    from paper_0910_0262_gb300.qcd import CloverWilson
    w = synth.WORKLOADS["c2_16^4_force"]
    U, _ = synth.make_problem(w["dims"], w["eps"], w["seed"], 1)
    ref = evenodd.SchurOperator(U, KAPPA, CSW, -1.0)
    c = CloverWilson(w["dims"], -1.0)
    c.load_gauge(to_dev(U), recon12=True)
    c.clover_build(KAPPA, CSW)
    F = to_np(c.fermion_force(None, clover_det=True)[0])
    assert rel_l2(F, force.lie_force(U, cloverdet.gradient(ref))) <= 1e-12
    le, lo = c.clover_logdet()
    we, wo = cloverdet.logdet(ref)
    assert abs(lo - wo) <= 1e-12 * abs(wo) and abs(le - we) <= 1e-12 * abs(we)
    c.close()
