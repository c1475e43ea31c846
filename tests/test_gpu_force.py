"""GPU fermion force and the autograd Function against the FP64 oracle.

* the Wirtinger gradient G and the Lie-algebra force F from given X, element by
  element against the oracle's path-insertion force (relative L2 1e-12);
* the force with the solve inside (phi given), summed over 2 RHS;
* CloverPseudofermionAction: S and dS/dU against the oracle, and against
  central differences of the GPU action along random complex directions.
"""

import numpy as np
import pytest
import torch

from oracle import evenodd, force as oforce
from paper_0910_0262_gb300 import synth
from gpu_util import require_gpu, to_dev, to_np, rel_l2

pytestmark = pytest.mark.gpu

KAPPA, CSW = 0.12, 1.0


@pytest.fixture(scope="module", params=[(4, 2, 6, 4), (6, 4, 4, 6)], ids=["4x2x6x4", "6x4x4x6"])
def setup(request):
    require_gpu()
    from paper_0910_0262_gb300.qcd import CloverWilson
    dims = request.param
    U, eta = synth.make_problem(dims, 0.25, 21, nrhs=2)
    ref = evenodd.SchurOperator(U, KAPPA, CSW, -1.0)
    c = CloverWilson(dims, -1.0)
    c.load_gauge(to_dev(U))
    c.clover_build(KAPPA, CSW)
    return dims, U, eta, ref, c


def test_gradient_and_force_from_solution(setup):
    dims, U, X, ref, c = setup
    G_ref = oforce.gradient(ref, X)
    F_ref = oforce.lie_force(U, G_ref)
    G, _ = c.fermion_force(to_dev(X), input_is_solution=True, gradient=True)
    F, _ = c.fermion_force(to_dev(X), input_is_solution=True, gradient=False)
    assert rel_l2(to_np(G), G_ref) <= 1e-12
    assert rel_l2(to_np(F), F_ref) <= 1e-12
    Fn = to_np(F)
    assert np.max(np.abs(Fn + np.conj(np.swapaxes(Fn, -1, -2)))) < 1e-13
    assert np.max(np.abs(np.trace(Fn, axis1=-2, axis2=-1))) < 1e-12


def test_force_with_solve(setup):
    dims, U, eta, ref, c = setup
    phi = np.stack([ref.Mhat_dag(e) for e in eta])
    from oracle import cg as ocg
    X = np.stack([ocg.cg(ref.MdagM, p, tol=1e-13)[0] for p in phi])
    F_ref = oforce.lie_force(U, oforce.gradient(ref, X))
    F, stats = c.fermion_force(to_dev(phi), tol=1e-12, inner_prec=32)
    assert all(s["true_rel_resid"] <= 1e-12 for s in stats)
    assert rel_l2(to_np(F), F_ref) <= 1e-8


def test_autograd_action(setup):
    from paper_0910_0262_gb300.qcd import CloverPseudofermionAction
    dims, U, eta, ref, c = setup
    phi = np.stack([ref.Mhat_dag(e) for e in eta[:1]])
    Ut = to_dev(U).requires_grad_(True)
    pt = to_dev(phi)
    kw = dict(tol=1e-12, inner_prec=32)
    S = CloverPseudofermionAction.apply(Ut, pt, c, KAPPA, CSW, kw, False)
    S.backward()
    from oracle import cg as ocg
    X = ocg.cg(ref.MdagM, phi[0], tol=1e-13)[0]
    S_ref = oforce.action(phi[0], X)
    assert abs(S.item() - S_ref) <= 1e-10 * abs(S_ref)
    G_ref = oforce.gradient(ref, X)
    assert rel_l2(to_np(Ut.grad), G_ref) <= 1e-8
    # central differences of the GPU action along random complex directions of single links
    rng = np.random.default_rng(2)
    h = 1e-5
    G = to_np(Ut.grad)
    for _ in range(2):
        site = tuple(int(rng.integers(0, n)) for n in U.shape[:4])
        mu = int(rng.integers(0, 4))
        D = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
        vals = []
        for sgn in (+1, -1):
            Up = U.copy()
            Up[site + (mu,)] += sgn * h * D
            vals.append(CloverPseudofermionAction.apply(to_dev(Up), pt, c, KAPPA, CSW, kw, False).item())
        fd = (vals[0] - vals[1]) / (2 * h)
        an = float(np.real(np.sum(np.conj(G[site + (mu,)]) * D)))
        assert abs(fd - an) <= 1e-5 * max(1.0, abs(an))


def test_autograd_recompute_matches(setup):
    from paper_0910_0262_gb300.qcd import CloverPseudofermionAction
    dims, U, eta, ref, c = setup
    phi = to_dev(np.stack([ref.Mhat_dag(e) for e in eta]))
    grads = []
    for recompute in (False, True):
        Ut = to_dev(U).requires_grad_(True)
        S = CloverPseudofermionAction.apply(Ut, phi, c, KAPPA, CSW, dict(tol=1e-12, inner_prec=16), recompute)
        S.backward()
        grads.append(to_np(Ut.grad))
    assert rel_l2(grads[1], grads[0]) <= 1e-9
