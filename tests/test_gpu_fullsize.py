"""GPU checks at the full sizes of the workloads.

8x8x16x16 (eps 0.2, seed 1): the plain FP64 solve and the full-field Mhat against the oracle.
16^4 (kappa 0.12, c_sw 1.0, eps 0.2, seeds 2 and 3):
  * Mhat / Mhat^dag Mhat in FP64 and FP32 element by element against the whole-lattice oracle;
  * mixed FP32 and FP16 solves: true residual <= 1e-8 recomputed by the oracle;
  * the force formula for a seeded field X against the oracle's path-insertion force;
  * the force from the solve against central differences of S (eps = 1e-5, FP64) along the
    8 generators at 64 seeded links: relative L2 <= 1e-6 over the 512 components (the
    differences of S are formed field by field, from the stationary estimate
    2 Re<phi, X> - |Mhat X|^2, so that FP64 rounding of S does not swamp the O(eps) change).
32^3 x 64 (eps 0.15, seed 4, 8 RHS):
  * the FP64 Mhat at sampled even sites against the single-site oracle;
  * Mhat and Mhat^dag in FP32 and FP16, for 1 and 8 RHS, at sampled even sites likewise;
  * one batched mixed-precision solve of all 8 RHS with FP16 inner iterations: every RHS
    reaches a true residual <= 1e-8 (recomputed with the FP64 operator checked above).
"""

import numpy as np
import pytest
import torch
from scipy.linalg import expm

from oracle import evenodd, force as oforce, local
from paper_0910_0262_gb300 import synth
from gpu_util import require_gpu, to_dev, to_np, rel_l2

pytestmark = pytest.mark.gpu

KAPPA, CSW, TBC = synth.KAPPA, synth.CSW, synth.T_BC


def true_residual_oracle(ref, x, b):
    return float(np.linalg.norm((b - ref.MdagM(x)).reshape(-1)) / np.linalg.norm(b.reshape(-1)))


def test_c0_plain_fp64_solve_against_oracle():
    """8x8x16x16 (eps 0.2, seed 1): plain FP64 CG to 1e-8 on the GPU; the true residual recomputed
    by the oracle's operator, the solution against the oracle's own CG solution, and the full-field
    Mhat in FP64 and FP32 element by element."""
    require_gpu()
    from paper_0910_0262_gb300 import qcd as Q
    from paper_0910_0262_gb300.qcd import CloverWilson
    from oracle import cg as ocg
    w = synth.WORKLOADS["c0_8x8x16x16"]
    U, b = synth.make_problem(w["dims"], w["eps"], w["seed"], 1)
    ref = evenodd.SchurOperator(U, KAPPA, CSW, TBC)
    op = CloverWilson(w["dims"], TBC)
    op.load_gauge(to_dev(U))
    op.clover_build(KAPPA, CSW)
    want = ref.Mhat(b[0])
    assert rel_l2(to_np(op.dslash(to_dev(b), Q.QCD_OP_MHAT, precision=64))[0], want) <= 1e-13
    assert rel_l2(to_np(op.dslash(to_dev(b), Q.QCD_OP_MHAT, precision=32))[0], want) <= 1e-6
    x, stats, ok = op.cg_solve(to_dev(b), tol=1e-8, inner_prec=64)
    assert ok
    x = to_np(x)[0]
    assert true_residual_oracle(ref, x, b[0]) <= 1e-8 * (1 + 1e-6)
    xo, iters, res = ocg.cg(ref.MdagM, b[0], tol=1e-8)
    assert abs(stats[0]["iters"] - iters) <= 2
    assert rel_l2(x, xo) <= 1e-6
    op.close()


@pytest.fixture(scope="module")
def c1():
    require_gpu()
    from paper_0910_0262_gb300.qcd import CloverWilson
    w = synth.WORKLOADS["c1_16^4"]
    U, b = synth.make_problem(w["dims"], w["eps"], w["seed"], 1)
    ref = evenodd.SchurOperator(U, KAPPA, CSW, TBC)
    op = CloverWilson(w["dims"], TBC)
    op.load_gauge(to_dev(U), recon12=True)
    op.clover_build(KAPPA, CSW)
    yield U, b, ref, op
    op.close()


def test_c1_operator_full_field(c1):
    from paper_0910_0262_gb300 import qcd as Q
    U, b, ref, op = c1
    want = ref.Mhat(b[0])
    assert rel_l2(to_np(op.dslash(to_dev(b), Q.QCD_OP_MHAT, precision=64))[0], want) <= 1e-13
    assert rel_l2(to_np(op.dslash(to_dev(b), Q.QCD_OP_MHAT, precision=32))[0], want) <= 1e-6
    want2 = ref.Mhat_dag(want)
    assert rel_l2(to_np(op.dslash(to_dev(b), Q.QCD_OP_MDAGM, precision=64))[0], want2) <= 1e-13
    assert rel_l2(to_np(op.dslash(to_dev(b), Q.QCD_OP_MDAGM, precision=32))[0], want2) <= 1e-6


@pytest.mark.parametrize("inner", [32, 16])
def test_c1_mixed_solve_true_residual(c1, inner):
    U, b, ref, op = c1
    x, stats, ok = op.cg_solve(to_dev(b), tol=1e-8, inner_prec=inner, reliable_every=50, reliable_delta=0.1)
    assert ok
    assert stats[0]["true_rel_resid"] <= 1e-8
    assert true_residual_oracle(ref, to_np(x)[0], b[0]) <= 1e-8 * (1 + 1e-6)


@pytest.fixture(scope="module")
def c2():
    require_gpu()
    from paper_0910_0262_gb300.qcd import CloverWilson
    w = synth.WORKLOADS["c2_16^4_force"]
    U, eta = synth.make_problem(w["dims"], w["eps"], w["seed"], 1)
    ref = evenodd.SchurOperator(U, KAPPA, CSW, TBC)
    phi = ref.Mhat_dag(eta[0])[None]
    op = CloverWilson(w["dims"], TBC)
    op.load_gauge(to_dev(U))
    op.clover_build(KAPPA, CSW)
    yield w, U, phi, ref, op
    op.close()


def test_c2_force_formula_against_oracle(c2):
    w, U, phi, ref, op = c2
    rng = np.random.Generator(np.random.PCG64(33))
    X = synth.gaussian_sources(w["dims"], 1, rng)
    G_ref = oforce.gradient(ref, X[0])
    F_ref = oforce.lie_force(U, G_ref)
    G, _ = op.fermion_force(to_dev(X), input_is_solution=True, gradient=True)
    F, _ = op.fermion_force(to_dev(X), input_is_solution=True)
    assert rel_l2(to_np(G), G_ref) <= 1e-12
    assert rel_l2(to_np(F), F_ref) <= 1e-12


def test_c2_force_against_finite_differences(c2):
    from paper_0910_0262_gb300 import qcd as Q
    w, U, phi, ref, op = c2
    dims = w["dims"]
    X_, Y_, Z_, T_ = dims
    kw = dict(tol=1e-12, inner_prec=32, reliable_every=50, reliable_delta=0.1)
    phit = to_dev(phi)
    Ut = to_dev(U)
    op.load_gauge(Ut)
    op.clover_build(KAPPA, CSW)
    F, st = op.fermion_force(phit, **kw)
    assert st[0]["true_rel_resid"] <= 1e-12
    x0, _, ok = op.cg_solve(phit, **kw)
    assert ok
    Fn = to_np(F)
    h = 1e-5
    links = synth.sample_links(dims, 64, seed=3)

    def solve_at(Unew):
        op.load_gauge(Unew)
        op.clover_build(KAPPA, CSW)
        x, _, ok = op.cg_solve(phit, x0=x0, **kw)
        assert ok
        return x, op.dslash(x, Q.QCD_OP_MHAT, precision=64)

    fds, ans = [], []
    for i, mu in links:
        xx, yy, zz, tt = i % X_, (i // X_) % Y_, (i // (X_ * Y_)) % Z_, i // (X_ * Y_ * Z_)
        u0 = U[tt, zz, yy, xx, mu]
        for a in range(8):
            res = []
            for sgn in (+1, -1):
                Up = Ut.clone()
                Up[tt, zz, yy, xx, mu] = torch.from_numpy(expm(sgn * 1j * h * synth.T_GEN[a]) @ u0)
                res.append(solve_at(Up))
            (xp, mp), (xm, mm) = res
            dS = 2.0 * torch.vdot(phit.reshape(-1), (xp - xm).reshape(-1)).real \
                - torch.vdot((mp - mm).reshape(-1), (mp + mm).reshape(-1)).real
            fds.append(dS.item() / (2 * h))
            ans.append(2.0 * float(np.imag(np.trace(Fn[tt, zz, yy, xx, mu] @ synth.T_GEN[a]))))
    fds, ans = np.array(fds), np.array(ans)
    # the force over the 512 sampled (link, generator) components within 1e-6 relative of the
    # central differences; single components, whose O(eps^2) truncation error is comparable
    # to the smallest of them, within 1e-5 of the sample's rms
    assert np.linalg.norm(fds - ans) / np.linalg.norm(ans) <= 1e-6
    assert np.max(np.abs(fds - ans)) <= 1e-5 * np.sqrt(np.mean(ans ** 2))
    op.load_gauge(Ut)
    op.clover_build(KAPPA, CSW)


@pytest.fixture(scope="module")
def c3():
    require_gpu()
    from paper_0910_0262_gb300.qcd import CloverWilson
    w = synth.WORKLOADS["c3_32^3x64"]
    U, b = synth.make_problem(w["dims"], w["eps"], w["seed"], w["nrhs"])
    op = CloverWilson(w["dims"], TBC)
    op.load_gauge(to_dev(U), recon12=True)
    op.clover_build(KAPPA, CSW)
    yield w, U, b, op
    op.close()


def test_c3_fp64_operator_at_sampled_sites(c3):
    from paper_0910_0262_gb300 import qcd as Q
    w, U, b, op = c3
    dims = w["dims"]
    out = to_np(op.dslash(to_dev(b[:1]), Q.QCD_OP_MHAT, precision=64))[0]
    outd = to_np(op.dslash(to_dev(b[:1]), Q.QCD_OP_MHAT, dagger=True, precision=64))[0]
    rng = np.random.default_rng(4)
    Vh = b.shape[1]
    num = den = numd = dend = 0.0
    # include boundary sites in t (antiperiodic sign) and random ones
    hs = list(rng.integers(0, Vh, 12)) + [0, Vh - 1]
    for h in hs:
        i = next(i for i in (2 * int(h), 2 * int(h) + 1) if sum(local.coords(dims, i)) % 2 == 0)
        c = local.coords(dims, i)
        want = local.mhat_site(U, b[0], dims, c, KAPPA, CSW, TBC)
        wantd = local.mhat_site(U, b[0], dims, c, KAPPA, CSW, TBC, dagger_op=True)
        num += np.sum(np.abs(out[int(h)] - want) ** 2)
        den += np.sum(np.abs(want) ** 2)
        numd += np.sum(np.abs(outd[int(h)] - wantd) ** 2)
        dend += np.sum(np.abs(wantd) ** 2)
    assert np.sqrt(num / den) <= 1e-13
    assert np.sqrt(numd / dend) <= 1e-13


@pytest.mark.parametrize("prec,tol", [(32, 1e-6), (16, 5e-3)])
@pytest.mark.parametrize("nrhs", [1, 8])
def test_c3_inner_precision_operator_at_sampled_sites(c3, prec, tol, nrhs):
    """Mhat and Mhat^dag in FP32 / FP16 on the 32^3 x 64 lattice (one thread per (site, RHS)
    kernel, for 1 and for 8 RHS) against the single-site FP64 oracle, RHS 0, 3 and 7."""
    from paper_0910_0262_gb300 import qcd as Q
    w, U, b, op = c3
    dims = w["dims"]
    src = to_dev(b[:nrhs])
    out = to_np(op.dslash(src, Q.QCD_OP_MHAT, precision=prec))
    outd = to_np(op.dslash(src, Q.QCD_OP_MHAT, dagger=True, precision=prec))
    rng = np.random.default_rng(7)
    Vh = b.shape[1]
    hs = list(rng.integers(0, Vh, 6)) + [0, Vh - 1]
    for r in [r for r in (0, 3, 7) if r < nrhs]:
        num = den = numd = dend = 0.0
        for h in hs:
            i = next(i for i in (2 * int(h), 2 * int(h) + 1) if sum(local.coords(dims, i)) % 2 == 0)
            c = local.coords(dims, i)
            want = local.mhat_site(U, b[r], dims, c, KAPPA, CSW, TBC)
            wantd = local.mhat_site(U, b[r], dims, c, KAPPA, CSW, TBC, dagger_op=True)
            num += np.sum(np.abs(out[r, int(h)] - want) ** 2)
            den += np.sum(np.abs(want) ** 2)
            numd += np.sum(np.abs(outd[r, int(h)] - wantd) ** 2)
            dend += np.sum(np.abs(wantd) ** 2)
        assert np.sqrt(num / den) <= tol, (prec, nrhs, r, np.sqrt(num / den))
        assert np.sqrt(numd / dend) <= tol, (prec, nrhs, r, np.sqrt(numd / dend))


def test_c3_batched_fp16_solve(c3):
    from paper_0910_0262_gb300 import qcd as Q
    w, U, b, op = c3
    bt = to_dev(b)
    x, stats, ok = op.cg_solve(bt, tol=1e-8, inner_prec=16, reliable_every=50, reliable_delta=0.1)
    assert ok
    Ax = op.dslash(x, Q.QCD_OP_MDAGM, precision=64)
    for r in range(b.shape[0]):
        tr = (torch.linalg.vector_norm(bt[r] - Ax[r]) / torch.linalg.vector_norm(bt[r])).item()
        assert tr <= 1e-8 * (1 + 1e-6), (r, tr)
        assert stats[r]["true_rel_resid"] <= 1e-8


# 48^3 x 96 (eps 0.15, seed 5, 4 pseudofermions): the largest workload.
#  * the FP64 Mhat at sampled even sites against the single-site oracle;
#  * the summed force of the 4 pseudofermions through the autograd Function with the solution
#    recomputed in backward (mixed FP16 inner solve to 1e-8), checked on a 1% sample of links
#    against the gradient recomputed with a plain FP64 GPU solve to 1e-11.


@pytest.fixture(scope="module")
def c4():
    require_gpu()
    from paper_0910_0262_gb300 import qcd as Q
    from paper_0910_0262_gb300.qcd import CloverWilson
    w = synth.WORKLOADS["c4_48^3x96"]
    U, eta = synth.make_problem(w["dims"], w["eps"], w["seed"], w["nrhs"])
    op = CloverWilson(w["dims"], TBC)
    op.load_gauge(to_dev(U), recon12=True)
    op.clover_build(KAPPA, CSW)
    # pseudofermions phi = Mhat^dag eta (the GPU path's own input; no oracle value depends on it)
    phi = op.dslash(to_dev(eta), Q.QCD_OP_MHAT, dagger=True, precision=64)
    yield w, U, eta, phi, op
    op.close()


def test_c4_fp64_operator_at_sampled_sites(c4):
    from paper_0910_0262_gb300 import qcd as Q
    w, U, eta, phi, op = c4
    dims = w["dims"]
    out = to_np(op.dslash(to_dev(eta[:1]), Q.QCD_OP_MHAT, precision=64))[0]
    rng = np.random.default_rng(5)
    Vh = eta.shape[1]
    num = den = 0.0
    for h in list(rng.integers(0, Vh, 8)) + [0, Vh - 1]:
        i = next(i for i in (2 * int(h), 2 * int(h) + 1) if sum(local.coords(dims, i)) % 2 == 0)
        want = local.mhat_site(U, eta[0], dims, local.coords(dims, i), KAPPA, CSW, TBC)
        num += np.sum(np.abs(out[int(h)] - want) ** 2)
        den += np.sum(np.abs(want) ** 2)
    assert np.sqrt(num / den) <= 1e-13


def test_c4_autograd_force_with_recomputation(c4):
    from paper_0910_0262_gb300.qcd import CloverPseudofermionAction
    w, U, eta, phi, op = c4
    Ut = to_dev(U).requires_grad_(True)
    S = CloverPseudofermionAction.apply(Ut, phi, op, KAPPA, CSW,
                                        dict(tol=1e-8, inner_prec=16, reliable_every=50, reliable_delta=0.1), True)
    S.backward()
    G_mixed = Ut.grad.detach()
    del Ut
    op.load_gauge(to_dev(U))
    op.clover_build(KAPPA, CSW)
    G64, st = op.fermion_force(phi, gradient=True, tol=1e-11, inner_prec=64)
    assert all(s["true_rel_resid"] <= 1e-11 for s in st)
    links = synth.sample_links(w["dims"], int(0.01 * np.prod(w["dims"]) * 4), seed=6)
    X_, Y_, Z_, T_ = w["dims"]
    idx = torch.tensor([[i // (X_ * Y_ * Z_), (i // (X_ * Y_)) % Z_, (i // X_) % Y_, i % X_, mu] for i, mu in links],
                       device=G64.device)
    a = G_mixed[idx[:, 0], idx[:, 1], idx[:, 2], idx[:, 3], idx[:, 4]]
    b = G64[idx[:, 0], idx[:, 1], idx[:, 2], idx[:, 3], idx[:, 4]]
    err = (torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item()
    # a 1e-8 solve leaves the force accurate to ~cond(Mhat^dag Mhat) * 1e-8
    assert err <= 1e-5, err
    assert np.isfinite(S.item()) and S.item() > 0
