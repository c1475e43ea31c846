"""GPU operator parity against the FP64 oracle, element by element.

Every op of qcd_dslash (D_eo, D_oe and their adjoints, Mhat, Mhat^dag,
Mhat^dag Mhat, A_ee, A_oo^-1) in FP64, FP32 and FP16, with 18- and 12-real link
storage, on lattices whose half volume leaves a ragged last thread block
(432 and 96 sites per parity: the 32-site blocks of the single-RHS kernels end
ragged at 432, the 64-site blocks of the 2-RHS kernel at 96), on the degenerate
extent-2 lattices where the forward and backward neighbours coincide (8 and 48
sites per parity: a single partial block), with 3 right-hand sides (a batch of
2 plus a batch of 1) and with 13 (8 + 4 + 1).

Tolerances (relative L2 per field): FP64 1e-13 and FP32 1e-6 (the targets of
the method's statement); FP16 with per-site norms is stated, gated at 5e-3.
"""

import numpy as np
import pytest

from oracle import evenodd
from paper_0910_0262_gb300 import synth
from gpu_util import require_gpu, to_dev, to_np, rel_l2, rand_eo

pytestmark = pytest.mark.gpu

KAPPA, CSW = 0.12, 1.0
TOL = {64: 1e-13, 32: 1e-6, 16: 5e-3}
NRHS = 3


@pytest.fixture(scope="module", params=[(6, 6, 4, 6), (4, 2, 6, 4), (2, 2, 2, 2), (2, 4, 2, 6)],
                ids=["6x6x4x6", "4x2x6x4", "2x2x2x2", "2x4x2x6"])
def lattice(request):
    require_gpu()
    from paper_0910_0262_gb300.qcd import CloverWilson
    dims = request.param
    U, _ = synth.make_problem(dims, 0.2, 3)
    ref = evenodd.SchurOperator(U, KAPPA, CSW, -1.0)
    ctxs = {}
    for recon in (18, 12):
        c = CloverWilson(dims, -1.0)
        c.load_gauge(to_dev(U), recon12=recon == 12)
        c.clover_build(KAPPA, CSW)
        ctxs[recon] = c
    vh = ref.A_ee.shape[0]
    rng = np.random.default_rng(5)
    return dims, U, ref, ctxs, rand_eo(NRHS, vh, rng)


def expected(ref, op, dagger, v):
    from paper_0910_0262_gb300 import qcd as Q
    if op == Q.QCD_OP_DSLASH_EO:
        return ref.D_oe_dag(v) if dagger else ref.D_eo(v)
    if op == Q.QCD_OP_DSLASH_OE:
        return ref.D_eo_dag(v) if dagger else ref.D_oe(v)
    if op == Q.QCD_OP_MHAT:
        return ref.Mhat_dag(v) if dagger else ref.Mhat(v)
    if op == Q.QCD_OP_MDAGM:
        return ref.MdagM(v)
    if op == Q.QCD_OP_CLOVER:
        return ref.site(ref.A_ee, v)
    return ref.site(ref.A_oo_inv, v)


OPS = [("DSLASH_EO", 0, 0), ("DSLASH_EO", 0, 1), ("DSLASH_OE", 1, 0), ("DSLASH_OE", 1, 1), ("MHAT", 2, 0),
       ("MHAT", 2, 1), ("MDAGM", 3, 0), ("CLOVER", 4, 0), ("CLOVER_INV", 5, 0)]


@pytest.mark.parametrize("prec,recon", [(64, 18), (32, 18), (32, 12), (16, 12), (16, 18)])
@pytest.mark.parametrize("name,op,dagger", OPS, ids=[f"{o[0]}{'_dag' if o[2] else ''}" for o in OPS])
def test_operator_parity(lattice, prec, recon, name, op, dagger):
    dims, U, ref, ctxs, fields = lattice
    if prec == 64 and recon == 12:
        pytest.skip("FP64 keeps 18 reals")
    out = to_np(ctxs[recon].dslash(to_dev(fields), op, dagger=bool(dagger), precision=prec))
    for r in range(NRHS):
        want = expected(ref, op, dagger, fields[r])
        err = rel_l2(out[r], want)
        assert err <= TOL[prec], f"{name} dag={dagger} p{prec} r{recon} rhs {r}: rel L2 {err:.3e}"


def test_fp64_is_linear_and_gamma5_hermitian_on_gpu(lattice):
    dims, U, ref, ctxs, fields = lattice
    from paper_0910_0262_gb300 import qcd as Q
    c = ctxs[18]
    a, b = fields[0:1], fields[1:2]
    Ma = to_np(c.dslash(to_dev(a), Q.QCD_OP_MHAT))
    Mdb = to_np(c.dslash(to_dev(b), Q.QCD_OP_MHAT, dagger=True))
    lhs = np.vdot(b, Ma)
    rhs = np.vdot(Mdb, a)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


BATCH_OPS = [o for o in OPS if o[0] in ("DSLASH_EO", "MHAT", "MDAGM", "CLOVER_INV")]


@pytest.mark.parametrize("prec,recon", [(64, 18), (32, 12), (32, 18), (16, 12)])
@pytest.mark.parametrize("name,op,dagger", BATCH_OPS, ids=[f"{o[0]}{'_dag' if o[2] else ''}" for o in BATCH_OPS])
def test_operator_parity_rhs_batches(lattice, prec, recon, name, op, dagger):
    """13 right-hand sides: batches of 8, 4 and 1 (the multi-RHS kernel with two RHS per warp, with
    one, and the single-RHS kernel), each RHS against the oracle."""
    dims, U, ref, ctxs, fields = lattice
    rng = np.random.default_rng(17)
    many = rand_eo(13, fields.shape[1], rng)
    out = to_np(ctxs[recon].dslash(to_dev(many), op, dagger=bool(dagger), precision=prec))
    for r in range(13):
        err = rel_l2(out[r], expected(ref, op, dagger, many[r]))
        assert err <= TOL[prec], f"{name} dag={dagger} p{prec} r{recon} rhs {r}: rel L2 {err:.3e}"
