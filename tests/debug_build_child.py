"""Child process of test_gpu_debug_build.py: loads the library named by QCD_LIB (the debug build) and
prints one JSON line with the errors against the oracle and the index-check bits.

Work: every operator of qcd_dslash in FP64, FP32 and FP16 on 13 right-hand sides (batches of 8, 4 and
1) of a lattice whose half volume leaves ragged blocks, a mixed FP32 and a mixed FP16 solve of three
RHS and a plain FP64 solve of one (the single-RHS persistent kernel and the multi-RHS graphs), the
force on the FP64 solution with the clover determinant term, a reconstruction of the odd sites, and
the operators on two t-slabs of the lattice through the library's in-process group (halo packing, the
halo hopping kernels reading the neighbour's send buffers in place).
"""

import json
import os
import sys

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

from oracle import evenodd  # noqa: E402
from paper_0910_0262_gb300 import qcd as Q, slab, synth  # noqa: E402
from gpu_util import to_dev, to_np, rel_l2, rand_eo  # noqa: E402

KAPPA, CSW, TBC = 0.12, 1.0, -1.0
DIMS = (4, 2, 6, 4)


def expected(ref, op, dagger, v):
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


def main():
    U, _ = synth.make_problem(DIMS, 0.2, 3)
    ref = evenodd.SchurOperator(U, KAPPA, CSW, TBC)
    vh = ref.A_ee.shape[0]
    rng = np.random.default_rng(11)
    v = rand_eo(13, vh, rng)
    op = Q.CloverWilson(DIMS, TBC)
    op.load_gauge(to_dev(U), recon12=True)
    op.clover_build(KAPPA, CSW)
    worst = {64: 0.0, 32: 0.0, 16: 0.0}
    ops = [(Q.QCD_OP_DSLASH_EO, 0), (Q.QCD_OP_DSLASH_OE, 1), (Q.QCD_OP_MHAT, 0), (Q.QCD_OP_MHAT, 1),
           (Q.QCD_OP_MDAGM, 0), (Q.QCD_OP_CLOVER, 0), (Q.QCD_OP_CLOVER_INV, 0)]
    for prec in (64, 32, 16):
        for code, dag in ops:
            out = to_np(op.dslash(to_dev(v), code, dagger=bool(dag), precision=prec))
            for r in range(13):
                worst[prec] = max(worst[prec], rel_l2(out[r], expected(ref, code, dag, v[r])))
    solves = {}
    for inner, n in ((32, 3), (16, 3), (64, 1)):
        x, st, ok = op.cg_solve(to_dev(v[:n]), tol=1e-8, inner_prec=inner)
        xn = to_np(x)
        solves[inner] = [max(rel_l2(ref.MdagM(xn[r]), v[r]) for r in range(n)), bool(ok),
                         max(t["true_rel_resid"] for t in st)]
    x, st, ok = op.cg_solve(to_dev(v[:1]), tol=1e-10, inner_prec=64)
    F, _ = op.fermion_force(x, input_is_solution=True, clover_det=True)
    force_finite = bool(torch.isfinite(torch.view_as_real(F)).all().item())
    # x_o = A_oo^-1 (b_o + kappa D_oe x_e) against the oracle's blocks
    b_o = rand_eo(1, vh, rng)
    x_o = to_np(op.reconstruct_odd(x, to_dev(b_o)))
    xe = to_np(x)
    recon_err = rel_l2(x_o[0], ref.site(ref.A_oo_inv, b_o[0] + KAPPA * ref.D_oe(xe[0])))
    # the t-slab operators against the whole-lattice context
    grp = slab.NativeSlabGroup(2)
    sops = []
    for r, (t0, tl) in enumerate([(0, 2), (2, 2)]):
        st = torch.cuda.Stream()
        sop = slab.SlabCloverWilson(DIMS, t0, tl, grp.member(r), TBC, stream=st)
        with torch.cuda.stream(st):
            sop.load_gauge(to_dev(slab.extended_links(U, t0, tl)), recon12=True)
        sop.clover_build(KAPPA, CSW)
        sops.append(sop)

    def job(r):
        s = sops[r]
        a, b = slab.slab_rows(DIMS, s.t_offset, s.t_local)
        with torch.cuda.stream(s.stream):
            y = s.dslash(to_dev(v[:2, a:b]), Q.QCD_OP_MHAT, dagger=False, precision=64)
            s.stream.synchronize()
        return to_np(y)

    parts = grp.run([lambda r=r: job(r) for r in range(2)])
    got = np.concatenate(parts, axis=1)
    slab_err = max(rel_l2(got[r], ref.Mhat(v[r])) for r in range(2))
    for s in sops:
        s.close()
    grp.close()
    viol, is_debug = Q.qcd_debug_violations(op.ctx)
    Q.qcd_selftest_debug_index(op.ctx)
    probe, _ = Q.qcd_debug_violations(op.ctx)
    after, _ = Q.qcd_debug_violations(op.ctx)
    op.close()
    print(json.dumps({"lib": Q.LIB_PATH, "is_debug": is_debug, "violations": viol, "selftest": probe,
                      "after_clear": after, "worst": {str(k): w for k, w in worst.items()},
                      "solves": {str(k): s for k, s in solves.items()}, "force_finite": force_finite,
                      "slab_err": slab_err, "recon_err": recon_err}))


if __name__ == "__main__":
    main()
