"""The time decomposition on the GPU, through the C ABI: slabs of one lattice, each a context of its
own driven by a host thread, exchanging their halos on one GPU through the library's in-process group
(NativeSlabGroup: native callbacks, CUDA events between the slabs' streams) or through device copies
made in Python (LocalSlabGroup).

* a single slab that is the whole lattice (its own neighbour) agrees with the ordinary context's
  operators;
* two, three and four slabs (even and uneven thicknesses) give the oracle's Mhat, Mhat^dag, M^dag M and
  hopping blocks on the whole lattice within the parity tolerances (FP64 1e-13, FP32 1e-6, FP16 5e-3);
* the CG solve on two slabs (FP64, and FP32 inner with FP64 reliable updates) reaches a true residual
  <= 1e-8 recomputed by the oracle on the gathered solution, in about the iterations of one context;
* calls that need an ordinary lattice refuse a slab context, and a failing callback is reported; an
  aborted native group fails its calls at once.
"""

import ctypes

import numpy as np
import pytest
import torch

from paper_0910_0262_gb300 import synth
from gpu_util import require_gpu, to_dev, to_np, rel_l2, rand_eo

pytestmark = pytest.mark.gpu

KAPPA, CSW, TBC = 0.12, 1.0, -1.0
TOL = {64: 1e-13, 32: 1e-6, 16: 5e-3}


def _slabs(dims, U, bounds, recon12=True, kind="python"):
    """The slabs of `bounds`, exchanging through a LocalSlabGroup (kind "python") or the library's
    in-process group (kind "native")."""
    from paper_0910_0262_gb300 import slab
    grp = slab.NativeSlabGroup(len(bounds)) if kind == "native" else slab.LocalSlabGroup(len(bounds))
    ops = []
    for r, (t0, tl) in enumerate(bounds):
        st = torch.cuda.Stream()
        op = slab.SlabCloverWilson(dims, t0, tl, grp.member(r), TBC, stream=st)
        with torch.cuda.stream(st):
            op.load_gauge(to_dev(slab.extended_links(U, t0, tl)), recon12=recon12)
        op.clover_build(KAPPA, CSW)
        ops.append(op)
    return grp, ops


def _apply(grp, ops, dims, v, op_code, dagger, prec, parity_in=0):
    """Apply op_code on every slab to its rows of the global field v [n, V/2, 4, 3]; gather the result."""
    from paper_0910_0262_gb300 import slab

    def job(r):
        op = ops[r]
        a, b = slab.slab_rows(dims, op.t_offset, op.t_local)
        with torch.cuda.stream(op.stream):
            x = v[:, a:b].contiguous()
            y = op.dslash(x, op_code, dagger=dagger, precision=prec)
            op.stream.synchronize()
        return to_np(y)

    parts = grp.run([lambda r=r: job(r) for r in range(len(ops))])
    return np.concatenate(parts, axis=1)


@pytest.fixture(scope="module")
def lattice():
    require_gpu()
    from oracle import evenodd
    dims = (4, 4, 4, 8)
    U, b = synth.make_problem(dims, 0.2, 1, nrhs=2)
    return dims, U, b, evenodd.SchurOperator(U, KAPPA, CSW, TBC)


@pytest.mark.parametrize("kind", ["python", "native"])
def test_whole_lattice_slab_matches_the_ordinary_context(lattice, kind):
    from paper_0910_0262_gb300 import qcd as Q
    from paper_0910_0262_gb300.qcd import CloverWilson
    dims, U, b, ref = lattice
    grp, ops = _slabs(dims, U, [(0, 8)], kind=kind)
    plain = CloverWilson(dims, TBC)
    plain.load_gauge(to_dev(U), recon12=True)
    plain.clover_build(KAPPA, CSW)
    v = to_dev(rand_eo(2, plain.Vh, np.random.default_rng(3)))
    for prec in (64, 32, 16):
        for opc in (Q.QCD_OP_MHAT, Q.QCD_OP_MDAGM, Q.QCD_OP_DSLASH_OE):
            for dag in (False, True):
                got = _apply(grp, ops, dims, v, opc, dag, prec)
                want = to_np(plain.dslash(v, opc, dagger=dag, precision=prec))
                # FP64: the same kernel arithmetic; FP32 / FP16 with two RHS the ordinary context runs
                # its one-thread-per-(site, RHS) kernel, which sums in another order
                tol = {64: 1e-14, 32: 1e-6, 16: 5e-3}[prec]
                assert rel_l2(got, want) <= tol, (kind, prec, opc, dag, rel_l2(got, want))
    plain.close()
    _close(grp, ops)


def _close(grp, ops):
    for op in ops:
        op.close()
    if hasattr(grp, "close"):
        grp.close()


@pytest.mark.parametrize("kind", ["python", "native"])
@pytest.mark.parametrize("bounds", [[(0, 4), (4, 4)], [(0, 2), (2, 6)], [(0, 2), (2, 2), (4, 4)],
                                    [(0, 2), (2, 2), (4, 2), (6, 2)]])
def test_split_lattice_matches_the_oracle(lattice, bounds, kind):
    from paper_0910_0262_gb300 import qcd as Q
    dims, U, b, ref = lattice
    grp, ops = _slabs(dims, U, bounds, kind=kind)
    rng = np.random.default_rng(11)
    ve = rand_eo(1, b.shape[1], rng)
    v = to_dev(ve)
    want = {"mhat": ref.Mhat(ve[0]), "mhat_dag": ref.Mhat_dag(ve[0]), "mdagm": ref.MdagM(ve[0]),
            "doe": ref.D_oe(ve[0])}
    for prec in (64, 32, 16):
        got = {"mhat": _apply(grp, ops, dims, v, Q.QCD_OP_MHAT, False, prec)[0],
               "mhat_dag": _apply(grp, ops, dims, v, Q.QCD_OP_MHAT, True, prec)[0],
               "mdagm": _apply(grp, ops, dims, v, Q.QCD_OP_MDAGM, False, prec)[0],
               "doe": _apply(grp, ops, dims, v, Q.QCD_OP_DSLASH_OE, False, prec)[0]}
        for k in want:
            err = rel_l2(got[k], want[k])
            assert err <= TOL[prec], (bounds, kind, prec, k, err)
    _close(grp, ops)


@pytest.mark.parametrize("kind", ["python", "native"])
@pytest.mark.parametrize("inner", [64, 32])
def test_split_lattice_cg_solve(lattice, inner, kind):
    from paper_0910_0262_gb300 import slab
    from paper_0910_0262_gb300.qcd import CloverWilson
    dims, U, b, ref = lattice
    bounds = [(0, 4), (4, 4)]
    grp, ops = _slabs(dims, U, bounds, kind=kind)
    bd = to_dev(b)
    kw = dict(tol=1e-8, inner_prec=inner, reliable_every=50, reliable_delta=0.1, max_iter=2000)

    def job(r):
        op = ops[r]
        a, c = slab.slab_rows(dims, op.t_offset, op.t_local)
        with torch.cuda.stream(op.stream):
            x, st, ok = op.cg_solve(bd[:, a:c].contiguous(), **kw)
            op.stream.synchronize()
        return to_np(x), st, ok

    res = grp.run([lambda r=r: job(r) for r in range(len(ops))])
    x = np.concatenate([r[0] for r in res], axis=1)
    for r in res:
        assert r[2]
    for k in range(b.shape[0]):
        true_res = np.linalg.norm((b[k] - ref.MdagM(x[k])).reshape(-1)) / np.linalg.norm(b[k].reshape(-1))
        assert true_res <= 1e-8 * (1 + 1e-6), (k, true_res)
    # every slab reports the same whole-lattice statistics
    assert res[0][1] == [dict(s, seconds=res[0][1][i]["seconds"]) for i, s in enumerate(res[1][1])]
    plain = CloverWilson(dims, TBC)
    plain.load_gauge(to_dev(U), recon12=True)
    plain.clover_build(KAPPA, CSW)
    _, st1, ok = plain.cg_solve(bd, **kw)
    assert ok
    for k in range(b.shape[0]):
        assert abs(res[0][1][k]["iters"] - st1[k]["iters"]) <= 2
    plain.close()
    _close(grp, ops)


def test_native_group_abort_fails_the_calls(lattice):
    """A native group released by qcd_local_group_abort (a rank that will not come) fails every call
    with QCD_ERR_COMM at once, without waiting at its barrier; joining twice is refused."""
    from paper_0910_0262_gb300 import qcd as Q
    dims, U, b, ref = lattice
    grp, ops = _slabs(dims, U, [(0, 4), (4, 4)], kind="native")
    with pytest.raises(Q.QCDError) as e:
        Q.qcd_local_group_join(grp.handle, 0, ops[0].ctx)
    assert e.value.status == 4
    Q.qcd_local_group_abort(grp.handle)
    v = torch.zeros((1, ops[0].Vh, 4, 3), dtype=torch.complex128, device="cuda")
    for op in ops:
        with pytest.raises(Q.QCDError) as e:
            op.dslash(v, Q.QCD_OP_DSLASH_OE, precision=64)
        assert e.value.status == 9
    _close(grp, ops)


def test_slab_refusals_and_failed_callback(lattice):
    from paper_0910_0262_gb300 import qcd as Q
    from paper_0910_0262_gb300 import slab
    dims, U, b, ref = lattice
    grp, ops = _slabs(dims, U, [(0, 4), (4, 4)])
    op = ops[0]
    L = Q.lib()
    v = torch.zeros((1, op.Vh, 4, 3), dtype=torch.complex128, device="cuda")
    out = torch.empty_like(v)
    assert L.qcd_dslash(op.ctx, Q._ptr(out), Q._ptr(v), Q.QCD_OP_MHAT, 0, 64, 1) == 4  # QCD_ERR_STATE
    assert "t-slab" in Q.qcd_last_error()
    assert L.qcd_fermion_force(op.ctx, Q._ptr(out), Q._ptr(v), 1, 1, None, None) == 4
    assert L.qcd_mhat_static(op.ctx, Q._ptr(out), Q._ptr(v), 0) == 4

    class Broken:
        def exchange(self, *a):
            raise RuntimeError("link down")

        def allreduce(self, v):
            pass

    op.comm = Broken()
    with pytest.raises(Q.QCDError) as e:
        op.dslash(v, Q.QCD_OP_DSLASH_OE, precision=64)
    assert e.value.status == 9
    with pytest.raises(Q.QCDError):
        Q.qcd_create_slab(dims, 1, 4)      # odd offset
    with pytest.raises(Q.QCDError):
        Q.qcd_create_slab(dims, 4, 6)      # past the end of the lattice
    for o in ops:
        o.close()
