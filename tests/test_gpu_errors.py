"""Error paths of the C ABI on the GPU.  No test faults, traps or hangs the GPU: every
failure is produced by arguments or inputs that the library checks itself."""

import ctypes

import numpy as np
import pytest
import torch

from paper_0910_0262_gb300 import synth
from gpu_util import require_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    require_gpu()
    from paper_0910_0262_gb300 import qcd
    return qcd


def test_state_errors(Q):
    c = Q.CloverWilson((4, 4, 4, 4))
    x = torch.zeros((1, 128, 4, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(Q.QCDError) as e:
        c.dslash(x, Q.QCD_OP_DSLASH_EO)
    assert e.value.status == 4
    with pytest.raises(Q.QCDError) as e:
        c.clover_build(0.12, 1.0)
    assert e.value.status == 4
    U, _ = synth.make_problem((4, 4, 4, 4), 0.2, 1)
    c.load_gauge(to_dev(U))
    c.dslash(x, Q.QCD_OP_DSLASH_EO)  # hopping alone needs no clover
    with pytest.raises(Q.QCDError) as e:
        c.dslash(x, Q.QCD_OP_MHAT)
    assert e.value.status == 4
    with pytest.raises(Q.QCDError) as e:
        c.cg_solve(x)
    assert e.value.status == 4


def test_argument_errors(Q):
    c = Q.CloverWilson((4, 4, 4, 4))
    U, _ = synth.make_problem((4, 4, 4, 4), 0.2, 1)
    c.load_gauge(to_dev(U))
    c.clover_build(0.12, 1.0)
    x = torch.zeros((1, 128, 4, 3), dtype=torch.complex128, device="cuda")
    L = Q.lib()
    p = ctypes.c_void_p(x.data_ptr())
    assert L.qcd_dslash(c.ctx, p, p, 2, 0, 64, 1) == 1          # in == out
    assert L.qcd_dslash(c.ctx, None, p, 2, 0, 64, 1) == 1       # null
    y = torch.zeros_like(x)
    q = ctypes.c_void_p(y.data_ptr())
    assert L.qcd_dslash(c.ctx, q, p, 99, 0, 64, 1) == 1         # op
    assert L.qcd_dslash(c.ctx, q, p, 2, 0, 24, 1) == 1          # precision
    assert L.qcd_dslash(c.ctx, q, p, 2, 0, 64, 0) == 1          # nrhs
    prm = Q.solver_params(tol=-1.0)
    assert L.qcd_cg_solve(c.ctx, q, p, 1, ctypes.byref(prm), None) == 1
    assert L.qcd_load_gauge(c.ctx, p, 1, 0x10) == 1             # flags


def test_not_positive_definite(Q):
    c = Q.CloverWilson((4, 4, 4, 4))
    U, _ = synth.make_problem((4, 4, 4, 4), 1.5, 3)
    c.load_gauge(to_dev(U))
    with pytest.raises(Q.QCDError) as e:
        c.clover_build(1.0, 40.0)
    assert e.value.status == 5


def test_not_converged_writes_best_x(Q):
    c = Q.CloverWilson((4, 4, 4, 4))
    U, b = synth.make_problem((4, 4, 4, 4), 0.2, 3)
    c.load_gauge(to_dev(U))
    c.clover_build(0.12, 1.0)
    x, stats, ok = c.cg_solve(to_dev(b), max_iter=3, inner_prec=32)
    assert not ok
    assert 0 < stats[0]["true_rel_resid"] < 1.0
    assert torch.count_nonzero(x) > 0


def test_nan_inputs(Q):
    c = Q.CloverWilson((4, 4, 4, 4))
    U, b = synth.make_problem((4, 4, 4, 4), 0.2, 3)
    Ubad = U.copy()
    Ubad[1, 2, 3, 0, 2, 1, 1] = np.nan
    with pytest.raises(Q.QCDError) as e:
        c.load_gauge(to_dev(Ubad))
    assert e.value.status == 7
    c.load_gauge(to_dev(U))
    c.clover_build(0.12, 1.0)
    bb = b.copy()
    bb[0, 5, 1, 2] = np.inf
    with pytest.raises(Q.QCDError) as e:
        c.cg_solve(to_dev(bb))
    assert e.value.status == 7
    # the context stays usable
    x, stats, ok = c.cg_solve(to_dev(b))
    assert ok


def test_host_gauge_pointer_matches_device(Q):
    dims = (4, 2, 2, 4)
    U, b = synth.make_problem(dims, 0.2, 4)
    c1 = Q.CloverWilson(dims)
    c1.load_gauge(to_dev(U))
    c2 = Q.CloverWilson(dims)
    c2.load_gauge(torch.from_numpy(U.copy()))
    xb = to_dev(b)
    assert torch.equal(c1.dslash(xb, Q.QCD_OP_DSLASH_OE), c2.dslash(xb, Q.QCD_OP_DSLASH_OE))


def test_barrier_wait_runs_out_and_context_survives(Q):
    """A grid-barrier wait with a block that never arrives gives up and reports QCD_ERR_TIMEOUT."""
    c = Q.CloverWilson((4, 4, 4, 4))
    assert Q.qcd_selftest_barrier_timeout(c.ctx) == 8
    assert "gave up" in Q.qcd_last_error()
    U, b = synth.make_problem((4, 4, 4, 4), 0.2, 3)
    c.load_gauge(to_dev(U))
    c.clover_build(0.12, 1.0)
    x, stats, ok = c.cg_solve(to_dev(b))
    assert ok and stats[0]["true_rel_resid"] <= 1e-8


def test_md_and_measurement_argument_and_state_errors(Q):
    """The determinant, R-algorithm and measurement entry points check their state and arguments."""
    dims = (4, 4, 4, 4)
    c = Q.CloverWilson(dims)
    L = Q.lib()
    out2 = (ctypes.c_double * 2)()
    assert L.qcd_clover_logdet(c.ctx, out2) == 4                 # no clover
    assert L.qcd_polyakov(c.ctx, out2) == 4                      # no links
    d = ctypes.c_double()
    assert L.qcd_plaquette(c.ctx, ctypes.byref(d)) == 4
    U, eta = synth.make_problem(dims, 0.2, 2, nrhs=9)
    Ut = to_dev(U)
    P = torch.zeros_like(Ut)
    pu, pp = ctypes.c_void_p(Ut.data_ptr()), ctypes.c_void_p(P.data_ptr())
    e = to_dev(eta)
    pe = ctypes.c_void_p(e.data_ptr())
    prm = Q.solver_params()
    assert L.qcd_r_step(c.ctx, pu, pp, pe, 1, ctypes.c_double(0.01), ctypes.c_double(5.6), 0,
                        ctypes.byref(prm), None) == 4            # no clover term yet
    c.load_gauge(Ut)
    c.clover_build(0.12, 1.0)
    assert L.qcd_update_links(c.ctx, pu, pu, ctypes.c_double(0.1)) == 1          # U and P overlap
    assert L.qcd_gauge_force(c.ctx, pp, ctypes.c_double(5.6), 0x40) == 1         # flags
    assert L.qcd_r_step(c.ctx, pu, pp, pe, 1, ctypes.c_double(0.01), ctypes.c_double(5.6), 2,
                        ctypes.byref(prm), None) == 1            # unknown flag
    vals = (ctypes.c_double * 9)()
    assert L.qcd_pbp(c.ctx, pe, pe, 9, vals, ctypes.byref(prm), None) == 1       # nrhs > 8
    assert L.qcd_fermion_force(c.ctx, pp, None, 0, 0, None, None) == 1           # nrhs 0 without the flag
    x = torch.zeros((1, 128, 4, 3), dtype=torch.complex128, device="cuda")
    px = ctypes.c_void_p(x.data_ptr())
    assert L.qcd_reconstruct_odd(c.ctx, px, px, None, 1) == 1                    # output overlaps input
    # the context stays usable
    assert abs(c.plaquette() - 1.0) < 0.5 and np.isfinite(c.clover_logdet()[1])
