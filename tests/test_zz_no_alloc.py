"""qcd_mhat_static: the FP64 Mhat apply that allocates no device memory.

It serves callers that cannot call cudaMalloc -- for example an application
whose memory pool already holds the GPU's free memory, or a latency-sensitive
loop that cannot take the synchronisation cudaMalloc / cudaFree may cause -- by
keeping its work fields in a fixed-size file-scope device array.  These tests
call it through the C ABI and compare it with the existing qcd_dslash(MHAT, FP64)
path and with the FP64 oracle's Mhat / Mhat^dag, on two calls in a row (the
shared array keeps the previous call's contents), for Mhat and Mhat^dag; check
that the caller's current device is the same after the call; and check that a
lattice too large for the array is rejected before any launch.  The file is
named so that pytest collects it last.
"""

import ctypes

import numpy as np
import pytest
import torch

from paper_0910_0262_gb300 import synth
from gpu_util import require_gpu, to_dev, to_np, rel_l2, rand_eo

pytestmark = pytest.mark.gpu

KAPPA, CSW = 0.12, 1.0
TOL_FP64 = 1e-13  # the FP64 parity tolerance of the operator tests


DIMS = (8, 8, 16, 16)


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    from paper_0910_0262_gb300.qcd import CloverWilson
    U, _ = synth.make_problem(DIMS, 0.2, 1)
    c = CloverWilson(DIMS, -1.0)
    c.load_gauge(to_dev(U))
    c.clover_build(KAPPA, CSW)
    yield c
    c.close()


@pytest.fixture(scope="module")
def oracle_op():
    from oracle import evenodd
    U, _ = synth.make_problem(DIMS, 0.2, 1)
    return evenodd.SchurOperator(U, KAPPA, CSW, -1.0)


@pytest.mark.parametrize("dagger", [0, 1])
def test_static_scratch_matches_dslash_two_calls(ctx, oracle_op, dagger):
    from paper_0910_0262_gb300 import qcd as Q
    L = Q.lib()
    rng = np.random.default_rng(7)
    for call in range(2):
        v_np = rand_eo(1, ctx.Vh, rng)
        v = to_dev(v_np)
        out = torch.empty_like(v)
        dev_before = torch.cuda.current_device()
        st = L.qcd_mhat_static(ctx.ctx, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(v.data_ptr()), dagger)
        assert st == Q.QCD_OK, Q.qcd_last_error()
        assert torch.cuda.current_device() == dev_before
        want = ctx.dslash(v, Q.QCD_OP_MHAT, dagger=bool(dagger), precision=64)
        torch.cuda.synchronize()
        err = rel_l2(to_np(out), to_np(want))
        assert err <= TOL_FP64, (call, err)
        ref = oracle_op.Mhat_dag(v_np[0]) if dagger else oracle_op.Mhat(v_np[0])
        err_oracle = rel_l2(to_np(out)[0], ref)
        assert err_oracle <= TOL_FP64, (call, err_oracle)


def test_static_scratch_rejects_large_lattice():
    require_gpu()
    from paper_0910_0262_gb300 import qcd as Q
    big = Q.qcd_create((32, 32, 32, 32), -1.0, None)
    try:
        x = torch.zeros(8, dtype=torch.complex128, device="cuda")
        y = torch.zeros(8, dtype=torch.complex128, device="cuda")
        st = Q.lib().qcd_mhat_static(big, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(x.data_ptr()), 0)
        assert st == 1
        assert "too large" in Q.qcd_last_error()
    finally:
        Q.qcd_destroy(big)
