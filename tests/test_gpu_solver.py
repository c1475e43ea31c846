"""CG on Mhat^dag Mhat x = b on the GPU: FP64, mixed FP32 and mixed FP16 (with FP64
reliable updates), several right-hand sides (batches of 1, 2, 4 and 8).  Every solution must have a true
relative residual <= 1e-8 recomputed by the FP64 oracle's operator."""

import numpy as np
import pytest

from oracle import evenodd, cg as ocg
from paper_0910_0262_gb300 import synth
from gpu_util import require_gpu, to_dev, to_np, rel_l2

pytestmark = pytest.mark.gpu

KAPPA, CSW = 0.12, 1.0


@pytest.fixture(scope="module")
def problem():
    require_gpu()
    from paper_0910_0262_gb300.qcd import CloverWilson
    dims = (6, 6, 4, 8)
    U, b = synth.make_problem(dims, 0.2, 11, nrhs=12)
    ref = evenodd.SchurOperator(U, KAPPA, CSW, -1.0)
    c = CloverWilson(dims, -1.0)
    c.load_gauge(to_dev(U), recon12=True)
    c.clover_build(KAPPA, CSW)
    return dims, U, b, ref, c


def true_residual(ref, x, b):
    return np.linalg.norm((b - ref.MdagM(x)).reshape(-1)) / np.linalg.norm(b.reshape(-1))


@pytest.mark.parametrize("inner", [64, 32, 16])
@pytest.mark.parametrize("nrhs", [1, 3, 12])
def test_cg_true_residual(problem, inner, nrhs):
    """nrhs = 3 runs batches of 2 and 1, nrhs = 12 batches of 8 and 4 (the multi-RHS kernels)."""
    dims, U, b, ref, c = problem
    bb = b[:nrhs]
    x, stats, ok = c.cg_solve(to_dev(bb), tol=1e-8, inner_prec=inner, max_iter=5000)
    assert ok
    x = to_np(x)
    xo, it, res = ocg.cg(ref.MdagM, bb[0], tol=1e-10)
    for r in range(nrhs):
        tr = true_residual(ref, x[r], bb[r])
        assert tr <= 1e-8 * (1 + 1e-6), (inner, r, tr)
        assert stats[r]["true_rel_resid"] <= 1e-8
        assert abs(stats[r]["true_rel_resid"] - tr) <= 1e-12
        assert stats[r]["iters"] > 0
        S = float(np.vdot(bb[r], x[r]).real)
        assert abs(stats[r]["b_dot_x"] - S) <= 1e-12 * abs(S)
    assert rel_l2(x[0], xo) < 1e-5


def test_cg_from_initial_guess(problem):
    dims, U, b, ref, c = problem
    x0, _, ok = c.cg_solve(to_dev(b[:1]), tol=1e-10, inner_prec=64)
    assert ok
    x, stats, ok = c.cg_solve(to_dev(b[:1]), x0=x0, tol=1e-8, inner_prec=32)
    assert ok and stats[0]["iters"] == 0
    assert true_residual(ref, to_np(x)[0], b[0]) <= 1e-8


def test_cg_zero_source(problem):
    dims, U, b, ref, c = problem
    z = np.zeros_like(b[:1])
    x, stats, ok = c.cg_solve(to_dev(z), inner_prec=32)
    assert ok and np.all(to_np(x) == 0) and stats[0]["iters"] == 0


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 4, 2, 6)], ids=["2x2x2x2", "2x4x2x6"])
@pytest.mark.parametrize("inner", [64, 32, 16])
def test_cg_on_degenerate_lattices(dims, inner):
    """Extent-2 lattices (forward and backward neighbours coincide; one partial block, so the
    persistent kernel runs a grid of one block): the true residual recomputed by the oracle."""
    require_gpu()
    from paper_0910_0262_gb300.qcd import CloverWilson
    U, b = synth.make_problem(dims, 0.3, 12, nrhs=2)
    ref = evenodd.SchurOperator(U, KAPPA, CSW)
    c = CloverWilson(dims, -1.0)
    c.load_gauge(to_dev(U), recon12=True)
    c.clover_build(KAPPA, CSW)
    for n in (1, 2):
        x, stats, ok = c.cg_solve(to_dev(b[:n]), tol=1e-8, inner_prec=inner, max_iter=5000)
        assert ok
        x = to_np(x)
        for r in range(n):
            assert true_residual(ref, x[r], b[r]) <= 1e-8 * (1 + 1e-6)
    c.close()


def _ctx(dims, U, persistent):
    import os
    from paper_0910_0262_gb300.qcd import CloverWilson
    old = os.environ.get("QCD_CG_PERSISTENT")
    os.environ["QCD_CG_PERSISTENT"] = "1" if persistent else "0"
    try:
        c = CloverWilson(dims, -1.0)
    finally:
        if old is None:
            del os.environ["QCD_CG_PERSISTENT"]
        else:
            os.environ["QCD_CG_PERSISTENT"] = old
    c.load_gauge(to_dev(U), recon12=True)
    c.clover_build(KAPPA, CSW)
    return c


@pytest.mark.parametrize("inner", [32, 16])
def test_persistent_rounds_beyond_the_prediction(problem, inner):
    """A reliable update every 5 iterations: far more rounds (persistent segment + gated update) than
    the first batch enqueues, so the solve takes several looks; it must agree with the graph path
    (one launch per pass) in iterations, reliable updates and the oracle's true residual."""
    dims, U, b, ref, _ = problem
    kw = dict(tol=1e-8, inner_prec=inner, reliable_every=5, reliable_delta=0.1, max_iter=5000)
    res = {}
    for persistent in (True, False):
        c = _ctx(dims, U, persistent)
        x, st, ok = c.cg_solve(to_dev(b[:1]), **kw)
        c.close()
        assert ok
        assert true_residual(ref, to_np(x)[0], b[0]) <= 1e-8 * (1 + 1e-6)
        res[persistent] = st[0]
    assert res[True]["reliable_updates"] >= res[True]["iters"] // 5
    assert abs(res[True]["iters"] - res[False]["iters"]) <= 2
    assert abs(res[True]["reliable_updates"] - res[False]["reliable_updates"]) <= 1


@pytest.mark.parametrize("inner", [32, 16])
def test_persistent_rounds_past_convergence(problem, inner):
    """From an initial guess good to ~1e-5 the mixed solve to 1e-8 needs few reliable updates while
    the first batch enqueues rounds for a solve from zero: the rounds after convergence must do
    nothing (no FP64 hopping launches in the profile beyond the set-up's and the updates that ran)."""
    dims, U, b, ref, c = problem
    x0, _, ok = c.cg_solve(to_dev(b[:1]), tol=1e-5, inner_prec=64)
    assert ok
    c.profile(True)
    x, st, ok = c.cg_solve(to_dev(b[:1]), x0=x0, tol=1e-8, inner_prec=inner, reliable_delta=0.1)
    rows = {r["name"]: r["launches"] for r in c.profile_read()}
    c.profile(False)
    assert ok
    assert true_residual(ref, to_np(x)[0], b[0]) <= 1e-8 * (1 + 1e-6)
    n = st[0]["reliable_updates"]
    assert 1 <= n <= 4
    # the set-up's true residual from x0 plus one M^dag M per reliable update that ran
    assert rows.get("dslash_p64_r18_cloverinv") == 2 * (n + 1)
    assert rows.get("dslash_p64_r18_xpay") == 2 * (n + 1)
    assert rows.get(f"cg_persistent_p{inner}") == n
