"""Per-kernel profiling of the solver (qcd_profile / qcd_profile_read).

The mixed single-RHS solve runs its iterations in the persistent kernel and enqueues its reliable
updates as CUDA graphs ahead of knowing whether each is due (gated on the device).  The profile must
count what ran: one persistent launch per reliable-update interval, four FP64 hopping launches per
reliable update that ran (not the gated rounds that returned at once), and the same counts in every
profiling session, including sessions that reuse graphs recorded in an earlier one.
"""

import numpy as np
import pytest

from paper_0910_0262_gb300 import synth
from gpu_util import require_gpu, to_dev

pytestmark = pytest.mark.gpu


def _session(op, b, **kw):
    op.profile(True)
    _, st, ok = op.cg_solve(b, **kw)
    rows = {r["name"]: r["launches"] for r in op.profile_read() if r["name"] != "launches_total"}
    op.profile(False)
    assert ok
    return rows, st[0]


@pytest.mark.parametrize("inner", [32, 16])
def test_profile_counts_match_the_work_in_every_session(inner):
    require_gpu()
    from paper_0910_0262_gb300.qcd import CloverWilson
    dims = (8, 8, 8, 8)
    U, b = synth.make_problem(dims, 0.2, 71, 1)
    op = CloverWilson(dims, -1.0)
    op.load_gauge(to_dev(U), recon12=True)
    op.clover_build(0.12, 1.0)
    kw = dict(tol=1e-8, inner_prec=inner, reliable_every=50, reliable_delta=0.1)
    sessions = [_session(op, to_dev(b), **kw) for _ in range(3)]
    op.close()
    first, st = sessions[0]
    for rows, s in sessions[1:]:
        assert rows == first
        assert (s["iters"], s["reliable_updates"]) == (st["iters"], st["reliable_updates"])
    n_rel = st["reliable_updates"]
    assert n_rel >= 2
    # two FP64 hopping launches of each epilogue per reliable update, none for the gated rounds
    assert first.get("dslash_p64_r18_cloverinv") == 2 * n_rel
    assert first.get("dslash_p64_r18_xpay") == 2 * n_rel
    # one persistent launch per interval between reliable updates
    pc = [k for k in first if k.startswith("cg_persistent")]
    assert pc == [f"cg_persistent_p{inner}"]
    assert first[pc[0]] == n_rel
