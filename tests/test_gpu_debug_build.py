"""The debug build (libqcd_debug.so, compiled with QCD_DEBUG=1): index checks in every kernel's field
accessors, reported through device words instead of traps.

* In a child process that loads the debug build, every operator in FP64/FP32/FP16 on a lattice with
  ragged blocks, the mixed FP32 / FP16 and plain FP64 solves, the force with the determinant term, the
  reconstruction of the odd sites and the t-slab operators run without a single index check firing, and agree with the oracle within the
  parity tolerances (FP64 1e-13, FP32 1e-6, FP16 5e-3; solves to a true residual of 1e-8, recomputed by
  the oracle within its rounding).
* The index self-test, which hands the spinor loader the site index V/2 (inside its scratch buffer, so
  that the load is harmless even unchecked), sets QCD_DBG_SPINOR in the debug build, and the next call
  finds the bits cleared.
* The release build reports itself as such and records nothing for the same self-test.
"""

import json
import os
import subprocess
import sys

import pytest

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_debug_build_runs_clean_and_reports_a_bad_index():
    require_gpu()
    from paper_0910_0262_gb300 import build, qcd as Q
    lib = build.build(debug=True)
    env = dict(os.environ, QCD_LIB=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_build_child.py")], env=env, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-4000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["lib"] == lib
    assert res["is_debug"] == 1
    assert res["violations"] == 0, res
    assert res["selftest"] == Q.QCD_DBG_SPINOR, res
    assert res["after_clear"] == 0, res
    assert res["worst"]["64"] <= 1e-13 and res["worst"]["32"] <= 1e-6 and res["worst"]["16"] <= 5e-3, res
    for inner, (tr, ok, reported) in res["solves"].items():
        assert ok and tr <= 1e-8 * (1 + 1e-6) and reported <= 1e-8, (inner, res["solves"])
    assert res["force_finite"], res
    assert res["slab_err"] <= 1e-13, res
    assert res["recon_err"] <= 1e-13, res


def test_release_build_has_no_checks():
    require_gpu()
    from paper_0910_0262_gb300 import qcd as Q
    op = Q.CloverWilson((4, 4, 4, 4), -1.0)
    Q.qcd_selftest_debug_index(op.ctx)
    v, is_debug = Q.qcd_debug_violations(op.ctx)
    op.close()
    assert (v, is_debug) == (0, 0)
