"""The oracle still reproduces its frozen output on a seeded 4x2x2x4 problem.

``tests/golden/oracle_small.json`` was written by ``tests/golden/make_golden.py``
(which calls only the oracle and the input generator).  A change to the oracle's
arithmetic that moves these numbers must cite the reading that justifies it.
"""

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402


def test_oracle_matches_frozen_values():
    with open(os.path.join(HERE, "golden", "oracle_small.json")) as f:
        want = json.load(f)
    got = make_golden.compute()
    for key in ("norm2_b", "norm2_Mhat_b", "action_S", "force_norm2"):
        assert abs(got[key] - want[key]) <= 1e-9 * abs(want[key]), key
    assert np.allclose(got["b_dot_Mhat_b"], want["b_dot_Mhat_b"], rtol=1e-10)
    assert np.allclose(got["force_000_mu3"], want["force_000_mu3"], rtol=1e-7, atol=1e-10)
