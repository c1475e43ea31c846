"""Write tests/golden/oracle_small.json: oracle values for a seeded 4x2x2x4 problem.

The paper prints no worked example (it reports only Cell/Xeon timings, Sec. 4),
so this fixture is not a physics pin; it freezes the oracle's own output so that
any later change to the oracle's arithmetic shows up as a failing test and has
to be justified.  It calls only ``oracle/`` and the seeded input generator.

Run:  python tests/golden/make_golden.py
"""

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import evenodd, cg, force  # noqa: E402
from paper_0910_0262_gb300 import synth  # noqa: E402


def compute():
    dims, eps, seed = (4, 2, 2, 4), 0.2, 1
    kappa, csw = 0.12, 1.0
    U, b = synth.make_problem(dims, eps, seed)
    op = evenodd.SchurOperator(U, kappa, csw)
    Mb = op.Mhat(b[0])
    x, iters, res = cg.cg(op.MdagM, b[0], tol=1e-13)
    F = force.lie_force(U, force.gradient(op, x))
    return {
        "dims": list(dims), "eps": eps, "seed": seed, "kappa": kappa, "csw": csw, "t_bc": -1.0,
        "norm2_b": float(np.vdot(b, b).real),
        "norm2_Mhat_b": float(np.vdot(Mb, Mb).real),
        "b_dot_Mhat_b": [float(np.vdot(b[0], Mb).real), float(np.vdot(b[0], Mb).imag)],
        "action_S": force.action(b[0], x),
        "force_norm2": float(np.sum(np.abs(F) ** 2)),
        "force_000_mu3": [[float(F[0, 0, 0, 0, 3, i, j].real), float(F[0, 0, 0, 0, 3, i, j].imag)]
                          for i in range(3) for j in range(3)],
    }


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_small.json")
    with open(out, "w") as f:
        json.dump(compute(), f, indent=1)
    print("wrote", out)
