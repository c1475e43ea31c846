"""The single-site oracle (used for sampled checks on large lattices) agrees with the
whole-lattice oracle, which the other oracle tests pin against the physics."""

import numpy as np

from oracle import local, evenodd, dirac, lattice
from paper_0910_0262_gb300 import synth


def test_local_matches_whole_lattice():
    dims = (4, 2, 6, 4)
    kappa, csw = 0.12, 1.0
    U, b = synth.make_problem(dims, 0.3, 5)
    op = evenodd.SchurOperator(U, kappa, csw, -1.0)
    x = b[0]
    Mx = op.Mhat(x)
    Mdx = op.Mhat_dag(x)
    rng = np.random.default_rng(1)
    X, Y, Z, T = dims
    A = dirac.clover_term(U, kappa, csw)
    for _ in range(6):
        h = int(rng.integers(0, x.shape[0]))
        # even site with half index h
        i = next(i for i in range(2 * h, 2 * h + 2) if sum(local.coords(dims, i)) % 2 == 0)
        c = local.coords(dims, i)
        assert np.max(np.abs(local.mhat_site(U, x, dims, c, kappa, csw, -1.0) - Mx[h])) < 1e-13
        assert np.max(np.abs(local.mhat_site(U, x, dims, c, kappa, csw, -1.0, dagger_op=True) - Mdx[h])) < 1e-13
        t, z, y, xx = c[3], c[2], c[1], c[0]
        assert np.max(np.abs(local.clover_site(U, dims, c, kappa, csw) - A[t, z, y, xx])) < 1e-14
    # hopping term at odd sites
    De = op.D_oe(x)
    for h in (0, 7, 20):
        i = next(i for i in range(2 * h, 2 * h + 2) if sum(local.coords(dims, i)) % 2 == 1)
        c = local.coords(dims, i)
        assert np.max(np.abs(local.hop_site(U, x, np.zeros_like(x), dims, c, -1.0) - De[h])) < 1e-13
