"""Plain, slow FP64 CPU oracle for the even-odd clover-Wilson hot path.

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only the test suite (``tests/``), the
``smoke()`` check in ``__graft_entry__`` and the CPU-baseline / reference arm
of ``bench.py`` may import it.  The product path (the CUDA library behind
``include/qcd.h`` and its Python binding) never imports, links or calls it,
and the two share no code: no kernels, headers, tables or helpers.

What it computes.  The paper (Shi, Kindratenko, Gottlieb, "Cell processor
implementation of a MILC lattice QCD application", Sec. 1) ports MILC's
``clover_dynamical`` application -- dynamical clover-improved Wilson fermions
in the hybrid-molecular-dynamics R algorithm.  It prints no formula, so every
definition here is the standard lattice-QCD one, fixed as a convention of this
project:

* ``lattice``  -- site order, shifts, even/odd split.
* ``dirac``    -- DeGrand-Rossi gammas; Wilson hopping term D and its explicit
  adjoint; clover leaves Q_{mu nu}, field strength F_{mu nu}; clover term
  A = 1 - kappa c_sw sum_{mu<nu} sigma_{mu nu} F_{mu nu}; the full operator
  M = A - kappa D and M^dagger.
* ``evenodd``  -- the Schur complement Mhat = A_ee - kappa^2 D_eo A_oo^-1 D_oe
  and its adjoint, with A_oo^-1 from numpy.linalg.inv.
* ``cg``       -- textbook conjugate gradient on Mhat^dagger Mhat.
* ``force``    -- dS/dU for S = phi^dagger (Mhat^dagger Mhat)^-1 phi by brute
  force insertion into every path (each hopping term, each clover leaf).
* ``cloverdet`` -- the clover determinant term S_det = -2 log det A_oo of the
  even-odd preconditioned action (numpy.linalg.slogdet per site) and its
  derivative by the same insertion; the full-lattice source preparation and
  odd-site reconstruction of the even-odd solve.
* ``md``       -- Wilson gauge action and force, momenta, the link update exp(eps P) U
  (scipy.linalg.expm) with reunitarisation, leapfrog, and the two-flavour R-algorithm step.
* ``measure``  -- Polyakov loop and the stochastic psi-bar psi estimate (the plaquette is in ``md``).
* ``local``    -- single-site evaluations of the operator for sampled checks of
  large lattices.

Every function is pinned by tests that do not reuse its own formula: the
free-field plane-wave closed form, gamma5-hermiticity and the explicit adjoint,
gauge covariance, abelian field-strength closed forms, dense brute-force solves
of the unpreconditioned M, and finite differences of S.  Parity with MILC 7.4's
own sign and normalisation conventions is unpinned (no MILC code or output is
available); the conventions are stated where they are defined.
"""

from . import lattice, dirac, evenodd, cg, force, cloverdet, md, measure, local  # noqa: F401
