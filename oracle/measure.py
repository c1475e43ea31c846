"""Measurements per trajectory (oracle; test infrastructure): plaquette, Polyakov loop and the
stochastic estimate of psi-bar psi.  The paper's application prints these each trajectory (Sec. 1
names only the application); the definitions are the standard ones, conventions of this project:

* mean plaquette  < Re tr P_{mu nu}(x) / 3 >  (``md.mean_plaquette``);
* Polyakov loop   L = < tr prod_{t=0}^{T-1} U_t(xvec, t) / 3 >  over the spatial sites, plain links
  (the antiperiodic sign is a boundary condition of the fermions only);
* psi-bar psi     Re eta^dag M^-1 eta / (2 V) per noise vector eta (complex Gaussian, unit variance
  per real, on all V sites): E[eta eta^dag] = 2, so this estimates Re Tr M^-1 / V without bias;
  M^-1 eta by the even-odd route of ``cloverdet`` (Mhat x_e = bhat_e by CG on the normal equations,
  then x_o).
"""

import numpy as np

from . import cg, cloverdet


def polyakov_loop(U):
    """Complex mean over spatial sites of tr prod_t U_t(x, t) / 3 (U: [T, Z, Y, X, 4, 3, 3])."""
    T = U.shape[0]
    prod = U[0, ..., 3, :, :]
    for t in range(1, T):
        prod = prod @ U[t, ..., 3, :, :]
    return complex(np.mean(np.trace(prod, axis1=-2, axis2=-1)) / 3.0)


def solve_full(op, b_e, b_o, tol=1e-12):
    """x = M^-1 b on both parities through the Schur complement (CG on Mhat^dag Mhat)."""
    bh = cloverdet.prepare_source(op, b_e, b_o)
    x_e, _, _ = cg.cg(op.MdagM, op.Mhat_dag(bh), tol=tol)
    return x_e, cloverdet.reconstruct_odd(op, x_e, b_o)


def pbp(op, eta_e, eta_o, tol=1e-12):
    """Re eta^dag M^-1 eta / (2 V): eta = (eta_e, eta_o); the factor 2 makes it an estimate of
    Re Tr M^-1 / V for complex Gaussian eta with unit variance per real component."""
    x_e, x_o = solve_full(op, eta_e, eta_o, tol)
    V = 2 * eta_e.shape[0]
    return float((np.vdot(eta_e.reshape(-1), x_e.reshape(-1)) + np.vdot(eta_o.reshape(-1), x_o.reshape(-1))).real
                 / (2.0 * V))
