"""Clover determinant term and full-lattice even-odd solve (oracle; test infrastructure).

Writing the clover-Wilson operator even-first, M = [[A_ee, -kappa D_eo], [-kappa D_oe, A_oo]],
its determinant factorises as det M = det A_oo det Mhat with the Schur complement Mhat of
``evenodd``.  The two-flavour action of the even-odd preconditioned R/HMC algorithm (the
application the paper ports, Sec. 1) is therefore the pseudofermion term plus

    S_det = -2 log det A_oo = -2 sum_{x odd} log det A(x),

which depends on the links through the clover term only (a convention of this project: the paper
prints no formula).

Its variation: dS_det = -2 sum_x tr(A(x)^-1 dA(x)) with dA = -kappa c_sw sum_{mu<nu} sigma_{mu nu}
(x) dF_{mu nu}.  With B_{mu nu}(x)_{ab} = sum_{s,t} [A(x)^-1]_{(s a),(t b)} sigma_{mu nu}[t, s] this
is 2 kappa c_sw sum tr(B dF), and since F = traceless (Q - Q^dag)/(8i) and S_det is real,

    dS_det = sum_{x odd} sum_{mu<nu} Re tr(C(x) dQ_{mu nu}(x)),
    C = -i (kappa c_sw / 4) (B~ + B~^dag),  B~ the traceless part of B,

the same form as the clover part of the pseudofermion force, so the derivative is taken by the
same brute-force insertion into every leaf (``force.insert``).

Full-lattice solve of M (x_e, x_o) = (b_e, b_o): eliminating x_o gives

    Mhat x_e = b_e + kappa D_eo A_oo^-1 b_o,    x_o = A_oo^-1 (b_o + kappa D_oe x_e).
"""

import numpy as np

from . import dirac
from .dirac import PLANES, sigma, dagger
from .force import insert
from .lattice import join_eo, split_eo
from .evenodd import SchurOperator


def logdet(op):
    """(sum over even sites, sum over odd sites) of log det A(x) (numpy.linalg.slogdet per site)."""
    A_e, A_o = op.A_ee, op.A_oo
    out = []
    for A in (A_e, A_o):
        sign, ld = np.linalg.slogdet(A)
        if np.any(sign.real <= 0.0):
            raise ValueError("clover block with non-positive determinant")
        out.append(float(np.sum(ld)))
    return tuple(out)


def action(op):
    """S_det = -2 sum_{x odd} log det A(x)."""
    return -2.0 * logdet(op)[1]


def coefficients(op):
    """C_{mu nu}(x) of the module header for every plane: [6, T, Z, Y, X, 3, 3], zero on even sites."""
    Ainv = op.A_oo_inv.reshape(op.A_oo_inv.shape[0], 4, 3, 4, 3)  # [n, s, a, t, b]
    Cs = []
    for mu, nu in PLANES:
        B = np.einsum('nsatb,ts->nab', Ainv, sigma(mu, nu))
        tr = np.trace(B, axis1=-2, axis2=-1)
        Bt = B - tr[..., None, None] * np.eye(3) / 3.0
        C_o = -1j * (op.kappa * op.csw / 4.0) * (Bt + dagger(Bt))
        Cs.append(join_eo(np.zeros_like(C_o), C_o, op.dims))
    return np.stack(Cs)


def gradient(op):
    """Wirtinger gradient G = dS_det/dRe U + i dS_det/dIm U."""
    G = np.zeros(op.U.shape, dtype=complex)
    C = coefficients(op)
    for k, (mu, nu) in enumerate(PLANES):
        for path in dirac.leaf_paths(mu, nu):
            insert(G, op.U, path, C[k])
    return G


def prepare_source(op, b_e, b_o):
    """b_e + kappa D_eo A_oo^-1 b_o: the even-site source of the Schur system."""
    return b_e + op.kappa * op.D_eo(SchurOperator.site(op.A_oo_inv, b_o))


def reconstruct_odd(op, x_e, b_o):
    """x_o = A_oo^-1 (b_o + kappa D_oe x_e)."""
    return SchurOperator.site(op.A_oo_inv, b_o + op.kappa * op.D_oe(x_e))
