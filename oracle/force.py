"""Fermion force for S = phi^dag (Mhat^dag Mhat)^-1 phi by brute-force path insertion (oracle).

The paper's R-algorithm application (Sec. 1, su3_rmd) moves the gauge field with
the derivative of the pseudofermion action; it prints no formula.  Derivation
used here (a convention of this project):

With X = (Mhat^dag Mhat)^-1 phi and Y = Mhat X, varying the links gives

    dS = -2 Re[ Y^dag dMhat X ]
       = -2 Re[ W^dag dA X ] + 2 kappa^2 Re[ Y^dag dD X ]

on full-lattice fields X = (X_e, X_o), Y = (Y_e, Y_o), W = (Y_e, kappa^2 Y_o) with
X_o = A_oo^-1 D_oe X_e and Y_o = A_oo^-1 D_eo^dag Y_e (from dA^-1 = -A^-1 dA A^-1).

Every term is Re tr(C(x) d path(x)) for a closed or open product of links:

* hopping, forward:  path U_mu(x), C = 2 kappa^2 s sum_s [(1-g_mu) X(x+mu)]_s Y(x)_s^dag
* hopping, backward: path U_mu(x-mu)^dag, C = 2 kappa^2 s sum_s [(1+g_mu) X(x-mu)]_s Y(x)_s^dag
* clover: each leaf of Q_{mu nu}(x), C = -i (kappa c_sw / 4) (S~ + S~^dag),
  S~ the traceless part of sum_s [sigma_{mu nu} X(x)]_s W(x)_s^dag.

For an occurrence path = P1 U P2 of a link, Re tr(C dpath) = Re tr(G^dag dU) with
G += (P2 C P1)^dag; for path = P1 U^dag P2, G += P2 C P1.  G is the Wirtinger
gradient dS/dRe U + i dS/dIm U of S as a function of unconstrained complex links
(the convention of torch.autograd).  The Lie-algebra force for left
multiplication U -> exp(omega) U, omega = i eps_a T_a, T_a = lambda_a / 2, is

    F = sum_a i T_a dS/d eps_a = -1/2 P_TA(U G^dag),
    P_TA(M) = (M - M^dag)/2 - tr(M - M^dag)/6.
"""

import numpy as np

from . import dirac
from .dirac import GAMMA, ONE4, PLANES, sigma, dagger, spin_mul, leaf_paths, path_link, unit
from .lattice import join_eo, translate, shift
from .evenodd import SchurOperator


def outer(v, w):
    """C[i, j] = sum_s v_s[i] conj(w_s[j]) for spinor fields v, w."""
    return np.einsum('...si,...sj->...ij', v, np.conj(w))


def insert(G, U, path, C):
    """Accumulate into G the derivative of Re sum_x tr(C(x) path(x)) w.r.t. every link on the path."""
    mats = [path_link(U, step) for step in path]
    eye = np.broadcast_to(np.eye(3, dtype=complex), C.shape)
    for k, (offset, d, dag) in enumerate(path):
        P1 = eye
        for m in mats[:k]:
            P1 = P1 @ m
        P2 = eye
        for m in mats[k + 1:]:
            P2 = P2 @ m
        M = P2 @ C @ P1
        contrib = M if dag else dagger(M)
        # contrib(x) belongs to the link at x + offset
        G[..., d, :, :] += translate(contrib, offset)


def gradient_from_fields(U, kappa, csw, t_bc, X, Y, W):
    """G = dS/dRe U + i dS/dIm U given full-lattice X, Y, W (see the module header)."""
    dims = (U.shape[3], U.shape[2], U.shape[1], U.shape[0])
    s = dirac.boundary_sign(dims, t_bc)
    G = np.zeros(U.shape, dtype=complex)
    k2 = kappa ** 2
    zero = (0, 0, 0, 0)
    for mu in range(4):
        # forward hop at x: Y(x)^dag (1-g) s U_mu(x) X(x+mu)
        C = 2 * k2 * s[..., mu, None, None] * outer(spin_mul(ONE4 - GAMMA[mu], shift(X, mu, +1)), Y)
        insert(G, U, [(zero, mu, False)], C)
        # backward hop at x: Y(x)^dag (1+g) s(x-mu) U_mu(x-mu)^dag X(x-mu)
        s_b = shift(s[..., mu], mu, -1)
        C = 2 * k2 * s_b[..., None, None] * outer(spin_mul(ONE4 + GAMMA[mu], shift(X, mu, -1)), Y)
        back = tuple(-c for c in unit(mu))
        insert(G, U, [(back, mu, True)], C)
    for mu, nu in PLANES:
        Sig = outer(spin_mul(sigma(mu, nu), X), W)
        tr = np.trace(Sig, axis1=-2, axis2=-1)
        St = Sig - tr[..., None, None] * np.eye(3) / 3.0
        C = -1j * (kappa * csw / 4.0) * (St + dagger(St))
        for path in leaf_paths(mu, nu):
            insert(G, U, path, C)
    return G


def solution_fields(op, X_e):
    """Full-lattice X, Y, W of the module header from the even-site solution X_e."""
    Y_e = op.Mhat(X_e)
    X_o = SchurOperator.site(op.A_oo_inv, op.D_oe(X_e))
    Y_o = SchurOperator.site(op.A_oo_inv, op.D_eo_dag(Y_e))
    k2 = op.kappa ** 2
    X = join_eo(X_e, X_o, op.dims)
    Y = join_eo(Y_e, Y_o, op.dims)
    W = join_eo(Y_e, k2 * Y_o, op.dims)
    return X, Y, W


def gradient(op, X_e):
    """Wirtinger gradient G of S for the solution X_e (summed over a leading RHS axis if present)."""
    if X_e.ndim == 4:
        return sum(gradient(op, x) for x in X_e)
    X, Y, W = solution_fields(op, X_e)
    return gradient_from_fields(op.U, op.kappa, op.csw, op.t_bc, X, Y, W)


def project_ta(M):
    """Traceless anti-Hermitian part: (M - M^dag)/2 - tr(M - M^dag)/6."""
    A = (M - dagger(M)) / 2.0
    tr = np.trace(A, axis1=-2, axis2=-1)
    return A - tr[..., None, None] * np.eye(3) / 3.0


def lie_force(U, G):
    """F_mu(x) = -1/2 P_TA(U G^dag): the force along U -> exp(i eps_a T_a) U."""
    return -0.5 * project_ta(U @ dagger(G))


def action(phi, X_e):
    """S = Re <phi, X> summed over right-hand sides."""
    return float(np.vdot(phi.reshape(-1), X_e.reshape(-1)).real)
