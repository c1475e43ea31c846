"""Molecular-dynamics step of the hybrid R algorithm for two flavours (oracle; test infrastructure).

The paper's application (Sec. 1) evolves the links with MILC's su3_rmd, the hybrid-molecular-dynamics
R algorithm of Gottlieb, Liu, Toussaint, Renken and Sugar (1987); the paper prints none of it.  The
definitions below are the standard ones, fixed as conventions of this project:

* Wilson gauge action  S_g = beta sum_x sum_{mu<nu} (1 - Re tr P_{mu nu}(x) / 3),
  P_{mu nu}(x) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag (plain links, no boundary sign).
* Momenta P_mu(x) = sum_a i p_a T_a (traceless anti-Hermitian, T_a = lambda_a / 2) conjugate to the
  coordinates of U -> exp(i eps_a T_a) U; kinetic energy K = sum_a p_a^2 / 2 = -sum tr(P^2).
* Equations of motion  dU/dtau = P U,  dP/dtau = -F(U),  F = sum_a i T_a dS/d eps_a the
  Lie-algebra force of ``force.lie_force`` (S = S_g + S_f + S_det), so H = K + S is conserved.
* Leapfrog: P -= eps/2 F; U = exp(eps P) U; P -= eps/2 F.
* R-algorithm step for the two flavours that Mhat^dag Mhat describes: the R algorithm evaluates the
  noisy pseudofermion phi = Mhat^dag eta at the time shifted by eps (1 - N_f / N_0) / 2 after the
  half step, with N_0 = 2 here, so the shift vanishes:
      U' = exp(eps/2 P) U;  phi = Mhat(U')^dag eta;
      P -= eps F(U', phi);  U = exp(eps/2 P) U'.
  eta (complex Gaussian, one field per pseudofermion) is an input: the random numbers are drawn by
  the caller.
* Links are reunitarised after every update: rows 0 and 1 by Gram-Schmidt, row 2 = conj(row 0 x
  row 1).
"""

import numpy as np
from scipy.linalg import expm

from .dirac import PLANES, dagger, path_product, unit
from .force import insert, lie_force, gradient as pf_gradient, action as pf_action
from .evenodd import SchurOperator
from . import cg, cloverdet


def plaquette_paths(mu, nu):
    """The plaquette U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag as a path of (offset, dir, dagger)."""
    z = (0, 0, 0, 0)
    return [(z, mu, False), (tuple(unit(mu)), nu, False), (tuple(unit(nu)), mu, True), (z, nu, True)]


def plaquette_field(U, mu, nu):
    return path_product(U, plaquette_paths(mu, nu))


def gauge_action(U, beta):
    s = 0.0
    for mu, nu in PLANES:
        P = plaquette_field(U, mu, nu)
        s += float(np.sum(1.0 - np.trace(P, axis1=-2, axis2=-1).real / 3.0))
    return beta * s


def mean_plaquette(U):
    """< Re tr P / 3 > over sites and the six planes."""
    return float(np.mean([np.mean(np.trace(plaquette_field(U, mu, nu), axis1=-2, axis2=-1).real / 3.0)
                          for mu, nu in PLANES]))


def gauge_gradient(U, beta):
    """Wirtinger gradient of S_g: -beta/3 Re tr P is Re tr(C P) with C = -beta/3 per plaquette."""
    G = np.zeros(U.shape, dtype=complex)
    C = np.broadcast_to(-beta / 3.0 * np.eye(3, dtype=complex), U.shape[:4] + (3, 3))
    for mu, nu in PLANES:
        insert(G, U, plaquette_paths(mu, nu), C)
    return G


def gauge_force(U, beta):
    return lie_force(U, gauge_gradient(U, beta))


def kinetic_energy(P):
    return float(-np.sum(np.trace(P @ P, axis1=-2, axis2=-1).real))


def reunitarise(U):
    r0 = U[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = U[..., 1, :] - np.sum(np.conj(r0) * U[..., 1, :], axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def update_links(U, P, eps):
    """exp(eps P) U link by link (scipy.linalg.expm), reunitarised."""
    E = np.empty_like(U)
    flatP = (eps * P).reshape(-1, 3, 3)
    flatE = E.reshape(-1, 3, 3)
    for k in range(flatP.shape[0]):
        flatE[k] = expm(flatP[k])
    return reunitarise(E @ U)


def fermion_force(U, kappa, csw, phis, with_det, tol=1e-12):
    """Lie force of sum_i phi_i^dag (Mhat^dag Mhat)^-1 phi_i (plus S_det): CG solves to tol."""
    op = SchurOperator(U, kappa, csw)
    G = np.zeros(U.shape, dtype=complex)
    for phi in phis:
        X, _, _ = cg.cg(op.MdagM, phi, tol=tol)
        G += pf_gradient(op, X)
    if with_det:
        G += cloverdet.gradient(op)
    return lie_force(U, G)


def total_force(U, beta, kappa, csw, phis, with_det):
    return gauge_force(U, beta) + fermion_force(U, kappa, csw, phis, with_det)


def r_step(U, P, eta, eps, beta, kappa, csw, with_det=True):
    """One R-algorithm step (module header) for pseudofermion noise fields eta [n, V/2, 4, 3]."""
    Uh = update_links(U, P, eps / 2.0)
    op = SchurOperator(Uh, kappa, csw)
    phis = [op.Mhat_dag(e) for e in eta]
    P = P - eps * total_force(Uh, beta, kappa, csw, phis, with_det)
    return update_links(Uh, P, eps / 2.0), P


def hamiltonian(U, P, beta, kappa, csw, phis, with_det):
    """K + S_g + S_f (fixed phi, dense-accuracy CG) + S_det."""
    op = SchurOperator(U, kappa, csw)
    H = kinetic_energy(P) + gauge_action(U, beta)
    for phi in phis:
        X, _, _ = cg.cg(op.MdagM, phi, tol=1e-13)
        H += pf_action(phi, X)
    if with_det:
        H += cloverdet.action(op)
    return H


def leapfrog(U, P, eps, nsteps, beta, kappa, csw, phis, with_det):
    """nsteps leapfrog steps with fixed pseudofermions phis."""
    F = total_force(U, beta, kappa, csw, phis, with_det)
    for _ in range(nsteps):
        P = P - eps / 2.0 * F
        U = update_links(U, P, eps)
        F = total_force(U, beta, kappa, csw, phis, with_det)
        P = P - eps / 2.0 * F
    return U, P
