"""Clover-improved Wilson operator on the full lattice (oracle; test infrastructure).

The paper's application is MILC's ``clover_dynamical`` (Sec. 1): Wilson fermions
with the Sheikholeslami-Wohlert clover term.  The paper gives no formula; this
module writes out the standard definitions, as conventions of this project:

Gamma basis (DeGrand-Rossi, chiral: gamma_5 = diag(1, 1, -1, -1)), rows listed.

Wilson-clover operator, kappa normalisation, mu = x, y, z, t:

    (M psi)(x) = A(x) psi(x) - kappa (D psi)(x)
    (D psi)(x) = sum_mu [ (1 - g_mu) U_mu(x) psi(x+mu)
                          + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu) ]
    A(x)       = 1 - kappa c_sw sum_{mu<nu} sigma_{mu nu} F_{mu nu}(x)
    sigma_{mu nu} = (i/2) [g_mu, g_nu]
    F_{mu nu}  = traceless part of (Q_{mu nu} - Q_{mu nu}^dag) / (8 i)

with Q_{mu nu}(x) the sum of the four plaquette "leaves" in the (mu, nu) plane
that start and end at x, all with the same orientation.  Boundary conditions:
periodic in x, y, z and antiperiodic in t, realised as a factor t_bc (= -1) on
U_t(x) at t = T - 1 in the hopping term only; clover leaves use the plain links.

Spinor fields are complex arrays [t, z, y, x, spin(4), colour(3)], gauge fields
[t, z, y, x, mu(4), 3, 3].  A site matrix acting on a spinor is a 12 x 12 array
indexed by 3*spin + colour.
"""

import numpy as np

from .lattice import shift, at_offset, lattice_shape

I = 1j

GAMMA = np.zeros((4, 4, 4), dtype=complex)
GAMMA[0] = [[0, 0, 0, I], [0, 0, I, 0], [0, -I, 0, 0], [-I, 0, 0, 0]]
GAMMA[1] = [[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]]
GAMMA[2] = [[0, 0, I, 0], [0, 0, 0, -I], [-I, 0, 0, 0], [0, I, 0, 0]]
GAMMA[3] = [[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]]
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
ONE4 = np.eye(4, dtype=complex)


def sigma(mu, nu):
    """sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu]."""
    return 0.5j * (GAMMA[mu] @ GAMMA[nu] - GAMMA[nu] @ GAMMA[mu])


PLANES = [(mu, nu) for mu in range(4) for nu in range(mu + 1, 4)]


def dagger(m):
    return np.conj(np.swapaxes(m, -1, -2))


def spin_mul(g, psi):
    """(g psi)_s = sum_t g[s, t] psi_t for a 4x4 spin matrix g."""
    return np.einsum('st,...ta->...sa', g, psi)


def colour_mul(u, psi):
    """(u psi)_{s a} = sum_b u[a, b] psi_{s b} for a site field of 3x3 matrices u."""
    return np.einsum('...ab,...sb->...sa', u, psi)


def gamma5(psi):
    return spin_mul(GAMMA5, psi)


def boundary_sign(dims, t_bc):
    """s_mu(x): t_bc on the t-links of the last time slice, 1 elsewhere."""
    s = np.ones(lattice_shape(dims) + (4,))
    s[-1, :, :, :, 3] = t_bc
    return s


def hopping(U, psi, t_bc):
    """(D psi)(x) = sum_mu (1-g_mu) s U_mu(x) psi(x+mu) + (1+g_mu) s U_mu(x-mu)^dag psi(x-mu)."""
    dims = psi.shape[3], psi.shape[2], psi.shape[1], psi.shape[0]
    s = boundary_sign(dims, t_bc)
    out = np.zeros_like(psi, dtype=complex)
    for mu in range(4):
        Umu = U[..., mu, :, :] * s[..., mu, None, None]
        fwd = colour_mul(Umu, shift(psi, mu, +1))
        out += spin_mul(ONE4 - GAMMA[mu], fwd)
        bwd = colour_mul(dagger(shift(Umu, mu, -1)), shift(psi, mu, -1))
        out += spin_mul(ONE4 + GAMMA[mu], bwd)
    return out


def hopping_dagger(U, chi, t_bc):
    """Explicit adjoint of ``hopping``:
    (D^dag chi)(y) = sum_mu (1-g_mu) s U_mu(y-mu)^dag chi(y-mu) + (1+g_mu) s U_mu(y) chi(y+mu).

    Written from the matrix elements of D (gamma_mu Hermitian), not from gamma_5;
    gamma_5-hermiticity is a test of the pair, not an assumption.
    """
    dims = chi.shape[3], chi.shape[2], chi.shape[1], chi.shape[0]
    s = boundary_sign(dims, t_bc)
    out = np.zeros_like(chi, dtype=complex)
    for mu in range(4):
        Umu = U[..., mu, :, :] * s[..., mu, None, None]
        from_below = colour_mul(dagger(shift(Umu, mu, -1)), shift(chi, mu, -1))
        out += spin_mul(dagger(ONE4 - GAMMA[mu]), from_below)
        from_above = colour_mul(Umu, shift(chi, mu, +1))
        out += spin_mul(dagger(ONE4 + GAMMA[mu]), from_above)
    return out


def unit(mu):
    e = [0, 0, 0, 0]
    e[mu] = 1
    return e


def vsum(*vs):
    return tuple(int(sum(c)) for c in zip(*vs))


def vneg(v):
    return tuple(-c for c in v)


def leaf_paths(mu, nu):
    """The four leaves of Q_{mu nu}(x): closed paths from x, same orientation.

    Each path is a list of links (offset, direction, daggered) meaning
    U_direction(x + offset), conjugate-transposed if daggered, multiplied in order:
      L1 = U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
      L2 = U_nu(x) U_mu(x-mu+nu)^dag U_nu(x-mu)^dag U_mu(x-mu)
      L3 = U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu)
      L4 = U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^dag
    """
    o = (0, 0, 0, 0)
    m = tuple(unit(mu))
    n = tuple(unit(nu))
    mm, nn = vneg(m), vneg(n)
    return [
        [(o, mu, False), (m, nu, False), (n, mu, True), (o, nu, True)],
        [(o, nu, False), (vsum(mm, n), mu, True), (mm, nu, True), (mm, mu, False)],
        [(mm, mu, True), (vsum(mm, nn), nu, True), (vsum(mm, nn), mu, False), (nn, nu, False)],
        [(nn, nu, True), (nn, mu, False), (vsum(nn, m), nu, False), (o, mu, True)],
    ]


def path_link(U, step):
    """Site field x -> U_d(x + offset) (daggered if asked) for one path step."""
    offset, d, dag = step
    u = at_offset(U[..., d, :, :], offset)
    return dagger(u) if dag else u


def path_product(U, path):
    prod = None
    for step in path:
        u = path_link(U, step)
        prod = u if prod is None else prod @ u
    return prod


def clover_leaves(U, mu, nu):
    """Q_{mu nu}(x): sum of the four leaves."""
    return sum(path_product(U, p) for p in leaf_paths(mu, nu))


def field_strength(U, mu, nu):
    """F_{mu nu} = (Q - Q^dag)/(8i) minus its trace/3 (traceless Hermitian)."""
    Q = clover_leaves(U, mu, nu)
    F = (Q - dagger(Q)) / (8j)
    tr = np.trace(F, axis1=-2, axis2=-1)
    return F - tr[..., None, None] * np.eye(3) / 3.0


def clover_term(U, kappa, csw):
    """A(x) = 1 - kappa c_sw sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(x), as [..., 12, 12]."""
    lat = U.shape[:4]
    A = np.zeros(lat + (4, 3, 4, 3), dtype=complex)
    A += np.einsum('st,ab->satb', ONE4, np.eye(3))
    for mu, nu in PLANES:
        F = field_strength(U, mu, nu)
        A -= kappa * csw * np.einsum('st,...ab->...satb', sigma(mu, nu), F)
    return A.reshape(lat + (12, 12))


def site_apply(A, psi):
    """(A psi)(x) for a site field of 12 x 12 matrices."""
    shape = psi.shape
    flat = psi.reshape(shape[:-2] + (12,))
    return np.einsum('...ij,...j->...i', A, flat).reshape(shape)


def apply_M(U, A, psi, kappa, t_bc):
    """M psi = A psi - kappa D psi."""
    return site_apply(A, psi) - kappa * hopping(U, psi, t_bc)


def apply_Mdag(U, A, psi, kappa, t_bc):
    """M^dag psi = A^dag psi - kappa D^dag psi."""
    return site_apply(dagger(A), psi) - kappa * hopping_dagger(U, psi, t_bc)
