"""Single-site evaluation of the operator (oracle; test infrastructure).

The same standard definitions as ``dirac`` and ``evenodd`` (the paper, Sec. 1,
names the MILC clover application and prints no formula), written for one
output site at a time with explicit index arithmetic, so that lattices too
large for the whole-lattice numpy oracle (32^3 x 64, 48^3 x 96) can be checked
at sampled sites:

    (D psi)(x)  = sum_mu (1 - g_mu) s U_mu(x) psi(x+mu) + (1 + g_mu) s U_mu(x-mu)^dag psi(x-mu)
    A(x)        = 1 - kappa c_sw sum_{mu<nu} sigma_{mu nu} F_{mu nu}(x)
    (Mhat x)(e) = A(e) x(e) - kappa^2 sum_hops (D [A^-1 D x])(e)

Gauge fields are canonical [T, Z, Y, X, 4, 3, 3]; even/odd fields [V/2, 4, 3] with
the half index of site i equal to i // 2.
"""

import numpy as np

from .dirac import GAMMA, ONE4, PLANES, sigma, dagger, leaf_paths


def lex(dims, c):
    X, Y, Z, T = dims
    x, y, z, t = (c[0] % X, c[1] % Y, c[2] % Z, c[3] % T)
    return x + X * (y + Y * (z + Z * t))


def coords(dims, i):
    X, Y, Z, T = dims
    return (i % X, (i // X) % Y, (i // (X * Y)) % Z, i // (X * Y * Z))


def wrap(dims, c):
    return tuple(int(c[k] % dims[k]) for k in range(4))


def step(c, mu, s):
    d = list(c)
    d[mu] += s
    return tuple(d)


def link(U, dims, c, mu):
    x, y, z, t = wrap(dims, c)
    return U[t, z, y, x, mu]


def parity(c):
    return (c[0] + c[1] + c[2] + c[3]) % 2


def spinor(fe, fo, dims, c):
    """Value of the even/odd field pair at site c."""
    c = wrap(dims, c)
    f = fe if parity(c) == 0 else fo
    return f[lex(dims, c) // 2]


def hop_site(U, fe, fo, dims, c, t_bc):
    """(D psi)(c) for psi given by the even/odd pair (only the parity opposite to c is read)."""
    out = np.zeros((4, 3), dtype=complex)
    T = dims[3]
    for mu in range(4):
        fwd = step(c, mu, +1)
        s_f = t_bc if (mu == 3 and wrap(dims, c)[3] == T - 1) else 1.0
        u = link(U, dims, c, mu) * s_f
        out += (ONE4 - GAMMA[mu]) @ (spinor(fe, fo, dims, fwd) @ u.T)
        bwd = step(c, mu, -1)
        s_b = t_bc if (mu == 3 and wrap(dims, bwd)[3] == T - 1) else 1.0
        ub = link(U, dims, bwd, mu) * s_b
        out += (ONE4 + GAMMA[mu]) @ (spinor(fe, fo, dims, bwd) @ np.conj(ub))
    return out


def leaf_product(U, dims, c, path):
    prod = np.eye(3, dtype=complex)
    for offset, d, dag in path:
        u = link(U, dims, tuple(c[k] + offset[k] for k in range(4)), d)
        prod = prod @ (dagger(u) if dag else u)
    return prod


def clover_site(U, dims, c, kappa, csw):
    """A(c) as a 12 x 12 matrix (index 3*spin + colour)."""
    A = np.eye(12, dtype=complex)
    for mu, nu in PLANES:
        Q = sum(leaf_product(U, dims, c, p) for p in leaf_paths(mu, nu))
        F = (Q - dagger(Q)) / (8j)
        F = F - np.trace(F) * np.eye(3) / 3.0
        A -= kappa * csw * np.kron(sigma(mu, nu), F)
    return A


def mhat_site(U, x_e, dims, c, kappa, csw, t_bc, dagger_op=False):
    """(Mhat x)(c) at an even site c; with dagger_op, (Mhat^dag x)(c) = (g5 Mhat g5 x)(c)."""
    g5 = np.diag([1.0, 1.0, -1.0, -1.0])
    xe = np.einsum('st,nta->nsa', g5, x_e) if dagger_op else x_e
    zero_o = np.zeros_like(x_e)
    # t(y) = A(y)^-1 (D x)(y) on the odd neighbours y of c
    t_vals = {}
    for mu in range(4):
        for sgn in (+1, -1):
            y = wrap(dims, step(c, mu, sgn))
            if y not in t_vals:
                Dx = hop_site(U, xe, zero_o, dims, y, t_bc)
                Ay = clover_site(U, dims, y, kappa, csw)
                t_vals[y] = np.linalg.solve(Ay, Dx.reshape(12)).reshape(4, 3)
    # (D t)(c) with t known on the odd neighbours
    to = np.zeros_like(x_e)
    for y, v in t_vals.items():
        to[lex(dims, y) // 2] = v
    Dt = hop_site(U, np.zeros_like(x_e), to, dims, wrap(dims, c), t_bc)
    Ac = clover_site(U, dims, c, kappa, csw)
    res = (Ac @ xe[lex(dims, c) // 2].reshape(12)).reshape(4, 3) - kappa ** 2 * Dt
    return g5 @ res if dagger_op else res
