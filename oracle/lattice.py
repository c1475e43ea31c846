"""Lattice geometry for the oracle (test infrastructure; see the package header).

The paper (Sec. 3) describes the MILC lattice as a 4-D grid of sites whose
kernels read data "in a lattice site" and "in the neighboring site"; it fixes
no index order.  Conventions of this project:

* a full-lattice field is an array indexed ``[t, z, y, x, ...]`` (C order), so
  the lexicographic site index is ``i = x + X*(y + Y*(z + Z*t))``;
* direction ``mu = 0, 1, 2, 3`` is ``x, y, z, t``;
* ``parity = (x + y + z + t) mod 2``; an even/odd field lists the sites of one
  parity in increasing lexicographic index.
"""

import numpy as np

# array axis holding direction mu
AXIS = (3, 2, 1, 0)


def lattice_shape(dims):
    """Array shape [T, Z, Y, X] of a lattice with extents dims = (X, Y, Z, T)."""
    X, Y, Z, T = dims
    return (T, Z, Y, X)


def volume(dims):
    X, Y, Z, T = dims
    return X * Y * Z * T


def shift(f, mu, step):
    """g(x) = f(x + step * mu_hat) with periodic wrap-around."""
    return np.roll(f, -step, axis=AXIS[mu])


def translate(f, offset):
    """g(y) = f(y - offset): moves a value computed at x to the site x + offset."""
    g = f
    for mu in range(4):
        if offset[mu]:
            g = np.roll(g, offset[mu], axis=AXIS[mu])
    return g


def at_offset(f, offset):
    """g(x) = f(x + offset) for a 4-vector offset (periodic)."""
    g = f
    for mu in range(4):
        if offset[mu]:
            g = np.roll(g, -offset[mu], axis=AXIS[mu])
    return g


def coords(dims):
    """Integer arrays x, y, z, t over the lattice, each of shape [T, Z, Y, X]."""
    t, z, y, x = np.indices(lattice_shape(dims))
    return x, y, z, t


def parity(dims):
    x, y, z, t = coords(dims)
    return (x + y + z + t) % 2


def split_eo(f, dims):
    """(f_even, f_odd): the sites of each parity in lexicographic order."""
    par = parity(dims).reshape(-1)
    flat = f.reshape((par.size,) + f.shape[4:])
    return flat[par == 0].copy(), flat[par == 1].copy()


def join_eo(f_even, f_odd, dims):
    """Inverse of split_eo; either half may be None (taken as zero)."""
    par = parity(dims).reshape(-1)
    ref = f_even if f_even is not None else f_odd
    out = np.zeros((par.size,) + ref.shape[1:], dtype=complex)
    if f_even is not None:
        out[par == 0] = f_even
    if f_odd is not None:
        out[par == 1] = f_odd
    return out.reshape(lattice_shape(dims) + ref.shape[1:])
