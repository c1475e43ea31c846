"""Small helpers for the tests: random fields and norms (no operator arithmetic)."""

import numpy as np


def rand_spinor(shape, rng):
    return rng.standard_normal(tuple(shape) + (4, 3)) + 1j * rng.standard_normal(tuple(shape) + (4, 3))


def rel_l2(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def lattice_shape(dims):
    X, Y, Z, T = dims
    return (T, Z, Y, X)
