"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds no arithmetic of the Dirac operator, the solver or the force:
it only draws random numbers and turns them into inputs.

Recipe (the paper's lattices -- 8x8x16x16 and 16^4, Sec. 4 -- stand in for MILC
gauge configurations, which are not available):

* links U_mu(x) = exp(i eps H) with H = sum_{a=1..8} h_a lambda_a / 2 and
  h_a ~ N(0, 1) (Gell-Mann matrices lambda_a), eps = 0.2 (0.15 on the large
  lattices), then projected to SU(3): Gram-Schmidt on rows 0 and 1 and
  row 2 = conj(row 0 x row 1), so det U = 1 to rounding;
* random numbers come from numpy ``Generator(PCG64(seed))``, drawn in the order
  [t][z][y][x][mu][a], then the sources;
* a source is complex Gaussian with unit variance per real component on the even
  sites, laid out [V/2][spin 4][colour 3].

Lattice dims are (X, Y, Z, T); gauge arrays are complex128 [T, Z, Y, X, 4, 3, 3].
"""

import os

import numpy as np

GELL_MANN = np.zeros((8, 3, 3), dtype=complex)
GELL_MANN[0][0, 1] = GELL_MANN[0][1, 0] = 1
GELL_MANN[1][0, 1] = -1j
GELL_MANN[1][1, 0] = 1j
GELL_MANN[2][0, 0] = 1
GELL_MANN[2][1, 1] = -1
GELL_MANN[3][0, 2] = GELL_MANN[3][2, 0] = 1
GELL_MANN[4][0, 2] = -1j
GELL_MANN[4][2, 0] = 1j
GELL_MANN[5][1, 2] = GELL_MANN[5][2, 1] = 1
GELL_MANN[6][1, 2] = -1j
GELL_MANN[6][2, 1] = 1j
GELL_MANN[7] = np.diag([1, 1, -2]) / np.sqrt(3)
T_GEN = GELL_MANN / 2.0  # T_a = lambda_a / 2, tr(T_a T_b) = delta_ab / 2

_CHUNK = 1 << 18


def _exp_i(H, eps):
    """exp(i eps H) for a stack of Hermitian 3x3 matrices (Taylor series to 1e-17)."""
    A = 1j * eps * H
    out = np.broadcast_to(np.eye(3, dtype=complex), A.shape).copy()
    term = out.copy()
    for k in range(1, 30):
        term = term @ A / k
        out += term
        if np.max(np.abs(term)) < 1e-18:
            break
    return out


def project_su3(U):
    """Gram-Schmidt rows 0, 1; row 2 = conj(row0 x row1)."""
    r0 = U[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = U[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def _links_from_normals(h, eps):
    """SU(3) links exp(i eps sum_a h_a T_a), projected, for a block of normal draws h [n, 8]."""
    H = np.einsum('na,aij->nij', h, T_GEN)
    return project_su3(_exp_i(H, eps))


def random_links(dims, eps, rng, workers=None):
    """Near-unit SU(3) links [T, Z, Y, X, 4, 3, 3] drawn from rng in [t][z][y][x][mu][a] order.

    All normals are drawn first, in order; large lattices then turn them into links in
    parallel worker processes (spawned), which does not change the result.
    """
    X, Y, Z, T = dims
    n = X * Y * Z * T * 4
    h = rng.standard_normal((n, 8))
    U = np.empty((n, 3, 3), dtype=complex)
    chunks = [(start, min(n, start + _CHUNK)) for start in range(0, n, _CHUNK)]
    if workers is None:
        workers = min(16, os.cpu_count() or 1) if n > (1 << 22) else 1
    if workers > 1:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            futs = [ex.submit(_links_from_normals, h[a:b], eps) for a, b in chunks]
            for (a, b), f in zip(chunks, futs):
                U[a:b] = f.result()
    else:
        for a, b in chunks:
            U[a:b] = _links_from_normals(h[a:b], eps)
    return U.reshape(T, Z, Y, X, 4, 3, 3)


def gaussian_sources(dims, nrhs, rng):
    """nrhs complex Gaussian even-site fields [nrhs, V/2, 4, 3]."""
    X, Y, Z, T = dims
    vh = X * Y * Z * T // 2
    z = rng.standard_normal((nrhs, vh, 4, 3, 2))
    return z[..., 0] + 1j * z[..., 1]


def make_problem(dims, eps, seed, nrhs=1):
    """(U, b): links then nrhs sources from one PCG64 stream seeded with seed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    U = random_links(dims, eps, rng)
    b = gaussian_sources(dims, nrhs, rng)
    return U, b


def random_su3_field(shape, rng, eps=1.0):
    """SU(3) matrices of a given leading shape (used for gauge transformations)."""
    n = int(np.prod(shape))
    h = rng.standard_normal((n, 8))
    H = np.einsum('na,aij->nij', h, T_GEN)
    return project_su3(_exp_i(H, eps)).reshape(tuple(shape) + (3, 3))


def sample_links(dims, count, seed):
    """count distinct (site index, mu) pairs, seeded; site index is lexicographic."""
    X, Y, Z, T = dims
    rng = np.random.Generator(np.random.PCG64(seed))
    flat = rng.choice(X * Y * Z * T * 4, size=count, replace=False)
    return [(int(f // 4), int(f % 4)) for f in flat]


# Workloads of the paper's lattices and their large-volume extensions: dims, eps, seed, rhs.
WORKLOADS = {
    'c0_8x8x16x16': dict(dims=(8, 8, 16, 16), eps=0.2, seed=1, nrhs=1),
    'c1_16^4': dict(dims=(16, 16, 16, 16), eps=0.2, seed=2, nrhs=1),
    'c2_16^4_force': dict(dims=(16, 16, 16, 16), eps=0.2, seed=3, nrhs=1),
    'c3_32^3x64': dict(dims=(32, 32, 32, 64), eps=0.15, seed=4, nrhs=8),
    'c4_48^3x96': dict(dims=(48, 48, 48, 96), eps=0.15, seed=5, nrhs=4),
    # a small lattice for quick checks of the bench's two arms
    't_4x4x4x8': dict(dims=(4, 4, 4, 8), eps=0.2, seed=1, nrhs=1),
}
KAPPA = 0.12
CSW = 1.0
T_BC = -1.0
