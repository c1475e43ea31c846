"""The seeded input generator: SU(3) links near unity, reproducible streams, shapes."""

import numpy as np

from paper_0910_0262_gb300 import synth


def test_links_are_su3_and_near_unit():
    U, b = synth.make_problem((4, 2, 2, 4), 0.2, 1, nrhs=3)
    assert U.shape == (4, 2, 2, 4, 4, 3, 3)
    assert b.shape == (3, 32, 4, 3)
    eye = np.eye(3)
    assert np.max(np.abs(U @ np.conj(np.swapaxes(U, -1, -2)) - eye)) < 1e-14
    assert np.max(np.abs(np.linalg.det(U) - 1)) < 1e-14
    # exp(i eps H) with eps = 0.2: |U - 1| stays O(eps)
    assert np.max(np.abs(U - eye)) < 1.5
    assert abs(np.mean(np.real(np.trace(U, axis1=-2, axis2=-1))) / 3 - 1) < 0.05


def test_generator_is_exp_of_hermitian():
    rng = np.random.Generator(np.random.PCG64(3))
    h = rng.standard_normal((5, 8))
    H = np.einsum('na,aij->nij', h, synth.T_GEN)
    from scipy.linalg import expm
    for n in range(5):
        assert np.max(np.abs(synth._exp_i(H[n:n + 1], 0.2)[0] - expm(0.2j * H[n]))) < 1e-14


def test_seeded_reproducible():
    U1, b1 = synth.make_problem((2, 2, 2, 2), 0.2, 7)
    U2, b2 = synth.make_problem((2, 2, 2, 2), 0.2, 7)
    assert np.array_equal(U1, U2) and np.array_equal(b1, b2)
    U3, _ = synth.make_problem((2, 2, 2, 2), 0.2, 8)
    assert not np.array_equal(U1, U3)
    s = synth.sample_links((4, 4, 4, 4), 64, 3)
    assert len(set(s)) == 64
