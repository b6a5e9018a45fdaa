"""Pins of the oracle's periodic mobility: splitting independence, Hasimoto's
finite-size coefficient, symmetry and positive definiteness (CPU only)."""

import numpy as np
import pytest

import oracle as O
from conftest import golden

PI = np.pi


def test_mobility_independent_of_splitting():
    rng = np.random.default_rng(11)
    L = 12.0
    pos = np.array([[1.0, 1.0, 1.0], [3.05, 1.2, 0.8], [7.0, 6.0, 9.0], [10.5, 2.0, 5.0]])
    # None: the oracle's own splitting and cut-offs (oracle_split)
    Ms = [O.mobility_dense(pos, L, xi=x) for x in (None, 0.55, 0.8, 1.3)]
    scale = np.abs(Ms[0]).max()
    for M in Ms[1:]:
        assert np.abs(M - Ms[0]).max() / scale < 1e-11


def test_mobility_symmetric_positive_definite():
    rng = np.random.default_rng(12)
    L = 15.0
    pos = rng.uniform(0, L, size=(5, 3))
    M = O.mobility_dense(pos, L)
    assert np.abs(M - M.T).max() < 1e-14
    np.linalg.cholesky(M)
    assert np.linalg.eigvalsh(M).min() > 0


def test_hasimoto_finite_size_coefficient():
    # mu(L)/mu0 = 1 - c1 a/L + (4 pi/3)(a/L)^3 + O((a/L)^6)
    c_paper = golden("hasimoto_coefficient")
    Ls = np.array([20.0, 40.0, 80.0])
    mu = np.array([O.mobility_dense(np.zeros((1, 3)), L)[0, 0] * 6 * PI for L in Ls])
    c1 = (1 - mu + 4 * PI / 3 / Ls ** 3) * Ls
    # Hasimoto: 2.837297...; the paper rounds to 2.84
    assert np.allclose(c1, 2.8372975, atol=2e-6)
    assert abs(c1[-1] - c_paper) < 0.005


def test_two_beads_far_box_reduce_to_free_pair():
    # at fixed separation, periodic corrections to the pair and self blocks
    # coincide to O(1/L): M_ij - M_ii -> M_free(r) - M_self
    L = 160.0
    x = np.array([3.0, -1.0, 2.0])
    pos = np.array([[10.0, 10.0, 10.0], [10.0, 10.0, 10.0] + x])
    M = O.mobility_dense(pos, L).reshape(2, 11, 2, 11)
    diff = M[1, :3, 0, :3] - M[0, :3, 0, :3]
    ref = O.free_blocks(x[None])[0][:3, :3] - O.self_block()[:3, :3]
    assert np.abs(diff - ref).max() < 2e-4 * np.abs(ref).max()


def test_applied_wave_sum_equals_dense_wave_matrix():
    # the matrix-free form of the wave-space sum (used where the dense matrix
    # of a fine grid's wave-vector range is too large) against the dense one,
    # in the cube and in a Lees-Edwards box, with several k chunks
    rng = np.random.default_rng(21)
    L = 11.0
    pos = rng.uniform(0, L, size=(5, 3))
    F = rng.normal(size=(5, 11))
    for tilt in (0.0, 2.3):
        Md = O.mobility_wave_dense(pos, L, 0.9, 6.0, tilt=tilt).reshape(55, 55)
        u = O.mobility_wave_apply(pos, F, L, 0.9, 6.0, tilt=tilt, chunk=700)
        ref = (Md @ F.reshape(-1)).reshape(5, 11)
        assert np.abs(u - ref).max() < 1e-13 * np.abs(ref).max()


def test_applied_wave_sum_completes_the_split_independently_of_xi():
    # real-space part (dense) + applied wave-space part = the same periodic
    # mobility for two splitting parameters (the Ewald sum does not depend on xi)
    rng = np.random.default_rng(22)
    L = 13.0
    pos = rng.uniform(0, L, size=(4, 3))
    F = rng.normal(size=(4, 11))
    res = []
    for xi in (0.7, 1.1):
        rc = 2.0 + np.sqrt(46.0) / xi
        Mr = O.mobility_real_dense(pos, L, xi, rc).reshape(44, 44)
        uw = O.mobility_wave_apply(pos, F, L, xi, 2.0 * xi * np.sqrt(46.0))
        res.append(Mr @ F.reshape(-1) + uw.reshape(-1))
    assert np.abs(res[0] - res[1]).max() < 1e-11 * np.abs(res[0]).max()
