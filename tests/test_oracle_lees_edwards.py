"""Pins of the oracle's Lees-Edwards box (the sheared periodic box of a
simple-shear run; lattice e1 = (L, 0, 0), e2 = (tilt, L, 0), e3 = (0, 0, L)):

* a tilt of L (or any tilt plus a multiple of L) is the same lattice, so the
  mobility must not change;
* the Ewald split stays exact: the mobility does not depend on xi;
* moving a bead by the lattice vector e2 changes nothing;
* the mobility stays symmetric and positive definite;
* the saddle solve with a tilt is translation invariant under e2 too;
* the minimum image returns a lattice-equivalent displacement inside the box.
"""

import numpy as np

import oracle as O
import synth


def beads(seed=3, n=4, L=12.0):
    rng = np.random.default_rng(seed)
    while True:
        p = rng.uniform(0.0, L, size=(n, 3))
        d = O.min_image(p[:, None, :] - p[None, :, :], L, 0.37 * L)
        r = np.linalg.norm(d, axis=-1) + np.eye(n) * 10
        if r.min() > 2.2:
            return p


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_minimum_image_reduces_into_the_box():
    # the reduced displacement differs from the input by a lattice vector
    # n1 e1 + n2 e2 + n3 e3 (integer n) and lies within half a box along every
    # axis (wrapped across y first, which moves it by the offset along x)
    rng = np.random.default_rng(17)
    L = 10.0
    for tilt in (0.0, 0.37 * L, -0.49 * L):
        d = rng.uniform(-1.6 * L, 1.6 * L, size=(400, 3))
        m = O.min_image(d, L, tilt)
        assert np.abs(m).max() <= 0.5 * L + 1e-12
        t = d - m
        n2 = t[:, 1] / L
        n1 = (t[:, 0] - n2 * tilt) / L
        n3 = t[:, 2] / L
        for nk in (n1, n2, n3):
            assert np.abs(nk - np.round(nk)).max() < 1e-9


def test_tilt_is_defined_modulo_L():
    L = 12.0
    p = beads()
    M0 = O.mobility_dense(p, L, tilt=0.0)
    M1 = O.mobility_dense(p, L, tilt=L)
    assert rel(M1, M0) < 1e-11
    Ma = O.mobility_dense(p, L, tilt=0.3 * L)
    Mb = O.mobility_dense(p, L, tilt=-0.7 * L)
    assert rel(Mb, Ma) < 1e-11
    assert rel(Ma, M0) > 1e-4  # the tilt matters


def test_split_independence_with_tilt():
    L = 12.0
    p = beads(4)
    Ma = O.mobility_dense(p, L, xi=0.45, tilt=0.37 * L)
    Mb = O.mobility_dense(p, L, xi=0.8, tilt=0.37 * L)
    assert rel(Ma, Mb) < 1e-10


def test_lattice_translation_and_spd():
    L, tilt = 12.0, 0.37 * 12.0
    p = beads(5)
    M = O.mobility_dense(p, L, tilt=tilt)
    q = p.copy()
    q[1] += np.array([tilt, L, 0.0])
    q[2] -= np.array([tilt, L, 0.0])
    assert rel(O.mobility_dense(q, L, tilt=tilt), M) < 1e-11
    assert np.abs(M - M.T).max() < 1e-12 * np.abs(M).max()
    assert np.linalg.eigvalsh(M).min() > 0.0


def test_solve_with_tilt_translation_invariant():
    L, tilt = 14.0, -0.41 * 14.0
    pos, body, _ = synth.config_doublets(3, L, seed=9)
    ft = synth.random_forces(3, 2)
    a = O.solve(pos, body, L, gamma=0.7, FT=ft, rlub=3.0, tilt=tilt)
    q = pos.copy()
    q[body == 1] += np.array([tilt, L, 0.0])
    b = O.solve(q, body, L, gamma=0.7, FT=ft, rlub=3.0, tilt=tilt)
    assert a["rel_residual"] < 1e-12
    # the background flow is gamma y x, so a body moved by e2 sees U_inf + gamma L x;
    # its disturbance velocity and everything else are unchanged
    assert np.allclose(b["dU"], a["dU"], rtol=1e-10, atol=1e-12)
    assert np.allclose(b["S"], a["S"], rtol=1e-10, atol=1e-12)
