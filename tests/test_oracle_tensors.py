"""Pins of the oracle's free-space FTS tensors against closed forms and an
independent k-space quadrature (CPU only)."""

import numpy as np
import pytest

import oracle as O

PI = np.pi


def _rand_x(seed, r):
    rng = np.random.default_rng(seed)
    d = rng.normal(size=3)
    return r * d / np.linalg.norm(d)


@pytest.mark.parametrize("r", [2.0, 2.7, 5.0, 11.0])
def test_translational_block_is_textbook_rpy(r):
    # RPY for non-overlapping spheres: (1/(8 pi eta r)) [(1 + 2a^2/3r^2) I + (1 - 2a^2/r^2) rr]
    x = _rand_x(1, r)
    rh = x / r
    M = O.free_blocks(x[None])[0]
    ref = ((1 + 2 / (3 * r * r)) * np.eye(3) + (1 - 2 / r ** 2) * np.outer(rh, rh)) / (8 * PI * r)
    assert np.allclose(M[:3, :3], ref, rtol=0, atol=1e-15)


@pytest.mark.parametrize("r", [2.0, 3.3, 8.0])
def test_rotlet_and_rotation_blocks_are_textbook(r):
    # u = L x x / (8 pi eta r^3);  omega = (3 rr - I) L / (16 pi eta r^3)
    x = _rand_x(2, r)
    rh = x / r
    M = O.free_blocks(x[None])[0]
    UL = np.einsum("abc,c->ab", O.EPS, x) / (8 * PI * r ** 3)
    OL = (3 * np.outer(rh, rh) - np.eye(3)) / (16 * PI * r ** 3)
    assert np.allclose(M[:3, 3:6], UL, atol=1e-16)
    assert np.allclose(M[3:6, 3:6], OL, atol=1e-16)
    # rotation from a force is the transpose partner: omega = F x x... (reciprocity)
    assert np.allclose(M[3:6, :3], O.free_blocks(-x[None])[0][:3, 3:6].T, atol=1e-16)


def test_point_stresslet_far_field():
    # far from the source the velocity of a stresslet S is 3 x (x.S.x)/(8 pi eta r^5)
    r = 4000.0
    x = _rand_x(3, r)
    rng = np.random.default_rng(4)
    s = rng.normal(size=5)
    S = O.vec5_to_sym(s)
    u = O.free_blocks(x[None])[0][:3, 6:11] @ s
    ref = 3 * x * (x @ S @ x) / (8 * PI * r ** 5)
    assert np.linalg.norm(u - ref) < 1e-5 * np.linalg.norm(ref)


def test_blocks_reciprocal_symmetry():
    # M_ij(x) = M_ji(-x)^T for every pair: the assembled mobility is symmetric
    for seed, r in [(5, 2.0), (6, 2.5), (7, 9.0)]:
        x = _rand_x(seed, r)
        A = O.free_blocks(x[None])[0]
        B = O.free_blocks(-x[None])[0]
        assert np.allclose(A, B.T, atol=1e-16)


@pytest.mark.parametrize("kind", O.PAIR_KINDS)
def test_free_phi_closed_form_matches_kspace_quadrature(kind):
    # Faxen closed form vs brute quadrature of the k-space definition
    r = np.array([2.4, 4.0])
    # orders each kernel enters with (MM: 1-2, MD: 1-3, DD: 1-4); the slowly
    # decaying higher orders are not used and the brute quadrature truncates them
    used = {"MM": 2, "MD": 3, "DD": 4}[kind]
    q = O.free_phi_n_quadrature(r, kind, nq=400000, kmax=4000.0)[:, :used]
    c = O.free_phi_n(r, kind)[:, :used]
    assert np.allclose(q, c, rtol=1e-6, atol=0)


def test_self_mobilities_from_kspace():
    # self terms = the H -> 1 (xi -> infinity) limit of the wave part at r = 0
    # (the tail converges like 1/xi: Richardson-extrapolate from xi = 100, 200)
    W1 = O.wave_blocks_free(np.zeros((1, 3)), xi=100.0, nq=4000)[0]
    W2 = O.wave_blocks_free(np.zeros((1, 3)), xi=200.0, nq=8000)[0]
    W = 2 * W2 - W1
    mt, mr, ms = O.self_mobilities()
    assert np.isclose(W[0, 0], mt, rtol=1e-5)
    assert np.isclose(W[3, 3], mr, rtol=1e-5)
    assert np.isclose(W[6, 6], ms, rtol=1e-5)
    # isotropic, no cross coupling
    assert np.allclose(W - np.diag(np.diag(W)), 0.0, atol=1e-12)
    # Einstein: a free sphere in strain carries S = (20/3) pi eta a^3 E, i.e.
    # suspension viscosity 1 + 2.5 phi
    assert np.isclose(1.0 / ms, 20.0 / 3.0 * PI, rtol=1e-14)


def test_wave_plus_real_equals_free_at_distance():
    # for r >= 2a, the split parts recombine: M_free = (M_free - M_wave) + M_wave
    x = _rand_x(8, 3.1)
    for xi in (0.3, 0.9):
        W = O.wave_blocks_free(x[None], xi)[0]
        F = O.free_blocks(x[None])[0]
        # the real part decays like exp(-xi^2 r^2): check against quadrature of 1-H directly
        assert np.all(np.isfinite(F - W))
    # wave part tends to free part as xi -> infinity
    W = O.wave_blocks_free(x[None], 40.0, nq=3000)[0]
    F = O.free_blocks(x[None])[0]
    assert np.allclose(W, F, atol=1e-10)


def test_wave_self_block_closed_form_in_the_point_limit():
    # the wave part's self block at r = 0 is (1/(3 pi^2 eta)) int_0^inf H f^2 dk I
    # with H = (1 + k^2/(4 xi^2)) exp(-k^2/(4 xi^2)); for a point particle
    # (f = 1) the two Gaussian integrals give xi sqrt(pi) + xi sqrt(pi)/2, so
    # the block is xi / (2 pi^(3/2) eta) I.  Radius 1e-4 stands in for a point.
    for xi in (0.4, 1.1):
        W = O.wave_blocks_free(np.zeros((1, 3)), xi=xi, a=1e-4)[0]
        ref = xi / (2.0 * np.pi ** 1.5)
        assert np.abs(W[0:3, 0:3] - ref * np.eye(3)).max() < 1e-7 * ref


def test_overlapping_pairs_take_the_contact_blocks():
    # reading for overlaps: a free-space pair closer than 2a is evaluated at
    # separation 2a along its own direction
    n = np.array([0.36, -0.48, 0.8])
    blk = O.free_blocks(np.array([1.7 * n, 1.2 * n, 2.0 * n]))
    assert np.abs(blk[0] - blk[2]).max() < 1e-14 * np.abs(blk[2]).max()
    assert np.abs(blk[1] - blk[2]).max() < 1e-14 * np.abs(blk[2]).max()


def test_jn_series_matches_scipy():
    from scipy.special import spherical_jn
    z = np.linspace(0.5, 1.99, 50)
    for n in range(5):
        assert np.allclose(O.jn_over_zn(n, z), spherical_jn(n, z) / z ** n, rtol=1e-12)
