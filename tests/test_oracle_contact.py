"""Pins of the Hertz contact oracle (oracle/contact_oracle.py; Sec. 4 normal
contact F_N = k_n delta^1.5 n): the closed form for one overlapping pair,
Newton's third law with central forces (forces and torques about a common
origin sum to zero), nothing without overlap or within one aggregate."""

import numpy as np

import synth
from oracle import contact_oracle as C
from oracle import fsd_oracle as F
from oracle import fsd_oracle as O


def test_single_pair_closed_form():
    L, kn, delta = 30.0, 1e4, 0.03
    d = np.array([1.0, 2.0, -2.0]) / 3.0
    pos = np.array([[5.0, 5.0, 5.0], [5.0, 5.0, 5.0] + (2.0 - delta) * d])
    out, fb = C.hertz_contact(pos, np.array([0, 1]), L, kn)
    f = kn * delta ** 1.5
    assert np.allclose(fb[1], f * d, rtol=1e-12) and np.allclose(fb[0], -f * d, rtol=1e-12)
    assert np.allclose(out[:, 3:], 0.0, atol=1e-12)  # single beads: no lever arm


def test_pair_forces_hertz_term_is_the_closed_form():
    # the combined interparticle-force routine with contact only: the same
    # Hertz law k_n delta^1.5 along the line of centres
    L, kn, delta = 30.0, 1e4, 0.03
    d = np.array([1.0, 2.0, -2.0]) / 3.0
    pos = np.array([[5.0, 5.0, 5.0], [5.0, 5.0, 5.0] + (2.0 - delta) * d])
    out, fb = C.pair_forces(pos, np.array([0, 1]), L, kn=kn)
    f = kn * delta ** 1.5
    assert np.allclose(fb[1], f * d, rtol=1e-12) and np.allclose(fb[0], -f * d, rtol=1e-12)


def test_pair_across_the_boundary():
    L, kn = 20.0, 10.0
    pos = np.array([[0.3, 4.0, 4.0], [L - 1.5, 4.0, 4.0]])  # 1.8 apart through the wall
    out, fb = C.hertz_contact(pos, np.array([0, 1]), L, kn)
    f = kn * 0.2 ** 1.5
    assert np.allclose(fb[0], [f, 0, 0], rtol=1e-12) and np.allclose(fb[1], [-f, 0, 0], rtol=1e-12)


def test_newton_third_law_for_rods():
    rng = np.random.default_rng(4)
    L = 40.0
    rods = [synth.rod(5) for _ in range(6)]
    pos, body = synth.pack_suspension(rods, L, rng, h_gen=0.1)
    # squeeze towards the box centre so that rods overlap, no periodic wrap
    c = pos.reshape(6, 5, 3).mean(axis=1)
    shift = 0.25 * (L / 2 - c)
    pos = (pos.reshape(6, 5, 3) + shift[:, None, :]).reshape(-1, 3)
    out, fb = C.hertz_contact(pos, body, L, 1e3)
    assert np.abs(fb).max() > 0
    unw, X, r = F.body_geometry(pos, body, L)
    assert np.abs(out[:, :3].sum(axis=0)).max() < 1e-9 * np.abs(out).max()
    tot = (np.cross(X, out[:, :3]) + out[:, 3:]).sum(axis=0)
    assert np.abs(tot).max() < 1e-9 * np.abs(out).max() * L


def test_no_force_without_overlap_or_within_a_body():
    pos, body, L = synth.config_doublets(8, 30.0, seed=2)  # gaps >= 0.1a, touching within doublets
    out, fb = C.hertz_contact(pos, body, L, 1e4)
    assert np.all(out == 0.0)
    # overlapping beads of one body exert nothing
    pos2 = np.array([[1.0, 1.0, 1.0], [2.5, 1.0, 1.0]])
    out2, _ = C.hertz_contact(pos2, np.array([0, 0]), 10.0, 1e4)
    assert np.all(out2 == 0.0)


def test_rod_generator():
    pos, body, L = synth.rod_suspension(20, 8, 0.01, seed=3)
    assert len(pos) == 160 and abs(20 * 8 * 4.18879 / L ** 3 - 0.01) < 1e-4
    for J in range(20):
        P = pos[body == J]
        d = np.linalg.norm(np.diff(P, axis=0), axis=1)
        assert np.allclose(d, 2.0, atol=1e-12)
        u = (P[-1] - P[0]) / np.linalg.norm(P[-1] - P[0])
        assert np.allclose(np.cross(P - P[0], u), 0.0, atol=1e-10)  # straight
    out, _ = C.hertz_contact(pos, body, L, 1e4)
    assert np.all(out == 0.0)  # inserted with gaps >= 0.1a


# ------------------------------------------------------------------ DLVO


def test_dlvo_force_is_minus_the_potential_derivative():
    # both parts, with the van der Waals regularisation, away from contact
    a, AH, Z, kappa, hc = 1.0, 15.0, 4.0, 1.0, 0.03
    for r in (2.01, 2.1, 2.5, 3.3, 5.0):
        e = 1e-6 * r
        fd = -(C.dlvo_potential(r + e, a, AH, Z, kappa, hc)
               - C.dlvo_potential(r - e, a, AH, Z, kappa, hc)) / (2 * e)
        f = C.dlvo_force_scalar(r, a, AH, Z, kappa, hc)
        assert abs(f - fd) < 1e-6 * max(abs(fd), 1e-3)


def test_van_der_waals_far_field_is_the_textbook_sphere_limit():
    # two equal spheres far apart: V -> -(16/9) A_H a^6 / r^6 (the leading
    # term of the Hamaker sphere-sphere energy); corrections O((2a/r)^2)
    # (a radius other than 1 separates 2 a1 a2 from the printed 2 a1 a2^2)
    AH = 15.0
    for a in (1.0, 1.7):
        for r in (40.0 * a, 80.0 * a):
            v = C.dlvo_potential(r, a, AH, 0.0, 1.0, 0.0)
            ref = -16.0 / 9.0 * AH * a ** 6 / r ** 6
            assert abs(v / ref - 1.0) < 40.0 * (2 * a / r) ** 2


def test_double_layer_screening_and_contact_value():
    # two radii, so that a and a^2 cannot stand in for each other
    for a in (1.0, 1.7):
        Z, kappa = 4.0, 2.0
        v0 = C.dlvo_potential(2.0 * a, a, 0.0, Z, kappa, 0.0)
        assert abs(v0 - a * a / (2 * a) * Z) < 1e-14 * max(1.0, abs(v0))
        v1 = C.dlvo_potential(2.0 * a + 1.0 / kappa, a, 0.0, Z, kappa, 0.0)
        assert abs(v1 / v0 - (2 * a / (2 * a + 1.0 / kappa)) * np.exp(-1.0)) < 1e-14


def test_van_der_waals_attraction_capped_under_overlap_and_finite_at_contact():
    a, AH, hc = 1.0, 15.0, 0.03
    f_contact = C.dlvo_force_scalar(2.0 * a, a, AH, 0.0, 1.0, hc)
    assert np.isfinite(f_contact) and f_contact < 0.0  # attractive
    for r in (1.99, 1.95, 1.9):
        assert C.dlvo_force_scalar(r, a, AH, 0.0, 1.0, hc) == f_contact
    # the attraction grows towards contact
    assert abs(C.dlvo_force_scalar(2.2, a, AH, 0.0, 1.0, hc)) < abs(f_contact)


def test_dlvo_and_hertz_newton_third_law_cutoff_and_intrabody():
    pos, body, L = synth.suspension(6, 4, 0.15, 3)
    pos, body, L = C.F.body_geometry(pos, body, L)[0] + L, np.asarray(body), 3.0 * L
    # (unwrapped aggregates in the middle of a box three times larger: no
    # pair acts across the periodic boundary, so torques about one origin
    # must cancel)
    kw = dict(kn=1e3, A_H=15.0, Z=4.0, kappa=1.0, h_c=0.03, r_cut=4.0)
    ft, fb = C.pair_forces(pos, body, L, **kw)
    assert np.abs(fb).max() > 0
    unw, X, r = O.body_geometry(pos, body, L)
    assert np.abs(ft[:, :3].sum(axis=0)).max() < 1e-10 * np.abs(ft).max()
    tot = ft[:, 3:].sum(axis=0) + np.cross(X, ft[:, :3]).sum(axis=0)
    assert np.abs(tot).max() < 1e-9 * np.abs(ft).max() * L
    # nothing beyond the cut-off (r_cut below every inter-body distance)
    d = O.min_image(unw[:, None] - unw[None], L)
    dist = np.linalg.norm(d, axis=-1)
    inter = np.asarray(body)[:, None] != np.asarray(body)[None]
    rmin = dist[inter].min()
    ft0, fb0 = C.pair_forces(pos, body, L, A_H=15.0, Z=4.0, kappa=1.0, r_cut=0.99 * rmin)
    assert np.abs(fb0).max() == 0.0
    # a single aggregate feels nothing from itself
    one = np.zeros(len(pos), dtype=int)
    _, fb1 = C.pair_forces(pos, one, L, **kw)
    assert np.abs(fb1).max() == 0.0
