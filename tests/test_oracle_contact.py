"""Pins of the Hertz contact oracle (oracle/contact_oracle.py; Sec. 4 normal
contact F_N = k_n delta^1.5 n): the closed form for one overlapping pair,
Newton's third law with central forces (forces and torques about a common
origin sum to zero), nothing without overlap or within one aggregate."""

import numpy as np

import synth
from oracle import contact_oracle as C
from oracle import fsd_oracle as F


def test_single_pair_closed_form():
    L, kn, delta = 30.0, 1e4, 0.03
    d = np.array([1.0, 2.0, -2.0]) / 3.0
    pos = np.array([[5.0, 5.0, 5.0], [5.0, 5.0, 5.0] + (2.0 - delta) * d])
    out, fb = C.hertz_contact(pos, np.array([0, 1]), L, kn)
    f = kn * delta ** 1.5
    assert np.allclose(fb[1], f * d, rtol=1e-12) and np.allclose(fb[0], -f * d, rtol=1e-12)
    assert np.allclose(out[:, 3:], 0.0, atol=1e-12)  # single beads: no lever arm


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
