"""Pins of the drift oracle (oracle/drift_oracle.py) against what the
definitions fix (Sec. 2.4 "Brownian drift"; appendix "Brownian drift":
Eq. rfd and the modified Fixman scheme):

* the displacement of a rigid configuration is a rigid motion whose first
  order part is h (v_t + v_w x r_b);
* the RFD summed over the basis vectors of dq is the divergence of the body
  mobility, kT d_k N_ik (E[dq dq^T] = I makes the Gaussian average that
  sum), here computed by central differences with exact (Rodrigues)
  rotations and unit body forces; the same for the stresslet response;
* a lone body: the mobility does not depend on the position in the periodic
  box, so the translational RFD vanishes;
* Fixman: for large m, (m/2)(U' - U0) is (dt/2) times the derivative of the
  Brownian solve along U0, again from central differences with exact
  rotations; the stresslet likewise with the sign the paper prints;
* the RFD identity holds in a Lees-Edwards box too, where the drift differs
  from the cubic box's.
"""

import numpy as np
import pytest

import oracle as O
import synth
from oracle import brownian_oracle as B
from oracle import drift_oracle as D


def rodrigues(w):
    th = np.linalg.norm(w)
    if th == 0.0:
        return np.eye(3)
    k = w / th
    K = np.array([[0.0, -k[2], k[1]], [k[2], 0.0, -k[0]], [-k[1], k[0], 0.0]])
    return np.eye(3) + np.sin(th) * K + (1.0 - np.cos(th)) * K @ K


def moved_exact(pos, body, L, v, h, tilt=0.0):
    """Rigid motion by translation h v_t and the exact rotation by the angle
    h |v_w| about v_w, per body."""
    unw, X, r = O.body_geometry(pos, body, L, tilt)
    v = np.asarray(v).reshape(-1, 6)
    new = unw.copy()
    for J in range(len(v)):
        idx = np.asarray(body) == J
        new[idx] = X[J] + h * v[J, :3] + r[idx] @ rodrigues(h * v[J, 3:]).T
    return new


@pytest.fixture(scope="module")
def doublets():
    pos, body, L = synth.config_doublets(2, 9.0, seed=6)
    return pos, body, L


def test_displacement_is_rigid_and_first_order_right(doublets):
    pos, body, L = doublets
    rng = np.random.default_rng(1)
    v = rng.normal(size=(2, 6))
    unw, X, r = O.body_geometry(pos, body, L)
    for h in (0.3, 1e-5):
        p = D.displaced(pos, body, L, v, h)
        for J in range(2):
            idx = np.nonzero(body == J)[0]
            d0 = np.linalg.norm(unw[idx[0]] - unw[idx[1]])
            assert abs(np.linalg.norm(p[idx[0]] - p[idx[1]]) - d0) < 1e-13
            assert np.allclose(p[idx].mean(axis=0), X[J] + h * v[J, :3], atol=1e-13)
    h = 1e-5
    p = D.displaced(pos, body, L, v, h)
    lin = unw + h * (v[body, :3] + np.cross(v[body, 3:], r))
    assert np.abs(p - lin).max() < 1e-9  # O(h^2)
    assert np.abs(p - lin).max() > 0.0


def test_rfd_basis_sum_is_the_mobility_divergence(doublets):
    pos, body, L = doublets
    n6 = 12
    h, eps, kT = 1e-4, 1e-4, 0.7
    div = np.zeros(n6)
    divS = np.zeros((2, 3, 3))
    rs = np.zeros(n6)
    rS = np.zeros((2, 3, 3))
    for i in range(n6):
        e = np.eye(n6)[i].reshape(-1, 6)
        op = O.solve(moved_exact(pos, body, L, e, h), body, L, gamma=0.0, FT=e, rlub=3.0)
        om = O.solve(moved_exact(pos, body, L, e, -h), body, L, gamma=0.0, FT=e, rlub=3.0)
        div += (op["U"] - om["U"]).reshape(-1) / (2 * h)
        divS += (op["SH"] - om["SH"]) / (2 * h)
        d, s, _ = D.rfd(pos, body, L, e, eps, kT=kT, rlub=3.0)
        rs += d.reshape(-1)
        rS += s
    assert np.linalg.norm(div) > 1e-4
    assert np.linalg.norm(rs - kT * div) < 1e-6 * np.linalg.norm(kT * div)
    assert np.linalg.norm(rS - kT * divS) < 1e-6 * np.linalg.norm(kT * divS)


def test_rfd_of_a_lone_body_has_no_translational_drift():
    rng = np.random.default_rng(2)
    shape = synth.random_attachment_aggregate(5, rng)
    pos = shape + np.array([3.0, 4.0, 5.0])
    body = np.zeros(5, dtype=int)
    dq = np.array([[0.3, -1.1, 0.7, 0.0, 0.0, 0.0]])
    d, s, (up, um) = D.rfd(pos, body, 11.0, dq, 0.05, rlub=0.0)
    assert np.abs(up["U"]).max() > 1e-3
    assert np.abs(d).max() < 1e-9 * np.abs(up["U"]).max() / 0.05


def test_fixman_large_m_is_the_directional_derivative(doublets):
    pos, body, L = doublets
    Nt = len(pos)
    rng = np.random.default_rng(3)
    uB = rng.normal(size=(Nt, 11))
    fB = rng.normal(size=(Nt, 6))
    dt, m, h = 0.5, 1e5, 1e-4
    U0, drift, SB, S0 = D.fixman(pos, body, L, uB, fB, dt, m, rlub=3.0)
    ref0 = B.solve_brownian(pos, body, L, uB, fB, gamma=0.0, rlub=3.0)
    assert np.allclose(U0, ref0["U"], rtol=1e-13, atol=1e-15)
    op = B.solve_brownian(moved_exact(pos, body, L, U0, h), body, L, uB, fB, gamma=0.0, rlub=3.0)
    om = B.solve_brownian(moved_exact(pos, body, L, U0, -h), body, L, uB, fB, gamma=0.0, rlub=3.0)
    dU = 0.5 * dt * (op["U"] - om["U"]) / (2 * h)
    dS = -0.5 * dt * (op["SH"] - om["SH"]) / (2 * h)
    assert np.linalg.norm(dU) > 1e-4
    # O(dt |U0| / m) from the finite step, O(h^2) from the differences
    assert np.linalg.norm(drift - dU) < 1e-4 * np.linalg.norm(dU)
    assert np.linalg.norm(SB - dS) < 1e-4 * np.linalg.norm(dS)


def test_rfd_in_the_sheared_box():
    # the same identity in a Lees-Edwards box: the displaced configurations
    # and the solves take the sheared images
    pos, body, L = synth.config_doublets(2, 9.0, seed=6)
    tilt = 0.3 * L
    n6, h, eps, kT = 12, 1e-4, 1e-4, 1.0
    div = np.zeros(n6)
    rs = np.zeros(n6)
    for i in range(n6):
        e = np.eye(n6)[i].reshape(-1, 6)
        op = O.solve(moved_exact(pos, body, L, e, h, tilt), body, L, gamma=0.0, FT=e, rlub=3.0, tilt=tilt)
        om = O.solve(moved_exact(pos, body, L, e, -h, tilt), body, L, gamma=0.0, FT=e, rlub=3.0, tilt=tilt)
        div += (op["U"] - om["U"]).reshape(-1) / (2 * h)
        rs += D.rfd(pos, body, L, e, eps, kT=kT, rlub=3.0, tilt=tilt)[0].reshape(-1)
    assert np.linalg.norm(rs - div) < 1e-6 * np.linalg.norm(div)
    div0 = np.zeros(n6)
    for i in range(n6):
        e = np.eye(n6)[i].reshape(-1, 6)
        div0 += D.rfd(pos, body, L, e, eps, kT=kT, rlub=3.0)[0].reshape(-1)
    assert np.linalg.norm(div0 - div) > 1e-3 * np.linalg.norm(div)
