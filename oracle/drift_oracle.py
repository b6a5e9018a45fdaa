"""Brownian drift and Brownian stresslet of the rigid-aggregate solve, as plain
FP64 definitions.

TEST INFRASTRUCTURE ONLY: imported by tests/ (and nothing in the product
path).  It uses fsd_oracle's dense solve and brownian_oracle's Brownian solve
and shares no code with the CUDA library.

What it computes (paper: Sec. 2.4 "Brownian drift"; appendix "Brownian
drift": Eq. rfd, the centred differences after it, and the modified Fixman
midpoint scheme):

* random finite differences (RFD): for a Gaussian body vector dq [N][6]
  (translation, rotation), solve the saddle-point system at the displaced
  configurations x +- (eps/2) dq with zero background flow and the body
  forcing dq (right-hand side (0; -dq)); U+-, S+- are the body velocities and
  hydrodynamic stresslets there, and
      U_drift = kT (U+ - U-) / eps,   S^B = kT (S+ - S-) / eps;
* modified Fixman: with the Brownian terms (u^B, F^B_nf) sampled at x, solve
  the Brownian system (Eq. SP2 with no deterministic forcing) at x -> U0, S0;
  move to x' = x + (dt/m) U0; solve the same system (same u^B, F^B_nf) at x'
  -> U', S'; then
      U_drift = (m/2) (U' - U0),   S^B = -(m/2) (S' - S0).

Readings (paper silent or garbled):
* a rigid configuration moves by h v (v [N][6]: translation, rotation
  vector) as X += h v_t and lever arms rotated by the unit quaternion
  normalise(1, (h/2) v_w), i.e. the Euler quaternion step of Eq. EM2 with
  Omega dt = h v_w: a rotation about v_w by 2 atan(h |v_w| / 2).  The two
  RFD displacements are exact mirror images, so the centred difference keeps
  its O(eps^2) truncation;
* S+- are each taken at their own configuration (the paper writes
  x + eps/2 in both);
* the stresslet that is differenced is the hydrodynamic one,
  S^ff - R_SU^nf Sigma^T U (no constraint part): the paper's S+-, S0, S';
* the Fixman right-hand side has no shear (E^inf = 0) and no applied force.

Pins (tests/test_oracle_drift.py): the displacement is a rigid motion whose
first-order part is h (v_t + v_w x r); the RFD summed over the basis vectors
of dq equals the divergence of the body mobility from central differences
with exact (Rodrigues) rotations, velocity and stresslet; a lone body has no
translational drift; the Fixman drift at large m is (dt/2) times the
derivative of the Brownian solve along U0 (exact-rotation central
differences), velocity and stresslet.  The Fixman drift summed over the
Brownian noise's basis vectors does not reproduce the divergence for this
formulation (the slip, not the aggregate force, is held fixed at x'); that
is a property of the scheme as printed, measured, not pinned.
"""

import numpy as np

from . import brownian_oracle as B
from . import fsd_oracle as F


def displaced(pos, body, L, v, h, tilt=0.0):
    """Bead positions of the rigid configuration moved by h v (see the
    reading in the module docstring); positions are returned unwrapped.
    tilt: the Lees-Edwards offset of the box (0: cubic)."""
    body = np.asarray(body)
    unw, X, r = F.body_geometry(pos, body, L, tilt)
    v = np.asarray(v, dtype=np.float64).reshape(-1, 6)
    q = np.concatenate([np.ones((len(v), 1)), 0.5 * h * v[:, 3:6]], axis=1)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    R = F.quat_to_matrix(q)
    Xn = X + h * v[:, 0:3]
    return Xn[body] + np.einsum("bij,bj->bi", R[body], r)


def rfd(pos, body, L, dq, eps, kT=1.0, rlub=3.0, a=1.0, eta=1.0, hmin=1e-3, tilt=0.0):
    """(U_drift [N][6], S^B [N][3][3], (out+, out-)) by random finite
    differences with the given dq."""
    dq = np.asarray(dq, dtype=np.float64).reshape(-1, 6)
    outs = []
    for s in (1.0, -1.0):
        p = displaced(pos, body, L, dq, 0.5 * s * eps, tilt)
        outs.append(F.solve(p, body, L, gamma=0.0, FT=dq, a=a, eta=eta, rlub=rlub, hmin=hmin,
                            tilt=tilt))
    up, um = outs
    return kT * (up["U"] - um["U"]) / eps, kT * (up["SH"] - um["SH"]) / eps, outs


def fixman(pos, body, L, uB, fB, dt, m, rlub=3.0, a=1.0, eta=1.0, hmin=1e-3):
    """(U0, U_drift, S^B, S0) of the modified Fixman scheme for the given
    Brownian terms (already scaled by sqrt(2 kT/dt))."""
    o0 = B.solve_brownian(pos, body, L, uB, fB, gamma=0.0, rlub=rlub, a=a, eta=eta, hmin=hmin)
    p1 = displaced(pos, body, L, o0["U"], dt / m)
    o1 = B.solve_brownian(p1, body, L, uB, fB, gamma=0.0, rlub=rlub, a=a, eta=eta, hmin=hmin)
    return o0["U"], 0.5 * m * (o1["U"] - o0["U"]), -0.5 * m * (o1["SH"] - o0["SH"]), o0["SH"]
