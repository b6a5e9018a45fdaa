"""Hertz normal contact between beads of different rigid aggregates, as a
plain FP64 definition.

TEST INFRASTRUCTURE ONLY: imported by tests/ (and nothing in the product
path); shares no code with the CUDA library.

What it computes (paper: Sec. 4, the normal contact force of the carbon-black
application, F_N = k_n delta^1.5 n with delta = a_1 + a_2 - r the overlap and
n the unit vector along the line of centres; the rod benchmark of Sec. 3.3
uses normal contact forces between rods): for every pair of beads i, j of
different aggregates at minimum-image distance r < 2a, bead i receives
k_n (2a - r)^1.5 (x_i - x_j)/r (repulsive) and bead j the opposite; per
aggregate J the force F_J = sum_b F_b and the torque about the centroid
T_J = sum_b r_b x F_b (r_b the lever arm of fsd_oracle.body_geometry).
Pairs of beads of one aggregate exert nothing (they are held by the rigid
constraint).

Pins (tests/test_oracle_contact.py): one overlapping pair gives the closed
form; forces and torques about a common origin sum to zero (Newton's third
law, central forces); no force without overlap; intra-aggregate overlaps
give none.
"""

import numpy as np

from . import fsd_oracle as F


def hertz_contact(pos, body, L, kn, a=1.0, tilt=0.0):
    """(N, 6) aggregate force and torque (about X_J) from Hertz contacts;
    also returns the per-bead forces (N_tot, 3).  tilt: the Lees-Edwards
    offset of the box (0: cubic)."""
    body = np.asarray(body)
    unw, X, r = F.body_geometry(pos, body, L, tilt)
    Nt = len(unw)
    fb = np.zeros((Nt, 3))
    for i in range(Nt):
        for j in range(i + 1, Nt):
            if body[i] == body[j]:
                continue
            d = F.min_image(unw[i] - unw[j], L, tilt)
            dist = np.linalg.norm(d)
            delta = 2.0 * a - dist
            if delta > 0.0:
                f = kn * delta ** 1.5 * d / dist
                fb[i] += f
                fb[j] -= f
    nb = int(body.max()) + 1
    out = np.zeros((nb, 6))
    for b in range(Nt):
        out[body[b], :3] += fb[b]
        out[body[b], 3:] += np.cross(r[b], fb[b])
    return out, fb
