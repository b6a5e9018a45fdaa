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

DLVO forces (Sec. 4, Eq. dlvo_potential and F = -grad V): between beads of
different aggregates with centre distance r < r_cut, the van der Waals
attraction of two spheres plus the screened double-layer repulsion
    V(r) = -(A_H/6) [2 a1 a2/(r^2 - (a1+a2)^2) + 2 a1 a2/(r^2 - (a1-a2)^2)
                     + ln((r^2 - (a1+a2)^2)/(r^2 - (a1-a2)^2))]
           + (a1 a2 / r) Z exp(-kappa (r - a1 - a2))
(the paper prints the first numerator as 2 a1 a2^2, which is not
dimensionless; the sphere-sphere Hamaker expression has 2 a1 a2).  The van
der Waals part is regularised by h -> h + h_c (h = r - a1 - a2, i.e. it is
evaluated at r + h_c), and for overlapping beads (h < 0) its force is held at
its value at contact.  Z is the double-layer strength in energy per length
(Z a1 a2 / r is an energy).

Pins (tests/test_oracle_contact.py): one overlapping pair gives the closed
form; forces and torques about a common origin sum to zero (Newton's third
law, central forces); no force without overlap; intra-aggregate overlaps
give none.  DLVO: the force is minus the derivative of the potential
(central differences); far from contact the van der Waals energy tends to
the textbook -(16/9) A_H a^6 / r^6 of two equal spheres; the attraction is
constant under overlap and finite at contact with h_c > 0; the screened
repulsion falls by e^-1 per Debye length beyond the a1 a2 / r factor;
Newton's third law for the aggregate sums; nothing beyond r_cut or within
one aggregate.
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


def dlvo_potential(r, a, A_H, Z, kappa, h_c=0.0):
    """V_vdW(r + h_c) + V_el(r) for two beads of radius a (Eq. dlvo_potential
    with a1 = a2 = a; the regularisation h -> h + h_c on the van der Waals
    part); r > 2a - h_c."""
    rv = r + h_c
    s2 = (2.0 * a) ** 2
    vdw = 0.0
    if A_H != 0.0:
        vdw = -A_H / 6.0 * (2.0 * a * a / (rv * rv - s2) + 2.0 * a * a / (rv * rv)
                            + np.log((rv * rv - s2) / (rv * rv)))
    el = a * a / r * Z * np.exp(-kappa * (r - 2.0 * a))
    return vdw + el


def dlvo_force_scalar(r, a, A_H, Z, kappa, h_c=0.0):
    """f(r) = -dV/dr (positive: repulsive) with the van der Waals part held at
    its contact value for r < 2a (overlap)."""
    dvdw = 0.0
    if A_H != 0.0:
        rv = max(r, 2.0 * a) + h_c
        s2 = (2.0 * a) ** 2
        # d/dr of the three van der Waals terms at rv
        d1 = -2.0 * a * a * 2.0 * rv / (rv * rv - s2) ** 2
        d2 = -2.0 * a * a * 2.0 / rv ** 3
        d3 = 2.0 * rv / (rv * rv - s2) - 2.0 / rv
        dvdw = -A_H / 6.0 * (d1 + d2 + d3)
    e = np.exp(-kappa * (r - 2.0 * a))
    del_ = a * a * Z * e * (-1.0 / (r * r) - kappa / r)
    return -(dvdw + del_)


def pair_forces(pos, body, L, kn=0.0, A_H=0.0, Z=0.0, kappa=1.0, h_c=0.0, r_cut=0.0, a=1.0,
                tilt=0.0):
    """(N, 6) aggregate force and torque (about X_J) from Hertz contact (kn)
    and DLVO forces (pairs with r < r_cut) between beads of different
    aggregates; also the per-bead forces (N_tot, 3)."""
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
            f = 0.0
            if kn > 0.0 and dist < 2.0 * a:
                f += kn * (2.0 * a - dist) ** 1.5
            if dist < r_cut and (A_H != 0.0 or Z != 0.0):
                f += dlvo_force_scalar(dist, a, A_H, Z, kappa, h_c)
            fb[i] += f * d / dist
            fb[j] -= f * d / dist
    nb = int(body.max()) + 1
    out = np.zeros((nb, 6))
    for b in range(Nt):
        out[body[b], :3] += fb[b]
        out[body[b], 3:] += np.cross(r[b], fb[b])
    return out, fb
