"""GPU parity of the interparticle physics of Sec. 4 against the oracle,
through the C ABI:

* fsd_interparticle_forces: Hertz contact plus DLVO (van der Waals
  attraction regularised by h_c and capped under overlap, screened double
  layer) between beads of different aggregates, summed per aggregate; in the
  cube and in a Lees-Edwards box.  FP64 on both sides with the same pair
  rule: relative 1e-12.
* surface roughness of the lubrication pairs (Eq. tan_fric, rough_alpha /
  rough_h0): the near-field operator RR_FU^nf (1e-12) and the FP64 solve
  (1e-6 on U, Omega and S at GMRES 1e-10, x_err 1e-8) against the oracle
  with the same roughness."""

import numpy as np
import pytest

import oracle as O
import synth
from oracle import contact_oracle as C

pytestmark = pytest.mark.gpu

DLVO = dict(kn=2.5e3, hamaker=15.0, zeta=4.0, kappa=1.0, h_c=0.03, r_cut=5.0)


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g

    g.build()
    import paper_2607_25161_gb300 as p

    return p


def squeezed_aggregates(seed=6, n=10, nb=4, L=30.0, squeeze=0.55):
    """Aggregates pushed towards the box centre: some overlapping bead pairs
    (Hertz) and many within the DLVO cut-off."""
    rng = np.random.default_rng(seed)
    shapes = [synth.random_attachment_aggregate(nb, rng) for _ in range(n)]
    pos, body = synth.pack_suspension(shapes, L, rng, h_gen=0.1)
    c = pos.reshape(n, nb, 3).mean(axis=1)
    pos = (pos.reshape(n, nb, 3) + squeeze * (L / 2 - c)[:, None, :]).reshape(-1, 3)
    return pos, body, L


@pytest.mark.parametrize("tilt_frac", [0.0, 0.31])
def test_hertz_and_dlvo_forces_match_oracle(pkg, tilt_frac):
    pos, body, L = squeezed_aggregates()
    tilt = tilt_frac * L
    ref, fb = C.pair_forces(pos, body, L, kn=DLVO["kn"], A_H=DLVO["hamaker"], Z=DLVO["zeta"],
                            kappa=DLVO["kappa"], h_c=DLVO["h_c"], r_cut=DLVO["r_cut"], tilt=tilt)
    d = O.min_image(pos[:, None] - pos[None], L, tilt)
    dist = np.linalg.norm(d, axis=-1)
    inter = body[:, None] != body[None]
    assert (dist[inter] < 2.0).any()  # overlaps: the capped attraction and Hertz
    s = pkg.Suspension(pos, body, L, xi=0.6, lub_cutoff=3.0, tilt=tilt)
    ft = s.interparticle(**DLVO)
    s.close()
    assert np.abs(ref).max() > 0
    assert np.linalg.norm(ft - ref) <= 1e-12 * np.linalg.norm(ref)


def test_each_part_of_the_pair_force(pkg):
    # van der Waals only, double layer only, Hertz only: each against the oracle
    pos, body, L = squeezed_aggregates(seed=7)
    s = pkg.Suspension(pos, body, L, xi=0.6, lub_cutoff=3.0)
    for kw in (dict(hamaker=15.0, h_c=0.03, r_cut=4.5), dict(zeta=4.0, kappa=2.0, r_cut=4.5),
               dict(kn=1e3)):
        ft = s.interparticle(**kw)
        ref, _ = C.pair_forces(pos, body, L, kn=kw.get("kn", 0.0), A_H=kw.get("hamaker", 0.0),
                               Z=kw.get("zeta", 0.0), kappa=kw.get("kappa", 1.0), h_c=kw.get("h_c", 0.0),
                               r_cut=kw.get("r_cut", 0.0))
        assert np.abs(ref).max() > 0
        assert np.linalg.norm(ft - ref) <= 1e-12 * np.linalg.norm(ref)
    s.close()


def test_interparticle_invalid_arguments(pkg):
    pos, body, L = squeezed_aggregates()
    s = pkg.Suspension(pos, body, L, xi=0.6, lub_cutoff=3.0)
    rc = s.params["rc"]
    with pytest.raises(pkg.FsdError):
        s.interparticle(hamaker=1.0, r_cut=rc + 1.0)  # beyond the neighbour lists
    with pytest.raises(pkg.FsdError):
        s.interparticle(zeta=1.0, kappa=0.0, r_cut=3.0)
    with pytest.raises(pkg.FsdError):
        s.interparticle(kn=-1.0)
    s.close()


ROUGH = dict(rough_alpha=0.05, rough_h0=0.2)
HI = dict(xi=1.2, P=12, xerr=1e-8, tol=1e-10, lub_cutoff=3.0)


def rough_system():
    """Doublets and a single bead with surface gaps 0.03a, 0.1a and 0.14a
    (inside the asperity height) plus a 3-bead aggregate further away."""
    pos = np.array([[3.0, 3.0, 3.0], [5.0, 3.0, 3.0],        # A
                    [7.03, 3.0, 3.0], [9.03, 3.0, 3.0],      # B: gap 0.03 to A
                    [5.5, 5.08, 3.0], [5.5, 7.08, 3.0],      # C: gap ~0.14 to A
                    [10.0, 10.0, 10.0], [12.0, 10.0, 10.0], [10.0, 12.0, 10.0],  # D
                    [3.0, 3.0, 5.1]])                        # E: gap 0.1 to A
    body = np.array([0, 0, 1, 1, 2, 2, 3, 3, 3, 4], dtype=np.int32)
    return pos, body, 14.0


def test_rough_lubrication_operator_and_solve_match_oracle(pkg):
    pos, body, L = rough_system()
    unw, X, r = O.body_geometry(pos, body, L)
    d = O.min_image(unw[:, None] - unw[None], L)
    gap = np.linalg.norm(d, axis=-1) - 2.0
    inter = np.asarray(body)[:, None] != np.asarray(body)[None]
    assert (gap[inter] < ROUGH["rough_h0"]).any()  # pairs inside the asperity height
    ft = synth.random_forces(int(body.max()) + 1, 5)
    sysd = O.assemble(pos, body, L, gamma=1.0, FT=ft, rlub=3.0, rough=(0.05, 0.2))
    smooth = O.assemble(pos, body, L, gamma=1.0, FT=ft, rlub=3.0, M=sysd["M"])
    assert rel(sysd["RRFU"], smooth["RRFU"]) > 1e-3  # the roughness matters here
    s = pkg.Suspension(pos, body, L, **HI, **ROUGH)
    rng = np.random.default_rng(9)
    dU = rng.normal(size=(sysd["nb"], 6))
    ref = (sysd["RRFU"] @ dU.reshape(-1)).reshape(-1, 6)
    assert rel(s.apply_lubrication(dU, 0), ref) < 1e-12
    sysd["body"] = np.asarray(body)
    out = O.outputs(sysd, np.linalg.solve(sysd["A"], sysd["b"]))
    vel, S, st, status = s.solve(ft, 1.0)
    s.close()
    assert rel(vel[:, :3], out["U"][:, :3]) < 1e-6
    assert rel(vel[:, 3:], out["U"][:, 3:]) < 1e-6
    assert rel(S, out["S"]) < 1e-6


def test_roughness_parameters_are_checked(pkg):
    pos, body, L = rough_system()
    with pytest.raises(pkg.FsdError):
        pkg.Suspension(pos, body, L, rough_alpha=0.01, rough_h0=0.0)
    with pytest.raises(pkg.FsdError):
        pkg.Suspension(pos, body, L, rough_alpha=-0.01, rough_h0=0.01)
