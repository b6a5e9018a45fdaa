"""GPU parity of the Hertz contact forces (fsd_contact_forces; Sec. 4 normal
contact, the rod workload of Sec. 3.3) against the contact oracle, through
the C ABI.  FP64 on both sides with the same pair rule: relative 1e-12."""

import numpy as np
import pytest

import synth
from oracle import contact_oracle as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g

    g.build()
    import paper_2607_25161_gb300 as p

    return p


def squeezed_rods(seed=4, n=12, nb=6, L=40.0, squeeze=0.5):
    rng = np.random.default_rng(seed)
    pos, body = synth.pack_suspension([synth.rod(nb) for _ in range(n)], L, rng, h_gen=0.1)
    c = pos.reshape(n, nb, 3).mean(axis=1)
    pos = (pos.reshape(n, nb, 3) + squeeze * (L / 2 - c)[:, None, :]).reshape(-1, 3)
    return pos, body, L


def test_contact_matches_oracle(pkg):
    pos, body, L = squeezed_rods()
    kn = 2.5e3
    ref, fb = C.hertz_contact(pos, body, L, kn)
    assert np.count_nonzero(np.abs(fb).sum(axis=1)) >= 4
    s = pkg.Suspension(pos, body, L, xi=0.5, lub_cutoff=3.0)
    ft = s.contact(kn)
    assert np.linalg.norm(ft - ref) <= 1e-12 * np.linalg.norm(ref)
    # device output, then used as the applied force of a solve
    import torch

    d = torch.zeros((body.max() + 1, 6), dtype=torch.float64, device="cuda")
    s.contact(kn, out=d)
    torch.cuda.synchronize()
    assert np.linalg.norm(d.cpu().numpy() - ref) <= 1e-12 * np.linalg.norm(ref)
    v1, _, _, _ = s.solve(d, 0.0, allow=(pkg.FSD_OK, pkg.FSD_EOVERLAP))
    v2, _, _, _ = s.solve(ref, 0.0, allow=(pkg.FSD_OK, pkg.FSD_EOVERLAP))
    s.close()
    assert np.allclose(v1, v2, rtol=1e-12, atol=1e-14)


def test_no_overlap_gives_zero(pkg):
    pos, body, L = synth.rod_suspension(30, 8, 0.02, seed=5)
    s = pkg.Suspension(pos, body, L)
    ft = s.contact(1e4)
    s.close()
    assert np.all(ft == 0.0)


def test_contact_across_the_boundary_and_invalid(pkg):
    L = 20.0
    pos = np.array([[0.3, 4.0, 4.0], [L - 1.5, 4.0, 4.0], [10.0, 10.0, 10.0]])
    body = np.array([0, 1, 2])
    s = pkg.Suspension(pos, body, L, xi=0.8)
    ft = s.contact(10.0)
    ref, _ = C.hertz_contact(pos, body, L, 10.0)
    assert np.linalg.norm(ft - ref) <= 1e-12 * np.linalg.norm(ref)
    with pytest.raises(pkg.FsdError):
        s.contact(-1.0)
    s.close()


def test_contact_full_size_rods_balance(pkg):
    # the 8-bead rod workload at phi 0.1 squeezed by 2 %: many contacts;
    # central pair forces sum to zero, and the torques about the origin of
    # the unwrapped bodies with them
    import oracle as O

    pos, body, L = synth.rod_suspension(4096, 8, 0.10, seed=7)
    c = O.body_geometry(pos, body, L)[1]
    pos = pos + (0.98 - 1.0) * c[body]  # move the centroids inward, rigidly
    s = pkg.Suspension(pos, body, L * 0.98, xi=0.5)
    ft = s.contact(1e4)
    s.close()
    assert np.count_nonzero(np.abs(ft).sum(axis=1)) > 10
    scale = np.abs(ft[:, :3]).max()
    assert np.abs(ft[:, :3].sum(axis=0)).max() < 1e-9 * scale * len(ft)
