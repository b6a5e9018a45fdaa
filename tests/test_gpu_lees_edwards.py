"""GPU parity of the Lees-Edwards (sheared periodic) box against the oracle's
sheared lattice (images at n1 e1 + n2 e2 + n3 e3, e2 = (tilt, L, 0);
reciprocal vectors (2 pi/L)(n1, n2 - tilt/L n1, n3)), through the C ABI.

Tolerances (relative L2) as for the cubic box: FP64 1e-6 at x_err = 1e-8,
P = 16, GMRES 1e-10; the FP32 operator (mixed) 1e-5."""

import numpy as np
import pytest

import oracle as O
import synth
from oracle import brownian_oracle as BO
from oracle import contact_oracle as C

pytestmark = pytest.mark.gpu

FP64, MIXED = 0, 1
HI = dict(xi=1.2, P=16, xerr=1e-8, tol=1e-10)


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g

    g.build()
    import paper_2607_25161_gb300 as p

    return p


@pytest.fixture(scope="module")
def sysLE():
    rng = np.random.default_rng(12)
    sizes = [1, 2, 3, 4, 2, 3]
    shapes = [synth.random_attachment_aggregate(n, rng) for n in sizes]
    L = 14.0
    pos, body = synth.pack_suspension(shapes, L, rng, h_gen=0.05)
    return pos, body, L


@pytest.mark.parametrize("tilt_frac", [0.3, -0.45])
@pytest.mark.parametrize("prec,tol", [(FP64, 1e-6), (MIXED, 1e-5)])
def test_mobility_matches_oracle_with_tilt(pkg, sysLE, tilt_frac, prec, tol):
    pos, body, L = sysLE
    tilt = tilt_frac * L
    rng = np.random.default_rng(3)
    F = rng.normal(size=(len(pos), 11))
    unw, X, r = O.body_geometry(pos, body, L, tilt)
    ref = O.mobility_dense(unw, L, tilt=tilt) @ F.reshape(-1)
    s = pkg.Suspension(pos, body, L, tilt=tilt, **HI)
    assert abs(s.params["tilt"] - tilt) < 1e-12
    u = s.apply_mobility(F, part=3, precision=prec)
    s.close()
    assert rel(u.reshape(-1), ref) < tol


def test_tilt_modulo_L_and_set_tilt(pkg, sysLE):
    pos, body, L = sysLE
    rng = np.random.default_rng(4)
    F = rng.normal(size=(len(pos), 11))
    a = pkg.Suspension(pos, body, L, tilt=0.3 * L, **HI)
    ua = a.apply_mobility(F, part=3)
    a.close()
    b = pkg.Suspension(pos, body, L, **HI)
    u0 = b.apply_mobility(F, part=3)
    b.set_tilt(-0.7 * L)
    assert abs(b.params["tilt"] - 0.3 * L) < 1e-12
    ub = b.apply_mobility(F, part=3)
    b.close()
    assert rel(ub, ua) < 1e-12
    assert rel(ua, u0) > 1e-4


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-6), (MIXED, 1e-5)])
def test_solve_matches_oracle_with_tilt(pkg, sysLE, prec, tol):
    pos, body, L = sysLE
    tilt = -0.37 * L
    ft = synth.random_forces(body.max() + 1, 5)
    ref = O.solve(pos, body, L, gamma=0.7, FT=ft, rlub=3.0, tilt=tilt)
    s = pkg.Suspension(pos, body, L, tilt=tilt, precision=prec, lub_cutoff=3.0, **HI)
    vel, S, st, status = s.solve(ft, 0.7)
    s.close()
    assert status == pkg.FSD_OK
    assert rel(vel, ref["U"]) < tol
    assert rel(S, ref["S"]) < tol


def test_lees_edwards_step_advances_the_box(pkg, sysLE):
    pos, body, L = sysLE
    gamma, dt = 0.8, 0.05
    s = pkg.Suspension(pos, body, L, flags=pkg.FSD_FLAG_LEES_EDWARDS, lub_cutoff=3.0, **HI)
    vel, _, _, _ = s.solve(None, gamma)
    p0, q0 = s.beads()
    s.step(None, gamma, dt)
    p1, q1 = s.beads()
    tilt1 = s.params["tilt"]
    for _ in range(9):
        s.step(None, gamma, dt)
    tilt10 = s.params["tilt"]
    s.close()
    wrap = lambda t: t - L * np.floor(t / L + 0.5)  # noqa: E731
    assert abs(tilt1 - wrap(gamma * L * dt)) < 1e-12
    assert abs(tilt10 - wrap(10 * gamma * L * dt)) < 1e-10
    # one step: every body moved rigidly by its full (lab-frame) velocity;
    # the centroids are those the library took from the set-up positions
    # (U_inf = gamma X_y depends on which periodic image X is)
    unw, X, r = O.body_geometry(pos, body, L, 0.0)
    N = body.max() + 1
    q = np.tile([1.0, 0.0, 0.0, 0.0], (N, 1))
    _, _, x1 = O.integrate(X, q, r, body, vel, dt)
    d = O.min_image(p1 - x1, L, tilt1)
    assert np.abs(d).max() < 1e-10


def test_contact_with_tilt(pkg):
    L, tilt = 20.0, 0.31 * 20.0
    # bead 1 is bead 0's neighbour through the sheared y boundary
    pos = np.array([[3.0, 0.4, 5.0], [3.0 + tilt - 0.5, L - 1.3, 5.0], [12.0, 10.0, 12.0]])
    body = np.array([0, 1, 2])
    ref, fb = C.hertz_contact(pos, body, L, 50.0, tilt=tilt)
    assert np.abs(fb).max() > 0
    s = pkg.Suspension(pos, body, L, xi=0.8, tilt=tilt)
    ft = s.contact(50.0)
    s.close()
    assert rel(ft, ref) < 1e-12


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-6), (MIXED, 1e-5)])
def test_brownian_slip_with_tilt(pkg, sysLE, prec, tol):
    # analytic wave part on the sheared reciprocal lattice + Lanczos square
    # root of the sheared real-space part, against the dense oracle
    pos, body, L = sysLE
    tilt = 0.27 * L
    s = pkg.Suspension(pos, body, L, tilt=tilt, precision=prec, nf_sampler=pkg.FSD_NF_LANCZOS, **HI)
    prm = s.params
    n, xi = prm["grid"], prm["xi"]
    rng = np.random.default_rng(17)
    field = BO.hermitian_field(n, rng)
    psi_r = rng.normal(size=(len(pos), 11))
    slip, _, st = s.brownian(1.0, 1.0, wave_field=field, psi_real=psi_r,
                             psi_nf=np.zeros((len(pos), 6)))
    s.close()
    unw, X, r = O.body_geometry(pos, body, L, tilt)
    uw = BO.brownian_wave_slip(unw, L, xi, n, field, tilt=tilt)
    rc = 2.0 + np.sqrt(46.0) / xi
    Mr = O.mobility_real_dense(unw, L, xi, rc, tilt=tilt).reshape(11 * len(pos), -1)
    ur = BO.sqrtm_apply(Mr, psi_r.reshape(-1)).reshape(-1, 11)
    assert rel(slip / np.sqrt(2.0), uw + ur) < tol
    # the tilt matters for the sample
    uw0 = BO.brownian_wave_slip(unw, L, xi, n, field)
    assert rel(uw0, uw) > 1e-3


def test_batch_lees_edwards_steps_match_single(pkg, sysLE):
    pos, body, L = sysLE
    rng = np.random.default_rng(8)
    shapes = [synth.random_attachment_aggregate(k, rng) for k in (2, 3, 2)]
    L2 = 15.0
    pos2, body2 = synth.pack_suspension(shapes, L2, rng, h_gen=0.05)
    prm = dict(flags=pkg.FSD_FLAG_LEES_EDWARDS, lub_cutoff=3.0, tilt=0.1 * L, **HI)
    prm2 = dict(prm, tilt=-0.2 * L2)
    B = pkg.Batch([(pos, body, L), (pos2, body2, L2)], params=[prm, prm2])
    rates = np.array([0.6, -0.9])
    for _ in range(3):
        B.step(None, rates, 0.02)
    pb, qb = B.beads()
    tilts = [B.system(k).params["tilt"] for k in range(2)]
    B.close()
    ref_p, ref_t = [], []
    for (p, b, Lk), kw, g in (((pos, body, L), prm, 0.6), ((pos2, body2, L2), prm2, -0.9)):
        s = pkg.Suspension(p, b, Lk, **kw)
        for _ in range(3):
            s.step(None, g, 0.02)
        ref_p.append(s.beads()[0])
        ref_t.append(s.params["tilt"])
        s.close()
    assert np.allclose(tilts, ref_t, rtol=0, atol=1e-12)
    assert abs(ref_t[0] - (0.1 * L + 3 * 0.6 * L * 0.02)) < 1e-12
    assert np.allclose(pb, np.concatenate(ref_p), rtol=0, atol=1e-9)


def test_rfd_drift_with_tilt(pkg, sysLE):
    # random finite differences in the sheared box: the displaced
    # configurations are wrapped with the sheared images on both sides
    from oracle import drift_oracle as DO

    pos, body, L = sysLE
    tilt = 0.33 * L
    dq = np.random.default_rng(21).normal(size=(body.max() + 1, 6))
    ref, refS, _ = DO.rfd(pos, body, L, dq, 0.05, kT=0.7, rlub=3.0, tilt=tilt)
    s = pkg.Suspension(pos, body, L, tilt=tilt, lub_cutoff=3.0, **HI)
    drift, _, SB, _, status = s.drift(pkg.FSD_DRIFT_RFD, 0.7, param=0.05, dq=dq)
    s.close()
    assert status == pkg.FSD_OK
    assert rel(drift, ref) < 1e-5
    assert rel(SB, refS) < 1e-5


def test_pairwise_near_field_sampler_with_tilt(pkg):
    # three lubrication pairs exist only through the sheared image across y
    # (bead B sits at A + d + (tilt, L, 0)); the pairwise sampler's forces
    # and torques must follow the sheared nearest image, as in the oracle
    L, tilt = 14.0, 0.3 * 14.0
    A = np.array([5.0, 0.3, 7.0])
    d = np.array([0.5, -2.2, 0.3])
    B = A + d + np.array([tilt, L, 0.0])
    B[0] = np.mod(B[0], L)
    pos = np.array([A, A + [0.0, 0.0, 2.0], B, B + [0.0, 0.0, 2.0], [10.0, 7.0, 3.0],
                    [2.0, 7.0, 12.0]])
    body = np.array([0, 0, 1, 1, 2, 3], dtype=np.int32)
    seed, step = 91, 3
    s = pkg.Suspension(pos, body, L, tilt=tilt, lub_cutoff=3.0, nf_sampler=pkg.FSD_NF_PAIRWISE,
                       **HI)
    _, fnf, st = s.brownian(1.0, 1.0, seed=seed, step=step, psi_real=np.zeros((len(pos), 11)))
    s.close()
    unw, X, r = O.body_geometry(pos, body, L, tilt)
    ref = BO.pairwise_nf_force(unw, body, L, seed, step, rlub=3.0, tilt=tilt)
    assert np.abs(ref[:4]).max() > 0 and np.abs(ref[4:]).max() == 0.0
    # in the cube the same beads have no near pairs at all
    assert np.abs(BO.pairwise_nf_force(unw, body, L, seed, step, rlub=3.0)).max() == 0.0
    assert rel(fnf / np.sqrt(2.0), ref) < 1e-12


def straddling_system():
    """Aggregates whose lubrication pairs exist only through the sheared image
    across y (at tilt 0.2 L), plus two free aggregates."""
    L, tilt = 14.0, 0.2 * 14.0
    A = np.array([5.0, 0.4, 7.0])
    B = A + np.array([0.5, -2.25, 0.3]) + np.array([tilt, L, 0.0])
    B[0] = np.mod(B[0], L)
    C = np.array([9.0, 13.5, 2.0])
    D = C + np.array([-0.4, 2.3, 0.2]) - np.array([tilt, L, 0.0])
    D[0] = np.mod(D[0], L)
    pos = np.array([A, A + [0.0, 0.0, 2.0], B, B + [2.0, 0.0, 0.0], C, C + [0.0, 0.0, 2.0], D,
                    [2.0, 7.0, 3.0], [4.0, 7.0, 3.0], [11.0, 6.0, 11.0]])
    body = np.array([0, 0, 1, 1, 2, 2, 3, 4, 4, 5], dtype=np.int32)
    return pos, body, L


@pytest.mark.parametrize("system", ["packed", "straddling"])
@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_graph_lees_edwards_steps_match_host_driven(pkg, sysLE, prec, system):
    # with FSD_FLAG_GRAPH a Lees-Edwards step is one captured graph whose
    # kernels read the box offset from device memory (one graph for every
    # offset); five steps must reproduce the host-driven loop's velocities,
    # beads, orientations and offsets, also with lubrication pairs that
    # exist only across the sheared boundary (every kernel of the graph must
    # take the current offset, not the one at capture)
    pos, body, L = sysLE if system == "packed" else straddling_system()
    gamma, dt = 0.7, 0.04
    out = []
    for flags in (pkg.FSD_FLAG_LEES_EDWARDS, pkg.FSD_FLAG_LEES_EDWARDS | pkg.FSD_FLAG_GRAPH):
        s = pkg.Suspension(pos, body, L, flags=flags, lub_cutoff=3.0, tilt=0.2 * L, precision=prec,
                           **HI)
        vels, tilts = [], []
        for _ in range(5):
            vel = np.zeros((body.max() + 1, 6))
            s.step(None, gamma, dt, vel=vel)
            vels.append(vel)
            tilts.append(s.params["tilt"])
        p, q = s.beads()
        s.close()
        out.append((np.array(vels), np.array(tilts), p, q))
    (v0, t0, p0, q0), (v1, t1, p1, q1) = out
    assert np.allclose(t1, t0, rtol=0, atol=1e-12)
    assert abs(t0[0] - (0.2 * L + gamma * L * dt)) < 1e-12
    assert rel(v1, v0) < 1e-9
    assert np.allclose(p1, p0, rtol=0, atol=1e-9)
    assert np.allclose(q1, q0, rtol=0, atol=1e-12)
