"""GPU parity of the Brownian drift (fsd_drift; Sec. 2.4, the appendix on the
drift: Eq. rfd and the modified Fixman scheme) against the drift oracle,
through the C ABI, on the same random inputs.

Tolerances (relative L2).  Each drift is a difference of two solves divided
by the displacement, so the operator error (~1e-8 relative at x_err = 1e-8,
P = 16) and the GMRES tolerance (1e-10) are amplified by |U| / |dU|:
  RFD with eps = 0.05:  drift and S^B 1e-5 (FP64 and mixed: the mixed path
    refines against the FP64 operator);
  Fixman with dt/m = 1e-3: U0 1e-6 FP64 / 1e-5 mixed, drift and S^B 1e-4.
"""

import numpy as np
import pytest

import oracle as O
import synth
from oracle import brownian_oracle as BO
from oracle import drift_oracle as DO

pytestmark = pytest.mark.gpu

FP64, MIXED = 0, 1
# the near-field noise these tests give is that of the Lanczos sampler
HI = dict(xi=1.2, P=16, xerr=1e-8, tol=1e-10, lub_cutoff=3.0, nf_sampler=0)


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g

    g.build()
    import paper_2607_25161_gb300 as p

    return p


@pytest.fixture(scope="module")
def sysD():
    rng = np.random.default_rng(5)
    sizes = [1, 2, 3, 5, 4, 6]
    shapes = [synth.random_attachment_aggregate(n, rng) for n in sizes]
    L = synth.box_for_phi(sum(sizes), 0.05)  # R_c = 5.6 < L/2 at xi 1.2, x_err 1e-8
    pos, body = synth.pack_suspension(shapes, L, rng, h_gen=0.05)
    dq = rng.normal(size=(len(sizes), 6))
    return dict(pos=pos, body=body, L=L, dq=dq, N=len(sizes))


@pytest.fixture(scope="module")
def rfd_ref(sysD):
    d = sysD
    drift, SB, outs = DO.rfd(d["pos"], d["body"], d["L"], d["dq"], 0.05, kT=0.7, rlub=3.0)
    return drift, SB


@pytest.mark.parametrize("prec,flags", [(FP64, 0), (MIXED, 0), (MIXED, 4)])
def test_rfd_matches_oracle(pkg, sysD, rfd_ref, prec, flags):
    d = sysD
    s = pkg.Suspension(d["pos"], d["body"], d["L"], precision=prec, flags=flags, **HI)
    ft = synth.random_forces(d["N"], 3)
    det, _, _, _ = s.solve(ft, 0.5)
    b0 = s.beads()
    drift, ub, SB, st, status = s.drift(pkg.FSD_DRIFT_RFD, 0.7, param=0.05, dq=d["dq"])
    assert status == pkg.FSD_OK
    assert rel(drift, rfd_ref[0]) < 1e-5
    assert rel(SB, rfd_ref[1]) < 1e-5
    assert st["iters"] > 0
    # the configuration is back where it was
    b1 = s.beads()
    assert np.array_equal(b0[0], b1[0]) and np.array_equal(b0[1], b1[1])
    # the next solve carries the drift, the one after does not
    v1, _, _, _ = s.solve(ft, 0.5)
    v2, _, _, _ = s.solve(ft, 0.5)
    s.close()
    assert rel(v1 - det, rfd_ref[0]) < 1e-5
    assert rel(v2, det) < 1e-8


def test_rfd_keeps_pending_brownian_terms(pkg, sysD, rfd_ref):
    d = sysD
    s = pkg.Suspension(d["pos"], d["body"], d["L"], **HI)
    Nt = len(d["pos"])
    rng = np.random.default_rng(9)
    n = s.params["grid"]
    field = BO.hermitian_field(n, rng)
    psi_r = rng.normal(size=(Nt, 11))
    psi_nf = rng.normal(size=(Nt, 6))
    kT, dt = 0.7, 0.01
    slip, fnf, _ = s.brownian(kT, dt, wave_field=field, psi_real=psi_r, psi_nf=psi_nf)
    s.drift(pkg.FSD_DRIFT_RFD, 0.7, param=0.05, dq=d["dq"])
    vel, _, _, _ = s.solve(None, 0.0)
    s.close()
    ref = BO.solve_brownian(d["pos"], d["body"], d["L"], slip, fnf, gamma=0.0, rlub=3.0)
    assert rel(vel, ref["U"] + rfd_ref[0]) < 1e-5


def test_internal_dq_matches_oracle_philox(pkg, sysD):
    d = sysD
    seed, step = 987654321, 17
    s = pkg.Suspension(d["pos"], d["body"], d["L"], **HI)
    drift, _, SB, _, _ = s.drift(pkg.FSD_DRIFT_RFD, 1.0, param=0.05, seed=seed, step=step)
    s.close()
    dq = BO.philox_psi(d["N"], seed, step, 4, 6)
    ref, refS, _ = DO.rfd(d["pos"], d["body"], d["L"], dq, 0.05, kT=1.0, rlub=3.0)
    assert rel(drift, ref) < 1e-5
    assert rel(SB, refS) < 1e-5


@pytest.mark.parametrize("prec,flags,tol0", [(FP64, 0, 1e-6), (MIXED, 4, 1e-5)])
def test_fixman_matches_oracle(pkg, sysD, prec, flags, tol0):
    d = sysD
    Nt = len(d["pos"])
    s = pkg.Suspension(d["pos"], d["body"], d["L"], precision=prec, flags=flags, **HI)
    rng = np.random.default_rng(13)
    n = s.params["grid"]
    field = BO.hermitian_field(n, rng)
    psi_r = rng.normal(size=(Nt, 11))
    psi_nf = rng.normal(size=(Nt, 6))
    kT, dt, m = 0.5, 0.01, 10.0
    ft = synth.random_forces(d["N"], 4)
    det, _, _, _ = s.solve(ft, 0.0)
    slip, fnf, _ = s.brownian(kT, dt, wave_field=field, psi_real=psi_r, psi_nf=psi_nf)
    drift, U0, SB, st, status = s.drift(pkg.FSD_DRIFT_FIXMAN, kT, dt=dt, param=m)
    assert status == pkg.FSD_OK
    rU0, rdrift, rSB, _ = DO.fixman(d["pos"], d["body"], d["L"], slip, fnf, dt, m, rlub=3.0)
    assert rel(U0, rU0) < tol0
    assert rel(drift, rdrift) < 1e-4
    assert rel(SB, rSB) < 1e-4
    # the next solve adds U0 + drift and no Brownian terms of its own
    v1, _, _, _ = s.solve(ft, 0.0)
    s.close()
    assert rel(v1 - det, rU0 + rdrift) < 10 * tol0


def test_invalid_drift_arguments(pkg, sysD):
    d = sysD
    s = pkg.Suspension(d["pos"], d["body"], d["L"], **HI)
    with pytest.raises(pkg.FsdError):
        s.drift(7, 1.0)
    with pytest.raises(pkg.FsdError):
        s.drift(pkg.FSD_DRIFT_RFD, -1.0)
    with pytest.raises(pkg.FsdError):
        s.drift(pkg.FSD_DRIFT_FIXMAN, 1.0, dt=0.01)  # no Brownian terms pending
    with pytest.raises(pkg.FsdError):
        s.drift(pkg.FSD_DRIFT_FIXMAN, 1.0, dt=0.0)
    # the context still works
    v, _, _, st = s.solve(None, 1.0)
    s.close()
    assert st == pkg.FSD_OK and np.all(np.isfinite(v))
