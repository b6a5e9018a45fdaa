"""GPU parity of the Brownian forcing (fsd_brownian; Sec. 2.2 stochastic
sampling, Eq. SP2, Eq. UBff, Algorithm 1 step 3) against the Brownian oracle,
through the C ABI, on the same random inputs.

Tolerances (relative L2):
  wave part (analytic PSE sample, grid rule x_err = 1e-8, P = 16: the
    interpolation's truncation error is ~1.5e-6 at P = 12, ~1e-8 at P = 16):
    1e-6 FP64, 1e-5 with the FP32 operator;
  real-space square root (Lanczos, coefficient change < 1e-7 on the
    real-space operator): 1e-6 FP64, 1e-5 FP32;
  near-field square root (block-Cholesky preconditioned Lanczos on the FP64
    bead blocks, against the oracle's preconditioned square root): 1e-6;
  Brownian solve at GMRES 1e-10: 1e-6 FP64, 1e-5 mixed.
"""

import numpy as np
import pytest

import oracle as O
import synth
from oracle import brownian_oracle as BO

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


def ragged_system(seed=3):
    rng = np.random.default_rng(seed)
    sizes = [1, 2, 3, 5, 8, 4, 6, 7]
    shapes = [synth.random_attachment_aggregate(n, rng) for n in sizes]
    L = synth.box_for_phi(sum(sizes), 0.1)
    pos, body = synth.pack_suspension(shapes, L, rng, h_gen=0.05)
    return pos, body, L


@pytest.fixture(scope="module")
def sysB(pkg):
    pos, body, L = ragged_system()
    s = pkg.Suspension(pos, body, L, **HI)
    prm = s.params
    s.close()
    n, xi = prm["grid"], prm["xi"]
    rng = np.random.default_rng(11)
    field = BO.hermitian_field(n, rng)
    psi_r = rng.normal(size=(len(pos), 11))
    psi_nf = rng.normal(size=(len(pos), 6))
    unw, X, r = O.body_geometry(pos, body, L)
    uw = BO.brownian_wave_slip(unw, L, xi, n, field)
    rc = 2.0 + np.sqrt(46.0) / xi
    Mr = O.mobility_real_dense(unw, L, xi, rc).reshape(11 * len(pos), -1)
    ur = BO.sqrtm_apply(Mr, psi_r.reshape(-1)).reshape(-1, 11)
    RFU = O.split_grand(O.lubrication_dense(unw, body, L, rcut=3.0), len(pos))[0]
    fnf = BO.block_precond_sqrt_apply(RFU, psi_nf.reshape(-1)).reshape(-1, 6)
    return dict(pos=pos, body=body, L=L, n=n, xi=xi, field=field, psi_r=psi_r, psi_nf=psi_nf,
                uw=uw, ur=ur, fnf=fnf)


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-6), (MIXED, 1e-5)])
def test_wave_slip_matches_oracle(pkg, sysB, prec, tol):
    d = sysB
    s = pkg.Suspension(d["pos"], d["body"], d["L"], precision=prec, **HI)
    z = np.zeros_like(d["psi_r"])
    slip, fnf, st = s.brownian(1.0, 1.0, wave_field=d["field"], psi_real=z,
                               psi_nf=np.zeros_like(d["psi_nf"]))
    s.close()
    assert rel(slip / np.sqrt(2.0), d["uw"]) < tol
    assert np.all(fnf == 0.0)


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-6), (MIXED, 1e-5)])
def test_real_space_lanczos_matches_dense_square_root(pkg, sysB, prec, tol):
    d = sysB
    s = pkg.Suspension(d["pos"], d["body"], d["L"], precision=prec, **HI)
    slip, fnf, st = s.brownian(2.0, 0.5, wave_field=np.zeros_like(d["field"]), psi_real=d["psi_r"],
                               psi_nf=np.zeros_like(d["psi_nf"]))
    s.close()
    assert 2 <= st["iters"] <= 60
    assert rel(slip / np.sqrt(2.0 * 2.0 / 0.5), d["ur"]) < tol


def test_near_field_lanczos_matches_dense_square_root(pkg, sysB):
    d = sysB
    assert np.abs(d["fnf"]).max() > 0
    s = pkg.Suspension(d["pos"], d["body"], d["L"], **HI)
    slip, fnf, st = s.brownian(1.0, 1.0, wave_field=np.zeros_like(d["field"]),
                               psi_real=np.zeros_like(d["psi_r"]), psi_nf=d["psi_nf"])
    s.close()
    assert st["outer_iters"] >= 2
    assert rel(fnf / np.sqrt(2.0), d["fnf"]) < 1e-6


@pytest.mark.parametrize("prec,tol,flags", [(FP64, 1e-6, 0), (MIXED, 1e-5, 0), (MIXED, 1e-5, 4)])
def test_brownian_solve_matches_oracle(pkg, sysB, prec, tol, flags):
    d = sysB
    kT, dt = 0.7, 0.01
    sc = np.sqrt(2.0 * kT / dt)
    uB = sc * (d["uw"] + d["ur"])
    fB = sc * d["fnf"]
    ft = synth.random_forces(d["body"].max() + 1, 12)
    ref = BO.solve_brownian(d["pos"], d["body"], d["L"], uB, fB, gamma=1.0, FT=ft, rlub=3.0)
    s = pkg.Suspension(d["pos"], d["body"], d["L"], precision=prec, flags=flags, **HI)
    slip, fnf, _ = s.brownian(kT, dt, wave_field=d["field"], psi_real=d["psi_r"], psi_nf=d["psi_nf"])
    assert rel(slip, uB) < tol and rel(fnf, fB) < 1e-6
    vel, S, st, status = s.solve(ft, 1.0)
    assert status == pkg.FSD_OK
    assert rel(vel, ref["U"]) < tol
    assert rel(S, ref["S"]) < tol
    # the terms are used once: the next solve is the deterministic one
    vel2, S2, _, _ = s.solve(ft, 1.0)
    s.close()
    det = O.solve(d["pos"], d["body"], d["L"], gamma=1.0, FT=ft, rlub=3.0)
    assert rel(vel2, det["U"]) < tol


def test_internal_generator_matches_oracle_philox(pkg, sysB):
    d = sysB
    seed, step = 123456789012345, 42
    s = pkg.Suspension(d["pos"], d["body"], d["L"], **HI)
    slip, fnf, st = s.brownian(1.0, 1.0, seed=seed, step=step)
    s.close()
    n, N = d["n"], len(d["pos"])
    field = BO.philox_wave_field(n, seed, step)
    psi_r = BO.philox_psi(N, seed, step, 2, 11)
    psi_nf = BO.philox_psi(N, seed, step, 3, 6)
    unw, X, r = O.body_geometry(d["pos"], d["body"], d["L"])
    uw = BO.brownian_wave_slip(unw, d["L"], d["xi"], n, field)
    rc = 2.0 + np.sqrt(46.0) / d["xi"]
    Mr = O.mobility_real_dense(unw, d["L"], d["xi"], rc).reshape(11 * N, -1)
    ur = BO.sqrtm_apply(Mr, psi_r.reshape(-1)).reshape(-1, 11)
    RFU = O.split_grand(O.lubrication_dense(unw, d["body"], d["L"], rcut=3.0), N)[0]
    f = BO.block_precond_sqrt_apply(RFU, psi_nf.reshape(-1)).reshape(-1, 6)
    assert rel(slip / np.sqrt(2.0), uw + ur) < 1e-6
    assert rel(fnf / np.sqrt(2.0), f) < 1e-6


def test_invalid_brownian_arguments(pkg, sysB):
    d = sysB
    s = pkg.Suspension(d["pos"], d["body"], d["L"], **HI)
    with pytest.raises(pkg.FsdError):
        s.brownian(-1.0, 1.0)
    with pytest.raises(pkg.FsdError):
        s.brownian(1.0, 0.0)
    s.close()


def test_wave_sample_on_a_grid_too_large_for_the_fused_fft(pkg):
    # n = 180: FP32 planes no longer fit shared memory, so the FP32 sample
    # takes the separate x and y passes (like FP64); the sample is the first
    # thing each fresh context runs
    rng = np.random.default_rng(21)
    pos = rng.uniform(0.0, 30.0, size=(6, 3))
    pos[:, 0] = np.arange(6) * 5.0 + 1.0
    body = np.arange(6)
    out = []
    for prec in (FP64, MIXED):
        s = pkg.Suspension(pos, body, 30.0, precision=prec, xi=0.5, grid=180)
        assert s.params["grid"] == 180
        z = np.zeros((6, 11))
        slip, _, _ = s.brownian(1.0, 1.0, seed=3, step=9, psi_real=z, psi_nf=np.zeros((6, 6)))
        s.close()
        out.append(slip)
    assert np.abs(out[0]).max() > 0
    assert rel(out[1], out[0]) < 1e-5


def test_pairwise_near_field_sampler_matches_oracle(pkg, sysB):
    # nf_sampler = FSD_NF_PAIRWISE: sum over lubrication pairs of K_p^T psi_p
    # (the pair's dissipation-form factor) with Philox pair noise, against
    # the oracle's sampler
    d = sysB
    seed, step = 77, 5
    s = pkg.Suspension(d["pos"], d["body"], d["L"], **dict(HI, nf_sampler=pkg.FSD_NF_PAIRWISE))
    slip, fnf, st = s.brownian(1.0, 1.0, seed=seed, step=step, psi_real=np.zeros_like(d["psi_r"]))
    with pytest.raises(pkg.FsdError):
        s.brownian(1.0, 1.0, psi_nf=d["psi_nf"])  # the pair noise is drawn, not given
    s.close()
    unw, X, r = O.body_geometry(d["pos"], d["body"], d["L"])
    ref = BO.pairwise_nf_force(unw, d["body"], d["L"], seed, step, rlub=3.0)
    assert np.abs(ref).max() > 0
    assert st["outer_iters"] == 0  # no near-field Lanczos steps
    assert rel(fnf / np.sqrt(2.0), ref) < 1e-12
