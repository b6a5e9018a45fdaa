"""GPU checks at the benchmark's full size and launch configuration: 32768
beads (4096 rigid 8-bead aggregates, phi 0.2, L 88.21), xi 0.5, the grid and
P of the defaulting rules, lubrication 3a, r_p = 2a.

The dense oracle does not fit at this size, so the checks are
* sampled outputs the oracle computes one by one: rows of the real-space sum
  at the library's (xi, R_c) and aggregate rows of the lubrication operator;
* properties that hold at any size: symmetry and positivity of the wave-space
  operator, invariance of the mobility under a rigid translation of the
  suspension, and agreement of the FP64 and mixed solves."""

import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

FP64, MIXED = 0, 1
PARAMS = dict(xi=0.5, lub_cutoff=3.0, precond_cutoff=2.0)


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def big():
    import __graft_entry__ as g

    g.build()
    import paper_2607_25161_gb300 as pkg

    pos, body, L = synth.suspension(4096, 8, 0.2, 1)
    s = pkg.Suspension(pos, body, L, **PARAMS)
    yield dict(pkg=pkg, pos=pos, body=body, L=L, s=s, prm=s.params)
    s.close()


def test_fullsize_real_space_sampled_rows(big):
    pos, L, s, prm = big["pos"], big["L"], big["s"], big["prm"]
    rng = np.random.default_rng(41)
    F = rng.normal(size=(len(pos), 11))
    rows = [0, 1, 777, 5003, 12345, 20000, 27777, len(pos) - 1]
    ref = O.mobility_real_rows(pos, L, prm["xi"], prm["rc"], rows, F)
    got64 = s.apply_mobility(F, part=1, precision=FP64)[rows]
    got32 = s.apply_mobility(F, part=1, precision=MIXED)[rows]
    assert rel(got64, ref) < 1e-9
    assert rel(got32, ref) < 5e-6


def test_fullsize_lubrication_sampled_aggregates(big):
    pos, body, L, s = big["pos"], big["body"], big["L"], big["s"]
    rng = np.random.default_rng(42)
    dU = rng.normal(size=(body.max() + 1, 6))
    bodies = [0, 17, 999, 2048, 3333, 4095]
    ref = O.lubrication_rows(pos, body, L, bodies, dU)
    got64 = s.apply_lubrication(dU, FP64)[bodies]
    got32 = s.apply_lubrication(dU, MIXED)[bodies]
    assert np.abs(ref).max() > 0
    assert rel(got64, ref) < 1e-12
    assert rel(got32, ref) < 1e-6


def test_fullsize_wave_space_symmetric_positive(big):
    s = big["s"]
    rng = np.random.default_rng(43)
    F = rng.normal(size=(s.n_beads, 11))
    G = rng.normal(size=(s.n_beads, 11))
    for prec, tol in ((FP64, 1e-11), (MIXED, 1e-5)):
        MF = s.apply_mobility(F, part=2, precision=prec)
        MG = s.apply_mobility(G, part=2, precision=prec)
        a, b = np.sum(G * MF), np.sum(F * MG)
        assert abs(a - b) < tol * np.sqrt(np.sum(F * MF) * np.sum(G * MG))
        assert np.sum(F * MF) > 0


def test_fullsize_mobility_translation_invariant(big):
    # a rigid translation of the whole suspension leaves M_inf F unchanged up
    # to the grid discretisation; at P = 12 and the xerr = 1e-8 rules that is
    # below 1e-6
    pkg, pos, body, L = big["pkg"], big["pos"], big["body"], big["L"]
    hi = dict(PARAMS, P=12, xerr=1e-8)
    rng = np.random.default_rng(44)
    F = rng.normal(size=(len(pos), 11))
    s1 = pkg.Suspension(pos, body, L, **hi)
    a = s1.apply_mobility(F, part=3, precision=FP64)
    s1.close()
    s2 = pkg.Suspension(pos + np.array([0.37, -1.13, 2.71]), body, L, **hi)
    b = s2.apply_mobility(F, part=3, precision=FP64)
    s2.close()
    assert rel(b, a) < 1e-6


def test_fullsize_fp64_and_mixed_solves_agree(big):
    pkg, pos, body, L = big["pkg"], big["pos"], big["body"], big["L"]
    out = {}
    for prec in (FP64, MIXED):
        s = pkg.Suspension(pos, body, L, precision=prec, tol=1e-8, **PARAMS)
        vel, S, st, status = s.solve(None, 1.0)
        s.close()
        assert status == pkg.FSD_OK
        assert st["rel_residual"] <= 1e-8
        out[prec] = (vel, S)
    assert rel(out[MIXED][0], out[FP64][0]) < 1e-5
    assert rel(out[MIXED][1], out[FP64][1]) < 1e-5


def test_fullsize_brownian_wave_sample_linear_and_scaled(big):
    # properties of u^B = sqrt(2 kT/dt) M_w^(1/2) psi_w at any size: linear in
    # the random field, scaled by sqrt(kT/dt), zero for a zero field
    from oracle import brownian_oracle as BO

    pkg, pos, body, L = big["pkg"], big["pos"], big["body"], big["L"]
    s = pkg.Suspension(pos, body, L, precision=MIXED, nf_sampler=pkg.FSD_NF_LANCZOS, **PARAMS)
    n = s.params["grid"]
    rng = np.random.default_rng(43)
    f1 = BO.hermitian_field(n, rng)
    f2 = BO.hermitian_field(n, rng)
    z11 = np.zeros((len(pos), 11))
    z6 = np.zeros((len(pos), 6))
    u1, _, _ = s.brownian(1.0, 1.0, wave_field=f1, psi_real=z11, psi_nf=z6)
    u2, _, _ = s.brownian(1.0, 1.0, wave_field=f2, psi_real=z11, psi_nf=z6)
    u12, _, _ = s.brownian(1.0, 1.0, wave_field=f1 + 0.5 * f2, psi_real=z11, psi_nf=z6)
    u1s, _, _ = s.brownian(4.0, 0.25, wave_field=f1, psi_real=z11, psi_nf=z6)
    u0, _, _ = s.brownian(1.0, 1.0, wave_field=0.0 * f1, psi_real=z11, psi_nf=z6)
    s.close()
    assert np.abs(u1).max() > 0
    assert rel(u12, u1 + 0.5 * u2) < 1e-5
    assert rel(u1s, 4.0 * u1) < 1e-12
    assert np.all(u0 == 0.0)
