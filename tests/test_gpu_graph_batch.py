"""GPU checks of the device-resident solve and of the batched form, through
the C ABI.

* FSD_FLAG_GRAPH runs each solve as one captured CUDA graph whose GMRES
  cycles, Arnoldi steps and refinement sweeps are conditional nodes.  It must
  match the FP64 oracle with the host-driven path's tolerances (1e-6 FP64
  path, 1e-5 mixed, at GMRES 1e-10), and match the host-driven path itself
  (same iteration count within one, solutions within 1e-9: the operator
  kernels are the same; spreading sums with atomics, so the two are not
  bitwise equal).
* fsd_*_batch solves independent suspensions of different sizes, boxes and
  aggregate-size mixes together.  Each system's result must match the oracle
  for that system (1e-6 at GMRES 1e-10) and the same system solved alone
  (1e-9); a batch step must move the beads as per-system steps do.
* FSD_FLAG_AUTOTUNE picks the splitting and real-space tile by timing; the
  tuned parameters must still meet the oracle (the accuracy rules fix R_c,
  the grid and P for whatever xi it picks).
"""

import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

FP64, MIXED = 0, 1
HI = dict(xi=1.2, P=12, xerr=1e-8, tol=1e-10, lub_cutoff=3.0)


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g

    g.build()
    import paper_2607_25161_gb300 as p

    return p


def ragged_system(seed=3):
    """Aggregates of 1, 2, 3, 5, 8, 4, 6 and 7 beads packed at phi ~ 0.1."""
    rng = np.random.default_rng(seed)
    sizes = [1, 2, 3, 5, 8, 4, 6, 7]
    shapes = [synth.random_attachment_aggregate(n, rng) for n in sizes]
    L = synth.box_for_phi(sum(sizes), 0.1)
    pos, body = synth.pack_suspension(shapes, L, rng, h_gen=0.05)
    return pos, body, L


def small_batch():
    """Three suspensions with different boxes, sizes and aggregate mixes."""
    out = [ragged_system(3)]
    pos, body, L = synth.config_doublets(6, 24.0, seed=5)
    out.append((pos, body, L))
    pos, body, L = synth.mixed_suspension(60, 0.1, 11, size_hi=12)
    out.append((pos, body, L))
    return out


@pytest.fixture(scope="module")
def oracle_refs():
    refs = []
    for k, (pos, body, L) in enumerate(small_batch()):
        ft = synth.random_forces(body.max() + 1, 10 + k)
        ref = O.solve(pos, body, L, gamma=1.0 + 0.5 * k, FT=ft, rlub=3.0)
        refs.append(dict(pos=pos, body=body, L=L, ft=ft, shear=1.0 + 0.5 * k, ref=ref))
    return refs


# ------------------------------------------------------------ graph path

@pytest.mark.parametrize("prec,tol,extra", [(FP64, 1e-6, 0), (MIXED, 1e-5, 0), (MIXED, 1e-5, 32)])
def test_graph_solve_matches_oracle(pkg, oracle_refs, prec, tol, extra):
    # extra 32: FSD_FLAG_FP32_KRYLOV (FP32 inner Krylov basis)
    r = oracle_refs[0]
    s = pkg.Suspension(r["pos"], r["body"], r["L"], precision=prec,
                       flags=pkg.FSD_FLAG_GRAPH | extra, **HI)
    vel, S, st, status = s.solve(r["ft"], r["shear"])
    s.close()
    assert status == pkg.FSD_OK
    assert st["rel_residual"] <= 1e-10
    assert st["kernel_launches"] > 0
    if prec == MIXED:
        assert st["matvec32"] > 0 and st["matvec64"] >= 1
    assert rel(vel, r["ref"]["U"]) < tol
    assert rel(S, r["ref"]["S"]) < tol


@pytest.mark.parametrize("prec,extra", [(FP64, 0), (MIXED, 0), (MIXED, 32)])
def test_graph_matches_host_driven_loop(pkg, oracle_refs, prec, extra):
    r = oracle_refs[2]
    out = {}
    for flags in (0, 4):
        s = pkg.Suspension(r["pos"], r["body"], r["L"], precision=prec, flags=flags | extra, **HI)
        vel, S, st, status = s.solve(r["ft"], r["shear"])
        s.close()
        assert status == pkg.FSD_OK
        out[flags] = (vel, S, st)
    assert abs(out[0][2]["iters"] - out[4][2]["iters"]) <= 1
    assert abs(out[0][2]["outer_iters"] - out[4][2]["outer_iters"]) <= 1
    assert rel(out[4][0], out[0][0]) < 1e-9
    assert rel(out[4][1], out[0][1]) < 1e-9


def test_graph_warm_start_and_repeat(pkg, oracle_refs):
    r = oracle_refs[1]
    s = pkg.Suspension(r["pos"], r["body"], r["L"],
                       flags=pkg.FSD_FLAG_GRAPH | pkg.FSD_FLAG_WARM_START, **HI)
    v1, S1, st1, _ = s.solve(r["ft"], r["shear"])
    v2, S2, st2, _ = s.solve(r["ft"], r["shear"])   # warm: already converged
    v3, S3, st3, _ = s.solve(r["ft"], r["shear"])   # the cached graph again
    s.close()
    assert st1["iters"] > 0 and st2["iters"] == 0 and st3["iters"] == 0
    assert rel(v2, v1) < 1e-12 and rel(v3, v1) < 1e-12
    assert rel(v1, r["ref"]["U"]) < 1e-6


def test_graph_zero_right_hand_side(pkg, oracle_refs):
    r = oracle_refs[0]
    s = pkg.Suspension(r["pos"], r["body"], r["L"], flags=pkg.FSD_FLAG_GRAPH, **HI)
    vel, S, st, status = s.solve(None, 0.0)
    s.close()
    assert status == pkg.FSD_OK
    assert st["iters"] == 0
    assert np.all(vel == 0.0) and np.all(S == 0.0)


def test_graph_no_convergence_reports_status(pkg, oracle_refs):
    r = oracle_refs[0]
    s = pkg.Suspension(r["pos"], r["body"], r["L"], flags=pkg.FSD_FLAG_GRAPH,
                       max_iter=2, restart=2, **HI)
    vel, S, st, status = s.solve(None, 1.0, allow=(pkg.FSD_ENOCONV,))
    s.close()
    assert status == pkg.FSD_ENOCONV
    assert st["iters"] == 2
    assert st["rel_residual"] > 1e-10 and np.all(np.isfinite(vel))


@pytest.mark.parametrize("comoving", [0, 2])
def test_graph_step_matches_host_driven_step(pkg, oracle_refs, comoving):
    r = oracle_refs[0]
    res = {}
    for flags in (0, 4):
        s = pkg.Suspension(r["pos"], r["body"], r["L"], flags=flags | comoving,
                           precision=MIXED, **HI)
        vel = np.zeros((r["body"].max() + 1, 6))
        for _ in range(3):
            s.step(r["ft"], r["shear"], 0.02, vel=vel)
        res[flags] = s.beads() + (vel.copy(),)
        s.close()
    assert rel(res[4][2], res[0][2]) < 1e-8
    assert np.abs(res[4][0] - res[0][0]).max() < 1e-9
    assert np.abs(res[4][1] - res[0][1]).max() < 1e-9


# --------------------------------------------------------------- batch

def test_batch_solve_matches_oracle_and_single(pkg, oracle_refs):
    systems = [(r["pos"], r["body"], r["L"]) for r in oracle_refs]
    b = pkg.Batch(systems, [dict(HI, precision=MIXED)] * len(systems))
    assert b.n_sys == 3
    assert list(b.agg_off) == list(np.cumsum([0] + [r["body"].max() + 1 for r in oracle_refs]))
    ft = np.concatenate([r["ft"] for r in oracle_refs])
    shear = np.array([r["shear"] for r in oracle_refs])
    vel, S, stats, status = b.solve(ft, shear)
    assert status == pkg.FSD_OK
    for k, r in enumerate(oracle_refs):
        sl = slice(b.agg_off[k], b.agg_off[k + 1])
        assert stats[k]["rel_residual"] <= 1e-10 and stats[k]["iters"] > 0
        assert rel(vel[sl], r["ref"]["U"]) < 1e-5
        assert rel(S[sl], r["ref"]["S"]) < 1e-5
        # the same system solved on its own
        s = pkg.Suspension(r["pos"], r["body"], r["L"], precision=MIXED, **HI)
        v1, S1, st1, _ = s.solve(r["ft"], r["shear"])
        s.close()
        assert rel(vel[sl], v1) < 1e-9 and rel(S[sl], S1) < 1e-9
    b.close()


def test_batch_fp64_matches_oracle(pkg, oracle_refs):
    systems = [(r["pos"], r["body"], r["L"]) for r in oracle_refs]
    b = pkg.Batch(systems, HI)
    ft = np.concatenate([r["ft"] for r in oracle_refs])
    shear = np.array([r["shear"] for r in oracle_refs])
    vel, S, stats, status = b.solve(ft, shear)
    b.close()
    assert status == pkg.FSD_OK
    for k, r in enumerate(oracle_refs):
        sl = slice(b.agg_off[k], b.agg_off[k + 1])
        assert rel(vel[sl], r["ref"]["U"]) < 1e-6
        assert rel(S[sl], r["ref"]["S"]) < 1e-6


def test_batch_step_matches_single_steps(pkg, oracle_refs):
    systems = [(r["pos"], r["body"], r["L"]) for r in oracle_refs]
    prm = dict(HI, precision=MIXED, flags=2)
    b = pkg.Batch(systems, prm)
    ft = np.concatenate([r["ft"] for r in oracle_refs])
    shear = np.array([r["shear"] for r in oracle_refs])
    for _ in range(2):
        b.step(ft, shear, 0.02)
    pos_b, q_b = b.beads()
    b.close()
    for k, r in enumerate(oracle_refs):
        s = pkg.Suspension(r["pos"], r["body"], r["L"], **prm)
        for _ in range(2):
            s.step(r["ft"], r["shear"], 0.02)
        x, q = s.beads()
        s.close()
        assert np.abs(pos_b[b.bead_off[k]:b.bead_off[k + 1]] - x).max() < 1e-9
        assert np.abs(q_b[b.agg_off[k]:b.agg_off[k + 1]] - q).max() < 1e-9


def test_batch_system_view_and_errors(pkg, oracle_refs):
    systems = [(r["pos"], r["body"], r["L"]) for r in oracle_refs]
    b = pkg.Batch(systems, HI)
    s1 = b.system(1)
    r = oracle_refs[1]
    vel, S, st, status = s1.solve(r["ft"], r["shear"])
    assert rel(vel, r["ref"]["U"]) < 1e-6
    with pytest.raises(IndexError):
        b.system(3)
    s1.close()  # a view: the batch still owns the context
    vel2, _, _, _ = b.solve(None, np.zeros(3))
    assert np.all(vel2 == 0.0)
    b.close()
    # a system whose real-space cut-off reaches L/2 is rejected with its index
    pos, body, L = synth.config_doublets(2, 10.0, seed=2)
    with pytest.raises(pkg.FsdError, match="system 1"):
        pkg.Batch([systems[0], (pos, body, L)], [HI, dict(xi=0.3)])


# ------------------------------------------------------------- autotune

def test_autotune_meets_oracle(pkg):
    pos, body, L = synth.mixed_suspension(100, 0.12, 21, size_hi=16)
    ft = synth.random_forces(body.max() + 1, 21)
    ref = O.solve(pos, body, L, gamma=1.0, FT=ft, rlub=3.0)
    s = pkg.Suspension(pos, body, L, flags=pkg.FSD_FLAG_AUTOTUNE | pkg.FSD_FLAG_GRAPH,
                       xerr=1e-8, P=12, tol=1e-10, lub_cutoff=3.0, precision=MIXED)
    prm = s.params
    assert prm["tile"] in (4, 8, 16, 32)
    assert prm["xi"] > 0 and prm["rc"] < 0.5 * L
    vel, S, st, status = s.solve(ft, 1.0)
    s.close()
    assert status == pkg.FSD_OK
    assert rel(vel, ref["U"]) < 1e-5 and rel(S, ref["S"]) < 1e-5
