"""GPU parity for aggregates larger than the aggregate-row kernels' lane
groups, against the FP64 oracle.

The aggregate-row, preconditioner and lubrication kernels give each
aggregate a power-of-two group of lanes covering its beads, at most 32: the
other parity suspensions (up to 12 beads per aggregate) stop at 16 lanes.
Here aggregates of 40, 21, 17, 3 and 1 beads (random attachment, packed at
bead volume fraction 0.025 so that every aggregate spans less than half the
box) take 32 lanes per aggregate, and the lanes of the 40-bead aggregate each
visit two of its beads.  Compared through the C ABI with the oracle on the
same inputs: the saddle operator, the aggregate lubrication operator, the
preconditioner and the solve (FP64, mixed, and the mixed solve as a captured
graph), at the tolerances of the other parity tests (relative L2):
  saddle operator FP64 1e-6, FP32 2e-5; lubrication FP64 1e-12, FP32 1e-6;
  preconditioner 1e-12; solve at GMRES 1e-10: FP64 1e-6, mixed 1e-5."""

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


@pytest.fixture(scope="module")
def sysL(pkg):
    rng = np.random.default_rng(7)
    sizes = [40, 21, 17, 3, 1]
    shapes = [synth.random_attachment_aggregate(n, rng) for n in sizes]
    L = synth.box_for_phi(sum(sizes), 0.025)
    pos, body = synth.pack_suspension(shapes, L, rng, h_gen=0.05)
    ft = synth.random_forces(len(sizes), 5)
    M = O.mobility_dense(pos, L)
    sysd = O.assemble(pos, body, L, gamma=1.0, FT=ft, rlub=3.0, M=M)
    sysd["body"] = body
    s = pkg.Suspension(pos, body, L, **HI)
    yield dict(pos=pos, body=body, L=L, ft=ft, s=s, sys=sysd)
    s.close()


def test_suspension_has_large_aggregates_and_lubrication_pairs(sysL):
    counts = np.bincount(sysL["body"])
    assert counts.max() == 40 and (counts > 16).sum() == 3
    assert np.abs(sysL["sys"]["RRFU"]).max() > 0


def test_saddle_operator_matches_oracle(sysL):
    s, A = sysL["s"], sysL["sys"]["A"]
    x = np.random.default_rng(8).normal(size=A.shape[0])
    ref = A @ x
    assert rel(s.apply_saddle(x, FP64), ref) < 1e-6
    assert rel(s.apply_saddle(x, MIXED), ref) < 2e-5


def test_lubrication_operator_matches_oracle(sysL):
    s, sd = sysL["s"], sysL["sys"]
    dU = np.random.default_rng(9).normal(size=(sd["nb"], 6))
    ref = (sd["RRFU"] @ dU.reshape(-1)).reshape(-1, 6)
    assert rel(s.apply_lubrication(dU, FP64), ref) < 1e-12
    assert rel(s.apply_lubrication(dU, MIXED), ref) < 1e-6


def test_preconditioner_matches_oracle(sysL):
    s, sd = sysL["s"], sysL["sys"]
    Pd = O.preconditioner_dense(sd, sd["unw"], sysL["body"], sysL["L"], rp=2.1, rlub=3.0)
    r = np.random.default_rng(10).normal(size=Pd.shape[0])
    assert rel(s.apply_precond(r), Pd @ r) < 1e-12


@pytest.mark.parametrize("precision,graph,tol", [(FP64, False, 1e-6), (MIXED, False, 1e-5),
                                                 (MIXED, True, 1e-5)])
def test_solve_matches_oracle(sysL, pkg, precision, graph, tol):
    sd = sysL["sys"]
    ref = O.outputs(sd, np.linalg.solve(sd["A"], sd["b"]))
    s = pkg.Suspension(sysL["pos"], sysL["body"], sysL["L"], precision=precision,
                       flags=pkg.FSD_FLAG_GRAPH if graph else 0, **HI)
    vel, S, st, status = s.solve(sysL["ft"], 1.0)
    s.close()
    assert status == pkg.FSD_OK
    assert rel(vel[:, :3], ref["U"][:, :3]) < tol
    assert rel(vel[:, 3:], ref["U"][:, 3:]) < tol
    assert rel(S, ref["S"]) < tol
