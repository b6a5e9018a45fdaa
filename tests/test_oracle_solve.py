"""Pins of the oracle's saddle-point solve, near-field resistance,
preconditioner and integrator (CPU only)."""

import numpy as np
import pytest

import oracle as O
import synth
from conftest import golden

PI = np.pi


@pytest.fixture(scope="module")
def doublets():
    pos, body, L = synth.config_doublets(n_agg=6, L=24.0, seed=3)
    FT = synth.random_forces(6, 3)
    out = O.solve(pos, body, L, gamma=1.0, FT=FT)
    return pos, body, L, FT, out


def test_residual_and_rigid_constraint(doublets):
    pos, body, L, FT, out = doublets
    assert out["rel_residual"] < 1e-13
    sys_ = out["system"]
    Nt = sys_["Nt"]
    # bead velocities follow rigid-body motion: M F = -(Sigma^T dU - E r) on u, omega rows
    n1 = 11 * Nt
    uF = (sys_["M"] @ out["x"][:n1]).reshape(Nt, 11)
    rigid = (sys_["ST"] @ out["x"][n1:]).reshape(Nt, 6)
    Er = sys_["Er"].reshape(Nt, 6)
    assert np.allclose(uF[:, :6], -(rigid - Er), atol=1e-13 * np.abs(rigid).max())
    # beads do not strain: the read-out strain equals E_inf
    assert np.allclose(uF[:, 6:], sys_["e5"][None, :], atol=1e-13)
    # force balance per aggregate: Sigma B^T F = -F^P (no lubrication here)
    FH = (sys_["ST"].T @ (sys_["Bm"].T @ out["x"][:n1])).reshape(-1, 6)
    assert np.allclose(FH, -FT, atol=1e-12)


def test_schur_route_equals_saddle_route(doublets):
    out = doublets[4]
    x2 = O.solve_schur(out["system"])
    assert np.abs(x2 - out["x"]).max() < 1e-12 * np.abs(out["x"]).max()


def test_single_bead_aggregates_reduce_to_sphere_fsd():
    # n_b = 1: Sigma = I, and Eq. spm_agg becomes the sphere system Eq. SP1
    rng = np.random.default_rng(4)
    L = 14.0
    pos = np.array([[1.0, 2.0, 3.0], [4.5, 2.5, 3.2], [9.0, 9.0, 1.0]])
    body = np.arange(3)
    FT = rng.normal(size=(3, 6))
    out = O.solve(pos, body, L, gamma=0.7, FT=FT, rlub=3.0)
    sys_ = out["system"]
    M = sys_["M"]
    N = 3
    Bm = O.B_op(N)
    Rg = O.lubrication_dense(pos, body, L, rcut=3.0)
    RFU, RFE, _, _ = O.split_grand(Rg, N)
    E, _ = O.shear_flow(0.7)
    e5 = O.sym_to_vec5(E)
    A = np.block([[M, Bm], [Bm.T, -RFU]])
    b = np.concatenate([np.tile(np.r_[np.zeros(6), e5], N), -(FT.reshape(-1) + RFE @ np.tile(e5, N))])
    x = np.linalg.solve(A, b)
    assert np.allclose(x, out["x"], rtol=0, atol=1e-12 * np.abs(x).max())


@pytest.mark.parametrize("L", [10.0, 30.0])
def test_single_sphere_in_periodic_shear(L):
    # cubic symmetry: the sphere co-rotates with the fluid, moves with it, and
    # its stresslet has only the xy component; as a/L -> 0 it tends to the
    # isolated-sphere value (20/3) pi eta a^3 E_xy
    out = O.solve(np.array([[0.3, 0.2, 0.1]]), np.array([0]), L, gamma=1.0)
    U = out["U"][0]
    assert np.allclose(U[3:6], [0, 0, -0.5], atol=1e-12)
    assert np.allclose(U[0:3], [0.2, 0, 0], atol=1e-12)
    S = out["S"][0]
    off = S.copy()
    off[0, 1] = off[1, 0] = 0.0
    assert np.abs(off).max() < 1e-12
    S0 = 20.0 / 3.0 * PI * 0.5
    # periodic correction is O((a/L)^3)
    assert abs(S[0, 1] / S0 - 1.0) < 10.0 / L ** 3


def test_doublet_in_shear_jeffery_form():
    # omega_z / gamma = -1/2 (1 + B cos 2 theta), theta from the gradient axis;
    # forces on a bead: F_r ~ sin 2 theta, F_t ~ cos 2 theta (Sec. 3.1.1)
    L = 60.0
    thetas = np.linspace(0, PI, 7, endpoint=False)
    om, Fr, Ft = [], [], []
    c = np.array([30.0, 30.0, 30.0])
    for th in thetas:
        n = np.array([np.sin(th), np.cos(th), 0.0])
        pos = np.array([c + n, c - n])
        out = O.solve(pos, np.array([0, 0]), L, gamma=1.0)
        om.append(out["U"][0, 5])
        F = out["F"][0, 0:3]  # hydrodynamic force on bead 0 (at c + n)
        t = np.array([np.cos(th), -np.sin(th), 0.0])
        Fr.append(F @ n)
        Ft.append(F @ t)
    om, Fr, Ft = map(np.array, (om, Fr, Ft))
    G = np.stack([np.ones_like(thetas), np.cos(2 * thetas)], 1)
    coef, res, *_ = np.linalg.lstsq(G, -2 * om, rcond=None)
    assert np.abs(G @ coef + 2 * om).max() < 1e-3
    assert abs(coef[0] - 1.0) < 2e-3
    B = coef[1]
    # FTS-RPY with the stresslet constraint gives B = 0.607 vs the exact 0.594
    assert abs(B - golden("doublet_jeffery_B")) < 0.03
    amp_r = np.linalg.lstsq(np.sin(2 * thetas)[:, None], Fr, rcond=None)[0][0]
    amp_t = np.linalg.lstsq(np.cos(2 * thetas)[:, None], Ft, rcond=None)[0][0]
    assert np.abs(amp_r * np.sin(2 * thetas) - Fr).max() < 0.02 * abs(amp_r)
    assert np.abs(amp_t * np.cos(2 * thetas) - Ft).max() < 0.02 * abs(amp_t)
    h1, h2 = golden("doublet_h1"), golden("doublet_h2")
    ref_r = PI / 2 * (h1 + h2)
    # both amplitudes come out ~7 % below the exact two-sphere values: the
    # truncated multipole expansion underestimates them (Sec. 3.1.1)
    assert 0.88 < abs(amp_r) / ref_r < 1.0
    assert 0.85 < abs(amp_t) / (PI / 2 * h1) < 1.0


# -------------------------------------------------------------- lubrication


def _two_body_pair(gap, seed=0):
    rng = np.random.default_rng(seed)
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    return np.zeros(3), (2.0 + gap) * n


@pytest.mark.parametrize("gap", [1e-4, 0.05, 0.4, 0.95])
def test_lubrication_pair_symmetric_psd_and_rigid_invariant(gap):
    xi, xj = _two_body_pair(gap, 1)
    R = O.lub_pair_matrix(xi, xj)
    assert np.abs(R - R.T).max() < 1e-12 * np.abs(R).max()
    assert np.linalg.eigvalsh(R).min() > -1e-10 * np.abs(R).max()
    # rigid translation and rotation of the pair (no strain) dissipate nothing
    rng = np.random.default_rng(2)
    V, W = rng.normal(size=3), rng.normal(size=3)
    c = 0.5 * (xi + xj)
    nu = np.zeros(22)
    for k, x in ((0, xi), (11, xj)):
        nu[k:k + 3] = -(V + np.cross(W, x - c))
        nu[k + 3:k + 6] = -W
    f = R @ nu
    assert np.abs(f).max() < 1e-9 * np.abs(R).max()
    # squeeze motion is resisted with the 1/eps singularity
    nu = np.zeros(22)
    d = (xj - xi) / np.linalg.norm(xj - xi)
    nu[0:3] = -d
    fi = (R @ nu)[0:3]
    A = O.lub_coefficients(gap)[0]
    assert np.allclose(fi, -A * d, rtol=1e-12, atol=1e-12)


def test_lubrication_coefficients_follow_equal_sphere_asymptotics():
    # Two-sphere lubrication theory (Jeffrey & Onishi 1984, J. Fluid Mech.
    # 139; Kim & Karrila 1991, Microhydrodynamics, ch. 11) gives, for spheres
    # of size ratio beta at dimensionless gap eps -> 0, the singular terms
    #   X^A_11 = g1 / eps + g2 ln(1/eps),  g1 = 2 beta^2 / (1 + beta)^3,
    #                                     g2 = beta (1 + 7 beta + beta^2) / (5 (1 + beta)^3)
    #   Y^A_11 = g2t ln(1/eps),            g2t = 4 beta (2 + beta + 2 beta^2) / (15 (1 + beta)^3)
    # and for equal spheres moving apart / sliding with relative velocity V
    # the force is 6 pi eta a X^A_11 V (squeeze) or 6 pi eta a Y^A_11 V
    # (sliding): the pair model's A and B.  Their differences between two gaps
    # cancel the cut-off shift.
    beta = 1.0
    g1 = 2 * beta ** 2 / (1 + beta) ** 3
    g2 = beta * (1 + 7 * beta + beta ** 2) / (5 * (1 + beta) ** 3)
    g2t = 4 * beta * (2 + beta + 2 * beta ** 2) / (15 * (1 + beta) ** 3)
    z0 = 6 * PI

    def AB(eps):
        A, B, _ = O.lub_coefficients(eps, hmin=1e-12)
        return A / z0, B / z0

    e1, e2 = 1e-7, 1e-5
    (A1, B1), (A2, B2) = AB(e1), AB(e2)
    # the Reynolds limit: eps A -> g1 (squeeze force (3/2) pi eta a^2 V / h)
    assert abs(e1 * A1 - g1) < 1e-5
    # logarithmic terms
    ln = np.log(e2 / e1)
    assert abs(((A1 - g1 / e1) - (A2 - g1 / e2)) / ln - g2) < 1e-3
    assert abs((B1 - B2) / ln - g2t) < 1e-3


def test_assembled_strain_blocks_equal_affine_bead_motion():
    # the pair model sees only relative surface velocities, so on the whole
    # suspension the strain response equals the response to every bead
    # moving with -E.x_b (no pair crosses the box here, so x_j - x_i needs no
    # image): R_FE e = R_FU (-E x, 0) and R_SE e = R_SU (-E x, 0), with the
    # blocks taken from the grand resistance by split_grand
    rng = np.random.default_rng(23)
    shapes = [synth.random_attachment_aggregate(k, rng) for k in (3, 2, 4)]
    L = 60.0
    pos, body = synth.pack_suspension(shapes, 9.0, rng, h_gen=0.05)
    pos = pos + 20.0  # a 9-box cluster in the middle of a 60-box
    Nt = len(pos)
    R = O.lubrication_dense(pos, body, L, rcut=3.0)
    RFU, RFE, RSU, RSE = O.split_grand(R, Nt)
    assert np.abs(RFE).max() > 0
    E = rng.normal(size=(3, 3))
    E = 0.5 * (E + E.T)
    E -= np.trace(E) / 3.0 * np.eye(3)
    e = np.tile(O.sym_to_vec5(E), Nt)
    v = np.zeros((Nt, 6))
    v[:, 0:3] = -(pos @ E.T)
    v = v.reshape(-1)
    assert np.abs(RFE @ e - RFU @ v).max() < 1e-10 * np.abs(RFU @ v).max()
    assert np.abs(RSE @ e - RSU @ v).max() < 1e-10 * np.abs(RSU @ v).max()


def test_lubrication_lowers_the_body_mobility():
    # near-field resistance can only lower the mobility: the body mobility N
    # (disturbance velocities per unit applied force and torque, Eq. FH_agg)
    # stays symmetric positive definite, and N without lubrication minus N
    # with it is positive semi-definite, and nonzero when pairs are near
    rng = np.random.default_rng(21)
    shapes = [synth.random_attachment_aggregate(k, rng) for k in (2, 3, 2)]
    L = synth.box_for_phi(7, 0.2)
    pos, body = synth.pack_suspension(shapes, L, rng, h_gen=0.05)
    M = O.mobility_dense(pos, L)
    nb = 3

    def N(rlub):
        return np.column_stack([O.solve(pos, body, L, gamma=0.0, FT=np.eye(6 * nb)[j].reshape(nb, 6),
                                        rlub=rlub, M=M)["U"].reshape(-1) for j in range(6 * nb)])

    N0, N1 = N(0.0), N(3.0)
    scale = np.abs(N0).max()
    for Nm in (N0, N1):
        assert np.abs(Nm - Nm.T).max() < 1e-10 * scale
        assert np.linalg.eigvalsh(0.5 * (Nm + Nm.T)).min() > 0
    w = np.linalg.eigvalsh(0.5 * ((N0 - N1) + (N0 - N1).T))
    assert w.min() > -1e-10 * scale
    assert w.max() > 1e-6 * scale


def test_lubrication_cutoff_and_intrabody():
    xi, xj = _two_body_pair(1.0 - 1e-12, 3)
    assert np.abs(O.lub_pair_matrix(xi, xj)).max() < 1e-9
    pos = np.array([[0.0, 0, 0], [2.05, 0, 0], [4.1, 0, 0]])
    # beads 0 and 1 in one body: only the (1, 2) pair contributes
    R = O.lubrication_dense(pos, np.array([0, 0, 1]), 50.0)
    assert np.abs(R[0:11, 11:22]).max() == 0.0
    assert np.abs(R[11:22, 22:33]).max() > 0.0
    assert np.abs(R[0:11, 22:33]).max() == 0.0


def test_aggregate_lubrication_psd_and_common_translation():
    pos, body, L = synth.suspension(12, 4, 0.15, 5)
    sys_ = O.assemble(pos, body, L, rlub=3.0, M=np.eye(11 * len(pos)))
    RR = sys_["RRFU"]
    assert np.abs(RR).max() > 0
    assert np.abs(RR - RR.T).max() < 1e-12 * np.abs(RR).max()
    assert np.linalg.eigvalsh(RR).min() > -1e-9 * np.abs(RR).max()
    dU = np.tile([0.3, -1.0, 0.5, 0, 0, 0], sys_["nb"])
    assert np.abs(RR @ dU).max() < 1e-9 * np.abs(RR).max()


# ----------------------------------------------------------- preconditioner


def test_preconditioner_exact_for_scalar_mobility_without_lubrication():
    # with M_inf = mu0 I exactly and no near field, the block factorisation of
    # Table 1 is the exact inverse
    pos, body, L = synth.config_doublets(n_agg=5, L=20.0, seed=2)
    Nt = len(pos)
    mu0 = 1.0 / (6 * PI)
    sys_ = O.assemble(pos, body, L, M=mu0 * np.eye(11 * Nt))
    P = O.preconditioner_dense(sys_, sys_["unw"], body, L, rp=2.1, rlub=0.0)
    assert np.abs(P @ sys_["A"] - np.eye(sys_["A"].shape[0])).max() < 1e-10


def test_preconditioner_counts_only_pairs_within_rp():
    # R~ of Table 1 holds the pairs closer than r_p (2.1a) only: moving a pair
    # that lies between r_p and the lubrication cut-off leaves P^-1 as it is,
    # moving a pair inside r_p changes it
    L = 30.0
    base = np.array([[5.0, 5, 5], [7.05, 5, 5], [5.0, 12, 5], [7.4, 12, 5]])
    body = np.array([0, 1, 2, 3])

    def P(pos):
        sys_ = O.assemble(pos, body, L, rlub=3.0, M=np.eye(11 * 4))
        return O.preconditioner_dense(sys_, sys_["unw"], body, L, rp=2.1, rlub=3.0)

    P0 = P(base)
    far = base.copy()
    far[3, 0] = 7.6  # pair (2, 3): 2.4a -> 2.6a, beyond r_p
    near = base.copy()
    near[1, 0] = 7.08  # pair (0, 1): 2.05a -> 2.08a, inside r_p
    assert np.abs(P(far) - P0).max() <= 1e-14 * np.abs(P0).max()
    assert np.abs(P(near) - P0).max() > 1e-6 * np.abs(P0).max()


def test_preconditioner_diagonal_blocks_match_per_body_solve():
    pos, body, L = synth.suspension(10, 3, 0.15, 9)
    sys_ = O.assemble(pos, body, L, rlub=3.0, M=np.eye(11 * len(pos)))
    P = O.preconditioner_dense(sys_, sys_["unw"], body, L, rp=3.0, rlub=3.0)
    # the lower-right block is -blockdiag[Sigma (zeta0 I + R) Sigma^T]^-1
    n1 = 11 * len(pos)
    z0 = 6 * PI
    big = sys_["ST"].T @ (z0 * np.eye(6 * len(pos)) + sys_["RFU"]) @ sys_["ST"]
    for J in range(sys_["nb"]):
        s = slice(6 * J, 6 * J + 6)
        blk = P[n1:, n1:][s, s]
        assert np.allclose(blk @ big[s, s], -np.eye(6), atol=1e-10)


# --------------------------------------------------------------- integrator


def test_bead_forces_balance_each_body():
    # a force-free, inertia-less aggregate carries no net load (Eq. FH_agg):
    # the far-field forces of its beads (the solution's F) and their
    # near-field forces (F^nf of the outputs), with torques about X, balance
    # the applied force and torque F^P
    pos, body, L = synth.suspension(6, 3, 0.2, 8)
    FT = synth.random_forces(6, 9)
    out = O.solve(pos, body, L, gamma=1.0, FT=FT, rlub=3.0)
    assert np.abs(out["Fnf"]).max() > 0
    r = out["system"]["r"]
    tot = np.zeros((6, 6))
    for b in range(len(pos)):
        J = body[b]
        f = out["F"][b, 0:3] + out["Fnf"][b, 0:3]
        tot[J, 0:3] += f
        tot[J, 3:6] += out["F"][b, 3:6] + out["Fnf"][b, 3:6] + np.cross(r[b], f)
    assert np.abs(tot + FT).max() < 1e-9 * np.abs(FT).max()


def test_solve_is_invariant_under_translation():
    # the periodic problem has no preferred origin: translating every bead
    # (and wrapping it into the box) leaves the disturbance velocities and
    # the stresslets unchanged; the shift puts aggregates and lubrication
    # pairs across every face of the box
    pos, body, L = synth.suspension(8, 4, 0.2, 12)
    FT = synth.random_forces(8, 13)
    a = O.solve(pos, body, L, gamma=0.8, FT=FT, rlub=3.0)
    moved = np.mod(pos + np.array([0.31, 0.47, 0.59]) * L, L)
    b = O.solve(moved, body, L, gamma=0.8, FT=FT, rlub=3.0)
    assert np.allclose(b["dU"], a["dU"], rtol=1e-9, atol=1e-12)
    assert np.allclose(b["S"], a["S"], rtol=1e-9, atol=1e-12)


def test_comoving_update_leaves_affine_motion_in_place():
    # in the co-moving frame only the disturbance motion moves a body: one
    # translating with the imposed flow at its centre, U_inf(X) = gamma X_y x,
    # and turning with Omega_inf = -gamma/2 z, stays where it is
    pos, body, L = synth.suspension(3, 4, 0.05, 2)
    unw, X, r = O.body_geometry(pos, body, L)
    q = np.tile([1.0, 0, 0, 0], (3, 1))
    g = 0.7
    U = np.zeros((3, 6))
    U[:, 0] = g * X[:, 1]
    U[:, 5] = -0.5 * g
    X2, q2, _ = O.integrate(X, q, r, body, U, 0.1, comoving_gamma=g)
    assert np.allclose(X2, X, rtol=0, atol=1e-14) and np.allclose(q2, q, rtol=0, atol=1e-14)


def test_integrator_keeps_bodies_rigid_and_quaternions_unit():
    rng = np.random.default_rng(6)
    pos, body, L = synth.suspension(5, 6, 0.05, 4)
    unw, X, r = O.body_geometry(pos, body, L)
    q = np.tile([1.0, 0, 0, 0], (5, 1))
    d0 = [np.linalg.norm(r[body == J][:, None] - r[body == J][None], axis=-1) for J in range(5)]
    for _ in range(100):
        U = rng.normal(size=(5, 6))
        X, q, x = O.integrate(X, q, r, body, U, 1e-2)
    assert np.allclose(np.linalg.norm(q, axis=1), 1.0, atol=1e-14)
    for J in range(5):
        xb = x[body == J]
        d = np.linalg.norm(xb[:, None] - xb[None], axis=-1)
        assert np.abs(d - d0[J]).max() < 1e-12
        assert np.allclose(xb.mean(axis=0), X[J], atol=1e-12)


def test_integrator_rotation_angle():
    # constant Omega about z for time T rotates the body by Omega T (O(dt) error)
    r = np.array([[1.0, 0, 0], [-1.0, 0, 0]])
    X = np.zeros((1, 3))
    q = np.array([[1.0, 0, 0, 0]])
    U = np.array([[0, 0, 0, 0, 0, 0.5]])
    for _ in range(1000):
        X, q, x = O.integrate(X, q, r, np.array([0, 0]), U, 1e-3)
    ang = np.arctan2(x[0, 1], x[0, 0])
    assert abs(ang - 0.5) < 1e-4


def test_integrator_rotates_in_the_lab_frame():
    # Omega is a lab-frame angular velocity: from the orientation q0 (90
    # degrees about x) a constant Omega along lab z turns the body about lab z,
    # R(t) = R_z(Omega t) R(q0), not about the body's own z axis.  A dimer
    # along body z points along lab -y at t = 0 and along
    # (sin theta, -cos theta, 0) after theta = Omega t.
    r = np.array([[0, 0, 1.0], [0, 0, -1.0]])
    X = np.zeros((1, 3))
    q = np.array([[np.cos(PI / 4), np.sin(PI / 4), 0, 0]])
    U = np.array([[0, 0, 0, 0, 0, 0.5]])
    _, _, x = O.integrate(X, q, r, np.array([0, 0]), np.zeros((1, 6)), 1e-3)
    assert np.allclose(x[0], [0, -1.0, 0], atol=1e-12)
    for _ in range(1000):
        X, q, x = O.integrate(X, q, r, np.array([0, 0]), U, 1e-3)
    th = 0.5
    assert np.abs(x[0] - [np.sin(th), -np.cos(th), 0]).max() < 2e-4


# ------------------------------------------------------- sampled-row helpers


def test_sampled_real_rows_equal_dense_rows():
    rng = np.random.default_rng(31)
    pos, body, L = synth.suspension(6, 4, 0.1, 7)
    xi, rc = 1.0, 2.0 + np.sqrt(46.0) / 1.0
    rc = min(rc, 0.49 * L)
    F = rng.normal(size=(len(pos), 11))
    dense = O.mobility_real_dense(pos, L, xi, rc).reshape(11 * len(pos), -1) @ F.reshape(-1)
    rows = [0, 5, len(pos) - 1]
    got = O.mobility_real_rows(pos, L, xi, rc, rows, F)
    assert np.allclose(got, dense.reshape(-1, 11)[rows], rtol=0, atol=1e-14 * np.abs(dense).max())


def test_sampled_lubrication_rows_equal_dense():
    rng = np.random.default_rng(32)
    pos, body, L = synth.suspension(12, 4, 0.15, 5)
    sys_ = O.assemble(pos, body, L, rlub=3.0, M=np.eye(11 * len(pos)))
    dU = rng.normal(size=(sys_["nb"], 6))
    dense = (sys_["RRFU"] @ dU.reshape(-1)).reshape(-1, 6)
    bodies = [0, 3, 11]
    got = O.lubrication_rows(pos, body, L, bodies, dU)
    assert np.allclose(got, dense[bodies], rtol=0, atol=1e-12 * np.abs(dense).max())


# ------------------------------------------------ reciprocity and the strain columns


def test_aggregate_reciprocity_of_velocity_and_stresslet():
    """Lorentz reciprocity of the aggregate grand mobility (Sec. 2.1 grand
    resistance convention, Eq. FH_agg, Eq. stress_comp a and d).  Eliminating
    F from (F; S) = R (U_inf - U; E) gives U - U_inf = R_FU^-1 (F^P + R_FE E)
    and S = -R_SU R_FU^-1 F^P + ..., with R_SU = R_FE^T, so the disturbance
    velocity per unit shear rate of body J equals minus the derivative of the
    suspension's total S_xy (hydrodynamic plus constraint parts) with respect
    to the applied force and torque on J.  Lubricated multi-bead bodies make
    both the lever-arm (constraint) stresslet and the near-field strain terms
    enter."""
    pos, body, L = synth.suspension(6, 3, 0.2, 11)
    body = np.asarray(body)
    nb = int(body.max()) + 1
    unw = O.body_geometry(pos, body, L)[0]
    assert np.abs(O.lubrication_dense(unw, body, L, rcut=3.0)).max() > 0.0  # near pairs present
    M = O.mobility_dense(unw, L)
    out = O.solve(pos, body, L, gamma=1.0, FT=np.zeros((nb, 6)), rlub=3.0, M=M)
    A = out["dU"]
    Bm = np.zeros((nb, 6))
    for J in range(nb):
        for k in range(6):
            FT = np.zeros((nb, 6))
            FT[J, k] = 1.0
            o = O.solve(pos, body, L, gamma=0.0, FT=FT, rlub=3.0, M=M)
            Bm[J, k] = o["S"][:, 0, 1].sum()
    # the constraint part is not negligible in this check
    assert np.abs(out["SC"]).max() > 0.05 * np.abs(out["S"]).max()
    assert np.linalg.norm(A + Bm) < 1e-10 * np.linalg.norm(A)


@pytest.mark.parametrize("gap", [1e-3, 0.07, 0.6])
def test_lubrication_strain_columns_equal_affine_bead_motion(gap):
    """The pair model (a dissipation form of the pair's relative surface
    velocity and relative rotation) sees an imposed strain E only through
    s = r E.n, which is exactly what the beads would see moving with
    nu = -E.x_b in still fluid (s = nu_i - nu_j): R (0, E) = R (-E x, 0) on
    every force and stresslet row."""
    rng = np.random.default_rng(int(gap * 1e4) + 5)
    xi, xj = _two_body_pair(gap, 7)
    xi = xi + rng.normal(size=3)
    xj = xj + (xi - np.zeros(3))
    R = O.lub_pair_matrix(xi, xj)
    for _ in range(3):
        E = rng.normal(size=(3, 3))
        E = 0.5 * (E + E.T)
        E -= np.trace(E) / 3.0 * np.eye(3)
        e5 = O.sym_to_vec5(E)
        nu_strain = np.zeros(22)
        nu_strain[6:11] = e5
        nu_strain[17:22] = e5
        nu_move = np.zeros(22)
        nu_move[0:3] = -E @ xi
        nu_move[11:14] = -E @ xj
        f1 = R @ nu_strain
        f2 = R @ nu_move
        assert np.abs(f1).max() > 1e-3 * np.abs(R).max() * np.abs(E).max()
        assert np.abs(f1 - f2).max() < 1e-12 * np.abs(R).max() * np.abs(E).max() * 4.0


# ------------------------------------------------- surface roughness (Sec. 4)


def test_roughness_enhances_only_the_tangential_modes_below_h0():
    rough = (0.01, 0.01)
    for h in (1e-3, 3e-3, 6e-3, 0.0099):
        A0, B0, D0 = O.lub_coefficients(h)
        A1, B1, D1 = O.lub_coefficients(h, rough=rough)
        assert A1 == A0  # squeeze untouched
        assert B1 > B0 and D1 > D0
        # the sliding and rolling increments are in the ratio of the two
        # normalisations, 6 pi eta a and 8 pi eta a^3
        assert abs((D1 - D0) / (B1 - B0) - 8.0 / 6.0) < 1e-12
    for h in (0.01, 0.02, 0.5):
        assert O.lub_coefficients(h, rough=rough) == O.lub_coefficients(h)
    # continuous at the asperity height
    below = O.lub_coefficients(0.01 * (1 - 1e-9), rough=rough)[1]
    assert abs(below - O.lub_coefficients(0.01)[1]) < 1e-6


def test_roughness_diverges_as_one_over_the_gap():
    # f(h) ~ alpha a / h as h -> 0: h (B_rough - B_smooth) -> 6 pi eta a alpha a
    alpha, h0 = 0.01, 0.01
    vals = []
    for h in (4e-3, 2e-3, 1e-3):
        dB = O.lub_coefficients(h, rough=(alpha, h0))[1] - O.lub_coefficients(h)[1]
        vals.append(h * dB / (6 * PI * alpha))
    # approaches 1 (in units of a) with corrections O(h / h0)
    assert vals[0] < vals[1] < vals[2] < 1.0 + 1e-12 and vals[2] > 0.69


@pytest.mark.parametrize("gap", [1e-3, 0.004, 0.02])
def test_rough_pair_symmetric_psd_and_rigid_invariant(gap):
    xi, xj = _two_body_pair(gap, 4)
    R = O.lub_pair_matrix(xi, xj, rough=(0.01, 0.01))
    assert np.abs(R - R.T).max() < 1e-12 * np.abs(R).max()
    assert np.linalg.eigvalsh(R).min() > -1e-10 * np.abs(R).max()
    rng = np.random.default_rng(5)
    V, W = rng.normal(size=3), rng.normal(size=3)
    c = 0.5 * (xi + xj)
    nu = np.zeros(22)
    for k, x in ((0, xi), (11, xj)):
        nu[k:k + 3] = -(V + np.cross(W, x - c))
        nu[k + 3:k + 6] = -W
    assert np.abs(R @ nu).max() < 1e-9 * np.abs(R).max()
