"""Plain FP64 CPU oracle for the rigid-aggregate FSD saddle-point solve.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline legs of bench.py, never by the product path.

What it computes (paper: Sec. 2.3, Eq. spm_agg, Algorithm 1 steps 1, 4, 5):
the aggregate saddle-point system

    [ M_inf        B Sigma^T ] [ F      ]   [ (E.(x-X) ; 0) ; E     ]
    [ Sigma B^T   -RR_FU^nf  ] [ U-U_inf] = [ -(FF^P + RR_FE^nf:E)   ]

with u^B = 0 and F^B = 0, assembled as ONE dense matrix and solved by LAPACK
(numpy.linalg.solve).  Its ingredients are plain definitions:

* M_inf: the periodic FTS-level Rotne-Prager-Yamakawa mobility (force, torque
  and stresslet sources; velocity, rotation and strain read-outs).  It is the
  Ewald sum of one k-space kernel (Sec. 2.2; the same Hasimoto split that PSE
  uses, Eq. UBff): a real-space image sum plus an explicit wave-vector sum.
  The result does not depend on the splitting parameter; the oracle picks its
  own.  No grid, no FFT, no Gaussian spreading.
* R_nf: the dense bead-level near-field resistance over bead pairs on
  different bodies closer than the lubrication cut-off (Alg. 1 step 1).
* Sigma: the rigid-body constraint of Eq. gc / Eq. sigma.

Readings of points where the paper is silent:
* E.(x - X) on the bead rows (Eq. spm_agg; the table's X - x is a typo).
* FTS source/read-out factors: j0(ka) for force / velocity, 3 j1(ka)/(ka)
  for torque, stresslet / rotation, strain.
* Stresslet / strain in an orthonormal 5-component basis (so M_inf is
  symmetric).
* Free-space pairs closer than 2a are evaluated at separation 2a along their
  true direction ("clamp").
* Near-field pair resistance: a dissipation form built from the leading
  two-sphere lubrication terms (squeeze 1/eps + log, sliding log, rolling
  log), shifted to vanish at the cut-off.
* Stresslet returned: S^H + S^C (Eq. stress_comp a, d), with F^C the
  negative total bead force.

Parity pins: tests/test_oracle_*.py; tests/test_oracle_pin_sensitivity.py
plants mistakes in a copy of this source and checks that the pins catch them.
One value is parity unpinned: the rolling coefficient of the pair model,
8 pi eta a^3 (1/10) ln(1/eps) in lub_coefficients (a reading of functions the
paper does not print; the two-sphere rotation functions it stands in for are
not of the dissipation form's shape, so no published number fixes it, and a
changed value passes every pin).  Everything else is pinned.
"""

import numpy as np
from numpy.polynomial.legendre import leggauss
from scipy.special import spherical_jn

PI = np.pi

# ---------------------------------------------------------------------------
# index tensors
# ---------------------------------------------------------------------------


def levi_civita():
    e = np.zeros((3, 3, 3))
    e[0, 1, 2] = e[1, 2, 0] = e[2, 0, 1] = 1.0
    e[0, 2, 1] = e[2, 1, 0] = e[1, 0, 2] = -1.0
    return e


def strain_basis():
    """Orthonormal basis E_m (m = 0..4) of symmetric traceless 3x3 matrices.

    A stresslet / strain is stored as its 5 coordinates s_m = E_m : S, so
    S : E = sum_m s_m e_m (Sec. 2.1: the reduced 5N space of stresslets / strains)."""
    E = np.zeros((5, 3, 3))
    s2, s6 = np.sqrt(2.0), np.sqrt(6.0)
    E[0, 0, 0], E[0, 1, 1] = 1 / s2, -1 / s2
    E[1, 0, 0], E[1, 1, 1], E[1, 2, 2] = -1 / s6, -1 / s6, 2 / s6
    E[2, 0, 1] = E[2, 1, 0] = 1 / s2
    E[3, 0, 2] = E[3, 2, 0] = 1 / s2
    E[4, 1, 2] = E[4, 2, 1] = 1 / s2
    return E


EPS = levi_civita()
EB = strain_basis()
I3 = np.eye(3)

# Faxen coefficients of the two source / read-out kinds: surface average
# (monopole: j0(ka) = 1 - (ka)^2/6 + ...) and volume average (dipole:
# 3 j1(ka)/(ka) = 1 - (ka)^2/10 + ...).
FAXEN_C = {"M": 1.0 / 6.0, "D": 1.0 / 10.0}
PAIR_KINDS = ("MM", "MD", "DD")


def sym_to_vec5(S):
    """3x3 (..., 3, 3) -> 5 basis coordinates (projects out trace / skew)."""
    return np.einsum("mab,...ab->...m", EB, S)


def vec5_to_sym(s):
    return np.einsum("mab,...m->...ab", EB, s)


# ---------------------------------------------------------------------------
# radial scalar functions
# ---------------------------------------------------------------------------
#
# Every 11x11 mobility block is a set of derivatives of ONE radial scalar
# Phi_st(r) per (source kind, read-out kind) pair, with
#     Phi_hat(k) = - W(k) f_s(ka) f_t(ka) / (eta k^4)
# (so that (I lap - grad grad) Phi is the Oseen-type velocity kernel).  W = 1
# for the free-space kernel, W = H(k, xi) (Hasimoto) for the wave part and
# 1 - H for the real part.  We need Phi_n := (r^-1 d/dr)^n Phi, n = 1..4.


def _laurent_D(poly):
    """(1/r d/dr) applied to sum_p c_p r^p  ->  sum_p p c_p r^(p-2)."""
    return {p - 2: p * c for p, c in poly.items() if p != 0 and c != 0.0}


def free_phi_n(r, kind, a=1.0, eta=1.0):
    """Phi_n, n=1..4, of the free-space kernel for r >= 2a.

    For non-overlapping spheres the Faxen operators act exactly on the
    biharmonic r/(8 pi eta):  Phi = (1 + c_s a^2 lap)(1 + c_t a^2 lap) r/(8 pi eta)
    = (r + 2 (c_s + c_t) a^2 / r) / (8 pi eta), since lap^2 r = 0 for r > 0.
    Returns array (..., 4)."""
    c = FAXEN_C[kind[0]] + FAXEN_C[kind[1]]
    poly = {1: 1.0 / (8 * PI * eta), -1: 2 * c * a * a / (8 * PI * eta)}
    r = np.asarray(r, dtype=np.float64)
    out = np.empty(r.shape + (4,))
    for n in range(4):
        poly = _laurent_D(poly)
        out[..., n] = sum(cp * r ** p for p, cp in poly.items())
    return out


def jn_over_zn(n, z):
    """j_n(z) / z^n, with the power series near z = 0 (no cancellation)."""
    z = np.asarray(z, dtype=np.float64)
    out = np.empty_like(z)
    small = z < 2.0
    zs = z[small]
    # sum_k (-z^2/2)^k / (k! (2n+2k+1)!!)
    dfact = 1.0
    for m in range(1, 2 * n + 2, 2):
        dfact *= m
    term = np.full_like(zs, 1.0 / dfact)
    acc = term.copy()
    for k in range(1, 30):
        term = term * (-(zs * zs) / 2.0) / (k * (2 * n + 2 * k + 1))
        acc = acc + term
    out[small] = acc
    zl = z[~small]
    out[~small] = spherical_jn(n, zl) / zl ** n
    return out


def form_factor(kind, z):
    """j0(z) for a monopole, 3 j1(z)/z for a dipole."""
    if kind == "M":
        return jn_over_zn(0, z)
    return 3.0 * jn_over_zn(1, z)


def hasimoto(k, xi):
    """H(k, xi) = (1 + k^2/(4 xi^2)) exp(-k^2/(4 xi^2)) (the PSE / Hasimoto split)."""
    x = k * k / (4.0 * xi * xi)
    return (1.0 + x) * np.exp(-x)


def wave_phi_n(r, kind, xi, a=1.0, eta=1.0, nq=320):
    """Phi_n, n=1..4, of the WAVE part (W = H) in free space, any r >= 0.

    (r^-1 d/dr)^n j0(kr) = (-k^2)^n j_n(kr)/(kr)^n gives
        Phi_n(r) = (-1)^(n+1) / (2 pi^2 eta) int_0^inf H f_s f_t k^(2n-2) j_n(kr)/(kr)^n dk
    evaluated by Gauss-Legendre on [0, K], H(K) < 1e-18."""
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    K = 2.0 * xi * np.sqrt(46.0)
    t, w = leggauss(nq)
    k = 0.5 * K * (t + 1.0)
    w = 0.5 * K * w
    g = hasimoto(k, xi) * form_factor(kind[0], k * a) * form_factor(kind[1], k * a)
    kr = np.outer(r, k)
    out = np.empty(r.shape + (4,))
    for n in range(1, 5):
        integrand = g * k ** (2 * n - 2) * jn_over_zn(n, kr)
        out[:, n - 1] = (-1.0) ** (n + 1) / (2 * PI * PI * eta) * (integrand @ w)
    return out


def free_phi_n_quadrature(r, kind, a=1.0, eta=1.0, kmax=4000.0, nq=200000):
    """Phi_n of the FREE kernel by brute 1D quadrature of its k-space
    definition (W = 1), for pins only: slow and ~1e-7 accurate."""
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    k = (np.arange(nq) + 0.5) * (kmax / nq)
    w = kmax / nq
    g = form_factor(kind[0], k * a) * form_factor(kind[1], k * a)
    out = np.empty(r.shape + (4,))
    for i, ri in enumerate(r):
        for n in range(1, 5):
            integrand = g * k ** (2 * n - 2) * jn_over_zn(n, k * ri)
            out[i, n - 1] = (-1.0) ** (n + 1) / (2 * PI * PI * eta) * integrand.sum() * w
    return out


def self_mobilities(a=1.0, eta=1.0):
    """Isolated-sphere self mobilities: translation 1/(6 pi eta a), rotation
    1/(8 pi eta a^3), strain-stresslet 3/(20 pi eta a^3) (per orthonormal
    strain component; a free sphere in strain E carries S = (20/3) pi eta a^3 E)."""
    return 1.0 / (6 * PI * eta * a), 1.0 / (8 * PI * eta * a ** 3), 3.0 / (20 * PI * eta * a ** 3)


def self_block(a=1.0, eta=1.0):
    mt, mr, ms = self_mobilities(a, eta)
    return np.diag([mt] * 3 + [mr] * 3 + [ms] * 5)


# ---------------------------------------------------------------------------
# 11x11 blocks from radial derivatives
# ---------------------------------------------------------------------------


def _derivative_tensors(x, ph):
    """Cartesian derivative tensors of a radial function.

    With Phi_n = (r^-1 d/dr)^n Phi and x the separation vector:
      d_a Phi        = Phi_1 x_a
      d_ab Phi       = Phi_2 x_a x_b + Phi_1 delta_ab
      d_abc Phi      = Phi_3 xxx + Phi_2 (delta x, 3 terms)
      d_abcd Phi     = Phi_4 xxxx + Phi_3 (delta xx, 6 terms) + Phi_2 (delta delta, 3 terms)
    x: (P, 3); ph: (P, 4).  Returns D2 (P,3,3), D3 (P,3,3,3), D4 (P,3,3,3,3)."""
    p1, p2, p3, p4 = ph[:, 0], ph[:, 1], ph[:, 2], ph[:, 3]
    d = I3
    xx = np.einsum("pa,pb->pab", x, x)
    D2 = p2[:, None, None] * xx + p1[:, None, None] * d
    xxx = np.einsum("pab,pc->pabc", xx, x)
    dx = (np.einsum("ab,pc->pabc", d, x) + np.einsum("ac,pb->pabc", d, x)
          + np.einsum("bc,pa->pabc", d, x))
    D3 = p3[:, None, None, None] * xxx + p2[:, None, None, None] * dx
    xxxx = np.einsum("pab,pcd->pabcd", xx, xx)
    dxx = (np.einsum("ab,pcd->pabcd", d, xx) + np.einsum("ac,pbd->pabcd", d, xx)
           + np.einsum("ad,pbc->pabcd", d, xx) + np.einsum("bc,pad->pabcd", d, xx)
           + np.einsum("bd,pac->pabcd", d, xx) + np.einsum("cd,pab->pabcd", d, xx))
    dd = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
          + np.einsum("ad,bc->abcd", d, d))
    D4 = (p4[:, None, None, None, None] * xxxx + p3[:, None, None, None, None] * dxx
          + p2[:, None, None, None, None] * dd[None])
    return D2, D3, D4


def _kernel_tensors(x, ph):
    """T = (I lap - grad grad) Phi and its first / second derivatives:
    T[p,a,b], dT[p,a,b,c] = d_c T_ab, ddT[p,a,b,c,d] = d_c d_d T_ab."""
    D2, D3, D4 = _derivative_tensors(x, ph)
    lap = np.einsum("paa->p", D2)
    glap = np.einsum("paac->pc", D3)
    hlap = np.einsum("paacd->pcd", D4)
    T = lap[:, None, None] * I3 - D2
    dT = np.einsum("ab,pc->pabc", I3, glap) - D3
    ddT = np.einsum("ab,pcd->pabcd", I3, hlap) - D4
    return T, dT, ddT


def blocks_from_phi(x, phMM, phMD, phDD):
    """The 11x11 mobility blocks (rows: u, omega, e5; cols: F, L, S5) for
    separation x = x_target - x_source, given the radial derivatives of the
    three kernels.  Sources in k-space: F f_M + (i/2) f_D k x L - i f_D S.k;
    read-outs: f_M u, f_D (1/2) curl u, f_D sym grad u; ik <-> grad_x.
    x: (P,3).  Returns (P, 11, 11)."""
    x = np.atleast_2d(x)
    P = x.shape[0]
    T_MM, _, _ = _kernel_tensors(x, phMM)
    _, dT_MD, _ = _kernel_tensors(x, phMD)
    _, _, ddT = _kernel_tensors(x, phDD)
    M = np.zeros((P, 11, 11))
    M[:, 0:3, 0:3] = T_MM
    M[:, 0:3, 3:6] = 0.5 * np.einsum("bcd,pabc->pad", EPS, dT_MD)
    M[:, 0:3, 6:11] = -np.einsum("pabc,mbc->pam", dT_MD, EB)
    M[:, 3:6, 0:3] = 0.5 * np.einsum("aef,pfbe->pab", EPS, dT_MD)
    M[:, 3:6, 3:6] = 0.25 * np.einsum("aef,bcd,pfbec->pad", EPS, EPS, ddT)
    M[:, 3:6, 6:11] = -0.5 * np.einsum("aef,pfbec,mbc->pam", EPS, ddT, EB)
    M[:, 6:11, 0:3] = np.einsum("mae,pabe->pmb", EB, dT_MD)
    M[:, 6:11, 3:6] = 0.5 * np.einsum("mae,bcd,pabec->pmd", EB, EPS, ddT)
    M[:, 6:11, 6:11] = -np.einsum("mae,pabec,nbc->pmn", EB, ddT, EB)
    return M


def free_blocks(x, a=1.0, eta=1.0):
    """Free-space FTS-RPY pair blocks; separations below 2a are clamped to
    2a along their own direction (reading for overlaps)."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    r = np.linalg.norm(x, axis=1)
    reff = np.maximum(r, 2.0 * a)
    xe = x * (reff / r)[:, None]
    ph = {k: free_phi_n(reff, k, a, eta) for k in PAIR_KINDS}
    return blocks_from_phi(xe, ph["MM"], ph["MD"], ph["DD"])


def wave_blocks_free(x, xi, a=1.0, eta=1.0, nq=320):
    """Wave (H-filtered) part of the free-space kernel at separations x."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    r = np.linalg.norm(x, axis=1)
    ph = {k: wave_phi_n(r, k, xi, a, eta, nq) for k in PAIR_KINDS}
    return blocks_from_phi(x, ph["MM"], ph["MD"], ph["DD"])


# ---------------------------------------------------------------------------
# periodic mobility by Ewald summation
# ---------------------------------------------------------------------------


def source_operator(k, a=1.0):
    """Q(k), 3x11 complex: g_hat = Q(k) . (F, L, S5) for a sphere at the origin.
    k: (K, 3) -> (K, 3, 11)."""
    kn = np.linalg.norm(k, axis=1)
    fM = form_factor("M", kn * a)
    fD = form_factor("D", kn * a)
    Q = np.zeros((k.shape[0], 3, 11), dtype=np.complex128)
    Q[:, :, 0:3] = fM[:, None, None] * I3
    kx = np.einsum("abc,pb->pac", EPS, k)  # (k x L)_a = eps_abc k_b L_c
    Q[:, :, 3:6] = 0.5j * fD[:, None, None] * kx
    Q[:, :, 6:11] = -1j * fD[:, None, None] * np.einsum("mab,pb->pam", EB, k)
    return Q


def oracle_split(L):
    """Splitting chosen by the oracle for a box of side L: real-space tail and
    wave-space tail both below ~1e-17 relative."""
    xi = max(6.5 / L, 0.08)
    rc = 2.0 + np.sqrt(46.0) / xi
    kmax = 2.0 * xi * np.sqrt(46.0)
    return xi, rc, kmax


def min_image(d, L, tilt=0.0):
    """Nearest periodic image of displacements d (..., 3) in a Lees-Edwards
    box of side L whose image across y is offset by `tilt` along x (tilt 0:
    the cubic box): wrap y first (shifting x by the offset), then x and z."""
    d = np.array(d, dtype=np.float64, copy=True)
    ny = np.round(d[..., 1] / L)
    d[..., 0] -= ny * tilt
    d[..., 1] -= ny * L
    d[..., 0] -= L * np.round(d[..., 0] / L)
    d[..., 2] -= L * np.round(d[..., 2] / L)
    return d


def _lattice(nmax):
    g = np.arange(-nmax, nmax + 1)
    return np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)


def mobility_real_dense(pos, L, xi, rc, a=1.0, eta=1.0, tilt=0.0):
    """Real-space Ewald part + self term, dense (N, 11, N, 11).  Images at
    n1 e1 + n2 e2 + n3 e3 with e1 = (L, 0, 0), e2 = (tilt, L, 0), e3 = (0, 0, L)
    (a Lees-Edwards box; tilt 0 the cube)."""
    pos = np.asarray(pos, dtype=np.float64)
    N = pos.shape[0]
    M = np.zeros((N, 11, N, 11))
    nimg = int(np.ceil(rc / L)) + 2
    lat = _lattice(nimg).astype(np.float64)
    shifts = lat * L
    shifts[:, 0] += lat[:, 1] * tilt
    for i in range(N):
        d = pos[i][None, :] - pos  # x_i - x_j
        x = (d[:, None, :] + shifts[None, :, :]).reshape(-1, 3)
        jj = np.repeat(np.arange(N), shifts.shape[0])
        r = np.linalg.norm(x, axis=1)
        keep = (r < rc) & (r > 0.0)
        x, jj, r = x[keep], jj[keep], r[keep]
        if x.shape[0] == 0:
            continue
        blk = free_blocks(x, a, eta) - wave_blocks_free(x, xi, a, eta)
        acc = np.zeros((N, 11, 11))
        np.add.at(acc, jj, blk)
        M[i] += acc.transpose(1, 0, 2)
    w0 = wave_blocks_free(np.zeros((1, 3)), xi, a, eta)[0]
    selfb = self_block(a, eta) - w0
    for i in range(N):
        M[i, :, i, :] += selfb
    return M


def wave_vectors(L, kmax, tilt=0.0):
    """Half of the reciprocal lattice within kmax.  For the Lees-Edwards box
    (lattice e1 = (L, 0, 0), e2 = (tilt, L, 0), e3 = (0, 0, L)) the
    reciprocal vectors are k = (2 pi / L) (n1, n2 - (tilt/L) n1, n3)."""
    tau = tilt / L
    nmax = int(np.ceil(kmax * L / (2 * PI) * (1.0 + abs(tau)))) + 1
    n = _lattice(nmax)
    # half space: first nonzero component positive
    first = np.where(n[:, 0] != 0, n[:, 0], np.where(n[:, 1] != 0, n[:, 1], n[:, 2]))
    n = n[first > 0].astype(np.float64)
    n[:, 1] -= tau * n[:, 0]
    k = 2 * PI * n / L
    kn = np.linalg.norm(k, axis=1)
    return k[kn <= kmax]


def mobility_wave_dense(pos, L, xi, kmax, a=1.0, eta=1.0, tilt=0.0):
    """Wave-space Ewald part, dense: (1/V) sum_{k != 0} e^{ik.(x_i-x_j)}
    Q^H (I - kk) Q H(k,xi)/(eta k^2).  The k = 0 mode is excluded (mean force
    balanced by the mean pressure gradient)."""
    pos = np.asarray(pos, dtype=np.float64)
    N = pos.shape[0]
    k = wave_vectors(L, kmax, tilt)
    kn = np.linalg.norm(k, axis=1)
    kh = k / kn[:, None]
    Q = source_operator(k, a)
    Pk = I3[None] - np.einsum("pa,pb->pab", kh, kh)
    A = np.einsum("pas,pab,pbt->pst", Q.conj(), Pk, Q)
    w = 2.0 * hasimoto(kn, xi) / (eta * kn * kn) / L ** 3  # x2: +k and -k
    Ar = A.real * w[:, None, None]
    Ai = A.imag * w[:, None, None]
    ph = k @ pos.T  # (K, N)
    C, S = np.cos(ph), np.sin(ph)
    M = np.zeros((N, 11, N, 11))
    for s in range(11):
        for t in range(11):
            ar, ai = Ar[:, s, t], Ai[:, s, t]
            M[:, s, :, t] = ((C * ar[:, None]).T @ C + (S * ar[:, None]).T @ S
                             - (S * ai[:, None]).T @ C + (C * ai[:, None]).T @ S)
    return M


def mobility_wave_apply(pos, F, L, xi, kmax, a=1.0, eta=1.0, tilt=0.0, chunk=100000):
    """The wave-space Ewald sum of `mobility_wave_dense` applied to moments
    F (N, 11) without forming the matrix:
        u_i = (1/V) sum_{k != 0} H(k,xi)/(eta k^2) e^{ik.x_i} Q(k)^H (I - kk)
              sum_j Q(k) e^{-ik.x_j} F_j
    over the half lattice (x2 and the real part for -k), in chunks of k.
    Returns (N, 11).  For boxes whose wave-vector count makes the dense
    matrix impractical (a 144^3-point grid's range of k)."""
    pos = np.asarray(pos, dtype=np.float64)
    F = np.asarray(F, dtype=np.float64).reshape(len(pos), 11)
    k_all = wave_vectors(L, kmax, tilt)
    u = np.zeros((len(pos), 11))
    for c0 in range(0, k_all.shape[0], chunk):
        k = k_all[c0:c0 + chunk]
        kn = np.linalg.norm(k, axis=1)
        kh = k / kn[:, None]
        Q = source_operator(k, a)
        ph = k @ pos.T  # (K, N)
        rho = np.exp(-1j * ph) @ F  # sum_j e^{-ik.x_j} F_j: (K, 11)
        g = np.einsum("pat,pt->pa", Q, rho)
        g = g - kh * np.einsum("pa,pa->p", kh, g)[:, None]  # (I - kk) g
        v = np.einsum("pas,pa->ps", Q.conj(), g)
        w = 2.0 * hasimoto(kn, xi) / (eta * kn * kn) / L ** 3
        u += (np.exp(1j * ph).T @ (v * w[:, None])).real
    return u


def mobility_dense(pos, L, a=1.0, eta=1.0, xi=None, tilt=0.0):
    """Periodic FTS mobility M_inf, dense (11N x 11N), bead-major (a
    Lees-Edwards box when tilt != 0)."""
    xo, rc, kmax = oracle_split(L)
    if xi is not None:
        xo = xi
        rc = 2.0 + np.sqrt(46.0) / xo
        kmax = 2.0 * xo * np.sqrt(46.0)
    N = len(pos)
    M = (mobility_real_dense(pos, L, xo, rc, a, eta, tilt)
         + mobility_wave_dense(pos, L, xo, kmax, a, eta, tilt))
    return M.reshape(11 * N, 11 * N)


# ---------------------------------------------------------------------------
# geometry, imposed flow, constraint
# ---------------------------------------------------------------------------


def body_geometry(pos, body, L, tilt=0.0):
    """Bead positions unwrapped per body (minimum image about the body's first
    bead), body centroids X (equal bead masses: the 'centre of mass', Sec. 2.3.1)
    and lever arms r_b = x_b - X_J."""
    pos = np.asarray(pos, dtype=np.float64)
    body = np.asarray(body)
    nb = int(body.max()) + 1
    unw = pos.copy()
    X = np.zeros((nb, 3))
    for J in range(nb):
        idx = np.nonzero(body == J)[0]
        ref = pos[idx[0]]
        d = min_image(pos[idx] - ref, L, tilt)
        unw[idx] = ref + d
        X[J] = unw[idx].mean(axis=0)
    r = unw - X[body]
    return unw, X, r


def shear_flow(gamma):
    """Simple shear, flow along x, gradient along y (Sec. 3.1.1): u_inf = gamma y x,
    E_inf = gamma/2 (xy + yx), Omega_inf = -gamma/2 z."""
    E = np.zeros((3, 3))
    E[0, 1] = E[1, 0] = 0.5 * gamma
    Om = np.array([0.0, 0.0, -0.5 * gamma])
    return E, Om


def sigma_T(r, body, nb):
    """Sigma^T (6 Nt x 6 N): (U, Omega)_J -> (U + Omega x r_b, Omega) (Eq. sigma)."""
    Nt = r.shape[0]
    ST = np.zeros((6 * Nt, 6 * nb))
    for b in range(Nt):
        J = body[b]
        ST[6 * b:6 * b + 3, 6 * J:6 * J + 3] = I3
        ST[6 * b + 3:6 * b + 6, 6 * J + 3:6 * J + 6] = I3
        # Omega x r = -r x Omega = -[r]x Omega;  [r]x_ac = eps_abc r_b
        ST[6 * b:6 * b + 3, 6 * J + 3:6 * J + 6] = -np.einsum("abc,b->ac", EPS, r[b])
    return ST


def B_op(Nt):
    """B (11 Nt x 6 Nt): (U, Omega) -> (U, Omega, 0) per bead."""
    Bm = np.zeros((11 * Nt, 6 * Nt))
    for b in range(Nt):
        Bm[11 * b:11 * b + 6, 6 * b:6 * b + 6] = np.eye(6)
    return Bm


# ---------------------------------------------------------------------------
# near-field lubrication resistance (inter-body pairs)
# ---------------------------------------------------------------------------


def lub_coefficients(h, a=1.0, eta=1.0, rcut=3.0, hmin=1e-3, rough=(0.0, 0.0)):
    """Pair resistance coefficients as functions of the surface gap h
    (eps = h/a, clamped below at hmin/a), each shifted to vanish at the
    cut-off gap eps_c = rcut/a - 2:
      A (squeeze)        6 pi eta a [1/(4 eps) + (9/40) ln(1/eps)]
      B (sliding)        6 pi eta a (1/6) ln(1/eps)
      D (relative roll)  8 pi eta a^3 (1/10) ln(1/eps)
    (leading two-sphere lubrication terms for equal spheres).  All >= 0 for
    eps <= eps_c, so the pair form is positive semi-definite.

    rough = (alpha, h0), alpha > 0: surface roughness (Sec. 4, Eq. tan_fric):
    below the asperity height h0 the tangential coefficients gain
    f(h) = alpha (a/h0) (h0/h - 3 h/h0 + 2 h^2/h0^2) (h the clamped gap),
    B += 6 pi eta a f and D += 8 pi eta a^3 f: sliding and rolling resist
    O(1/h) instead of O(ln 1/h); the squeeze term is unchanged."""
    ec = rcut / a - 2.0
    e = max(h / a, hmin / a)

    def sq(x):
        return 1.0 / (4.0 * x) + (9.0 / 40.0) * np.log(1.0 / x)

    A = 6 * PI * eta * a * (sq(e) - sq(ec))
    B = 6 * PI * eta * a * (1.0 / 6.0) * np.log(ec / e)
    D = 8 * PI * eta * a ** 3 * 0.1 * np.log(ec / e)
    alpha, h0 = rough
    hc = e * a
    if alpha > 0.0 and h0 > 0.0 and hc < h0:
        f = alpha * (a / h0) * (h0 / hc - 3.0 * hc / h0 + 2.0 * hc * hc / (h0 * h0))
        B += 6 * PI * eta * a * f
        D += 8 * PI * eta * a ** 3 * f
    return A, B, D


def lub_pair_matrix(xi, xj, a=1.0, eta=1.0, rcut=3.0, hmin=1e-3, rough=(0.0, 0.0)):
    """22x22 grand resistance of one inter-body pair acting on
    nu = (U_inf - U, E_inf) per bead (11 each: 6 velocity, 5 strain),
    returning (F, S) per bead (the grand-resistance convention of Sec. 2.1).

    Relative surface velocity of the pair (n from i to j, lever r/2 so that
    a rigid motion of the pair gives zero):
        s = (du_j - du_i) + (r/2) n x (dw_i + dw_j) + r E.n
        t = dw_i - dw_j
    Dissipation s.G.s + t.Gt.t with G = A nn + B (I - nn), Gt = D (I - nn)."""
    x = xj - xi
    r = np.linalg.norm(x)
    n = x / r
    A, B, D = lub_coefficients(r - 2 * a, a, eta, rcut, hmin, rough)
    nn = np.outer(n, n)
    G = A * nn + B * (I3 - nn)
    Gt = D * (I3 - nn)
    nx = np.einsum("abc,b->ac", EPS, n)  # n x v = [n]x v
    # s as a linear map of nu = (-du_i, -dw_i, E_i, -du_j, -dw_j, E_j)
    Ls = np.zeros((3, 22))
    Ls[:, 0:3] = I3                 # du_i enters as -du_i -> +I on nu
    Ls[:, 3:6] = -0.5 * r * nx      # (r/2) n x dw_i with dw_i = -nu
    Ls[:, 6:11] = 0.5 * r * np.einsum("mab,b->am", EB, n)
    Ls[:, 11:14] = -I3
    Ls[:, 14:17] = -0.5 * r * nx
    Ls[:, 17:22] = 0.5 * r * np.einsum("mab,b->am", EB, n)
    Lt = np.zeros((3, 22))
    Lt[:, 3:6] = -I3
    Lt[:, 14:17] = I3
    return Ls.T @ G @ Ls + Lt.T @ Gt @ Lt


def lub_pair_factor(xi, xj, a=1.0, eta=1.0, rcut=3.0, hmin=1e-3, rough=(0.0, 0.0)):
    """K (6 x 12) with K^T K = the FU block of lub_pair_matrix (velocities
    and rotations of i, then of j): the dissipation form's own factor,
    K = [G^(1/2) Ls; Gt^(1/2) Lt] restricted to the velocity columns, with
    G^(1/2) = sqrt(A) nn + sqrt(B) (I - nn), Gt^(1/2) = sqrt(D) (I - nn)."""
    x = xj - xi
    r = np.linalg.norm(x)
    n = x / r
    A, B, D = lub_coefficients(r - 2 * a, a, eta, rcut, hmin, rough)
    nn = np.outer(n, n)
    Gh = np.sqrt(A) * nn + np.sqrt(B) * (I3 - nn)
    Gth = np.sqrt(D) * (I3 - nn)
    nx = np.einsum("abc,b->ac", EPS, n)
    Ls = np.zeros((3, 12))
    Ls[:, 0:3] = I3
    Ls[:, 3:6] = -0.5 * r * nx
    Ls[:, 6:9] = -I3
    Ls[:, 9:12] = -0.5 * r * nx
    Lt = np.zeros((3, 12))
    Lt[:, 3:6] = -I3
    Lt[:, 9:12] = I3
    return np.vstack([Gh @ Ls, Gth @ Lt])


def lubrication_dense(pos, body, L, a=1.0, eta=1.0, rcut=3.0, hmin=1e-3, tilt=0.0, rough=(0.0, 0.0)):
    """Bead-level grand near-field resistance (11 Nt x 11 Nt), per bead
    ordering (6 velocity, 5 strain), summed over inter-body pairs with
    r < rcut (minimum image).  Intra-body pairs are excluded (Alg. 1 step 1)."""
    pos = np.asarray(pos, dtype=np.float64)
    Nt = pos.shape[0]
    R = np.zeros((11 * Nt, 11 * Nt))
    if rcut <= 2.0 * a:
        return R
    for i in range(Nt):
        for j in range(i + 1, Nt):
            if body[i] == body[j]:
                continue
            d = pos[j] - pos[i]
            d = min_image(d, L, tilt)
            if np.linalg.norm(d) >= rcut:
                continue
            Rp = lub_pair_matrix(np.zeros(3), d, a, eta, rcut, hmin, rough)
            ii = np.r_[11 * i:11 * i + 11]
            jj = np.r_[11 * j:11 * j + 11]
            idx = np.r_[ii, jj]
            R[np.ix_(idx, idx)] += Rp
    return R


def split_grand(R, Nt):
    """Split the bead-level grand resistance into R_FU (6Nt x 6Nt),
    R_FE (6Nt x 5Nt), R_SU (5Nt x 6Nt), R_SE (5Nt x 5Nt)."""
    v = np.concatenate([np.arange(11 * b, 11 * b + 6) for b in range(Nt)]) if Nt else np.zeros(0, int)
    e = np.concatenate([np.arange(11 * b + 6, 11 * b + 11) for b in range(Nt)]) if Nt else np.zeros(0, int)
    return R[np.ix_(v, v)], R[np.ix_(v, e)], R[np.ix_(e, v)], R[np.ix_(e, e)]


# ---------------------------------------------------------------------------
# the saddle-point system and its solution
# ---------------------------------------------------------------------------


def assemble(pos, body, L, gamma=1.0, FT=None, a=1.0, eta=1.0, rlub=0.0, M=None,
             hmin=1e-3, tilt=0.0, rough=(0.0, 0.0)):
    """Dense saddle-point matrix and right-hand side of Eq. spm_agg.

    Unknowns: (F (11 per bead), U - U_inf (6 per body)).  Returns a dict with
    A, b and the pieces needed for the outputs."""
    body = np.asarray(body)
    Nt = len(pos)
    nb = int(body.max()) + 1
    unw, X, r = body_geometry(pos, body, L, tilt)
    if M is None:
        M = mobility_dense(unw, L, a, eta, tilt=tilt)
    E, Om = shear_flow(gamma)
    e5 = sym_to_vec5(E)
    ST = sigma_T(r, body, nb)
    Bm = B_op(Nt)
    BST = Bm @ ST
    if rlub > 2.0 * a:
        Rg = lubrication_dense(unw, body, L, a, eta, rlub, hmin, tilt, rough)
    else:
        Rg = np.zeros((11 * Nt, 11 * Nt))
    RFU, RFE, RSU, RSE = split_grand(Rg, Nt)
    RRFU = ST.T @ RFU @ ST
    # E.(x - X) and its rotational zero, per bead (6-vector)
    Er = np.zeros(6 * Nt)
    for bb in range(Nt):
        Er[6 * bb:6 * bb + 3] = E @ r[bb]
    Erep = np.tile(e5, Nt)
    # aggregate near-field strain term: Sigma [R_FU (E r; 0) + R_FE E]
    RRFE_E = ST.T @ (RFU @ Er + RFE @ Erep)
    FP = np.zeros(6 * nb) if FT is None else np.asarray(FT, dtype=np.float64).reshape(-1)
    n1 = 11 * Nt
    A = np.zeros((n1 + 6 * nb, n1 + 6 * nb))
    A[:n1, :n1] = M
    A[:n1, n1:] = BST
    A[n1:, :n1] = BST.T
    A[n1:, n1:] = -RRFU
    b = np.zeros(n1 + 6 * nb)
    for bb in range(Nt):
        b[11 * bb:11 * bb + 3] = E @ r[bb]
        b[11 * bb + 6:11 * bb + 11] = e5
    b[n1:] = -(FP + RRFE_E)
    return dict(A=A, b=b, M=M, ST=ST, Bm=Bm, RFU=RFU, RFE=RFE, RSU=RSU, RSE=RSE,
                RRFU=RRFU, X=X, r=r, unw=unw, E=E, Om=Om, e5=e5, Er=Er, Erep=Erep,
                Nt=Nt, nb=nb, gamma=gamma, FP=FP)


def outputs(sys_, sol):
    """Aggregate velocities (lab frame) and stresslets from the solution.

    U = (U - U_inf) + U_inf(X), U_inf(X) = gamma X_y x (origin y = 0);
    Omega = dOmega + Omega_inf.  Per body (Eq. stress_comp a, d):
      S^H_J = sum_b [S_b^ff + S_b^nf],  S_b^nf = R_SU (U_inf - u)_b + R_SE E
      S^C_J = 1/2 sum_b [r_b (x) F_b + F_b (x) r_b],  F_b = F_b^ff + F_b^nf
    (F^C_b = -F_b: the constraint force balances the bead's hydrodynamic force)."""
    Nt, nb = sys_["Nt"], sys_["nb"]
    n1 = 11 * Nt
    Fm = sol[:n1].reshape(Nt, 11)
    dU = sol[n1:].reshape(nb, 6)
    X = sys_["X"]
    U = dU.copy()
    U[:, 0] += sys_["gamma"] * X[:, 1]
    U[:, 3:6] += sys_["Om"]
    # bead relative velocities du = Sigma^T dU - (E r; 0)
    dv = sys_["ST"] @ sol[n1:] - sys_["Er"]
    Fnf = -(sys_["RFU"] @ dv) + sys_["RFE"] @ sys_["Erep"]
    Snf = -(sys_["RSU"] @ dv) + sys_["RSE"] @ sys_["Erep"]
    Fnf = Fnf.reshape(Nt, 6)
    Snf = Snf.reshape(Nt, 5)
    body = np.asarray(sys_["body"])
    r = sys_["r"]
    S = np.zeros((nb, 3, 3))
    SH = np.zeros((nb, 3, 3))
    SC = np.zeros((nb, 3, 3))
    for bb in range(Nt):
        J = body[bb]
        SH[J] += vec5_to_sym(Fm[bb, 6:11] + Snf[bb])
        Ft = Fm[bb, 0:3] + Fnf[bb, 0:3]
        SC[J] += 0.5 * (np.outer(r[bb], Ft) + np.outer(Ft, r[bb]))
    S = SH + SC
    return dict(U=U, dU=dU, S=S, SH=SH, SC=SC, F=Fm, Fnf=Fnf, Snf=Snf)


def solve(pos, body, L, gamma=1.0, FT=None, a=1.0, eta=1.0, rlub=0.0, M=None, hmin=1e-3, tilt=0.0,
          rough=(0.0, 0.0)):
    """Dense direct solve of Eq. spm_agg (LAPACK gesv).  Returns outputs plus
    the relative residual ||A x - b|| / ||b||.  tilt != 0: the Lees-Edwards
    box (images across y offset by tilt along x)."""
    sys_ = assemble(pos, body, L, gamma, FT, a, eta, rlub, M, hmin, tilt, rough)
    sys_["body"] = np.asarray(body)
    x = np.linalg.solve(sys_["A"], sys_["b"])
    res = np.linalg.norm(sys_["A"] @ x - sys_["b"]) / max(np.linalg.norm(sys_["b"]), 1e-300)
    out = outputs(sys_, x)
    out["x"] = x
    out["rel_residual"] = res
    out["system"] = sys_
    return out


def solve_schur(sys_):
    """Brute-force Schur-complement route (pin only): eliminate F,
        (Sigma B^T M^-1 B Sigma^T + RR_nf) dU = Sigma B^T M^-1 b1 - b2
    then F = M^-1 (b1 - B Sigma^T dU)."""
    Nt = sys_["Nt"]
    n1 = 11 * Nt
    A, b = sys_["A"], sys_["b"]
    M = A[:n1, :n1]
    BST = A[:n1, n1:]
    Minv = np.linalg.inv(M)
    Sch = BST.T @ Minv @ BST - A[n1:, n1:]
    rhs = BST.T @ Minv @ b[:n1] - b[n1:]
    dU = np.linalg.solve(Sch, rhs)
    F = Minv @ (b[:n1] - BST @ dU)
    return np.concatenate([F, dU])


def preconditioner_dense(sys_, pos, body, L, a=1.0, eta=1.0, rp=2.1, hmin=1e-3, rlub=3.0):
    """The block-triangular preconditioner inverse of Table 1 (aggregates
    column), with M_inf ~ mu0 I, i.e. (M_inf)^-1 ~ zeta0 I, zeta0 = 6 pi eta a:

      P^-1 = [I, -zeta0 B Sigma^T; 0, I] [zeta0 I, 0; 0, S^-1] [I, 0; -zeta0 Sigma B^T, I]
      S    = -blockdiag_J [ Sigma (zeta0 I + R~_FU) Sigma^T ]_JJ

    with R~ the near-field resistance restricted to inter-body pairs r < rp.
    Returned as a dense matrix (pins / parity only)."""
    Nt, nb = sys_["Nt"], sys_["nb"]
    n1 = 11 * Nt
    z0 = 6 * PI * eta * a
    unw = sys_["unw"]
    # R~ uses the same pair functions as R_nf (cut-off shift at rlub),
    # restricted to pairs closer than rp
    if rp > 2 * a and rlub > 2 * a:
        Rg = lubrication_dense_cut(unw, body, L, a, eta, rp, rlub, hmin)
    else:
        Rg = np.zeros((11 * Nt, 11 * Nt))
    RFU = split_grand(Rg, Nt)[0]
    ST = sys_["ST"]
    big = ST.T @ (z0 * np.eye(6 * Nt) + RFU) @ ST
    Sinv = np.zeros((6 * nb, 6 * nb))
    for J in range(nb):
        blk = big[6 * J:6 * J + 6, 6 * J:6 * J + 6]
        Sinv[6 * J:6 * J + 6, 6 * J:6 * J + 6] = -np.linalg.inv(blk)
    BST = sys_["A"][:n1, n1:]
    Upper = np.eye(n1 + 6 * nb)
    Upper[:n1, n1:] = -z0 * BST
    Mid = np.zeros((n1 + 6 * nb,) * 2)
    Mid[:n1, :n1] = z0 * np.eye(n1)
    Mid[n1:, n1:] = Sinv
    Lower = np.eye(n1 + 6 * nb)
    Lower[n1:, :n1] = -z0 * BST.T
    return Upper @ Mid @ Lower


def lubrication_dense_cut(pos, body, L, a, eta, rpair, rlub, hmin=1e-3, tilt=0.0):
    """R_nf with the pair functions of cut-off rlub, restricted to pairs r < rpair."""
    pos = np.asarray(pos, dtype=np.float64)
    Nt = pos.shape[0]
    R = np.zeros((11 * Nt, 11 * Nt))
    for i in range(Nt):
        for j in range(i + 1, Nt):
            if body[i] == body[j]:
                continue
            d = pos[j] - pos[i]
            d = min_image(d, L, tilt)
            if np.linalg.norm(d) >= min(rpair, rlub):
                continue
            Rp = lub_pair_matrix(np.zeros(3), d, a, eta, rlub, hmin)
            idx = np.r_[11 * i:11 * i + 11, 11 * j:11 * j + 11]
            R[np.ix_(idx, idx)] += Rp
    return R


# ---------------------------------------------------------------------------
# time integration (Sec. 2.4, Eq. EM1-EM3)
# ---------------------------------------------------------------------------


def quat_mul(p, q):
    w1, v1 = p[..., 0], p[..., 1:]
    w2, v2 = q[..., 0], q[..., 1:]
    w = w1 * w2 - np.sum(v1 * v2, axis=-1)
    v = w1[..., None] * v2 + w2[..., None] * v1 + np.cross(v1, v2)
    return np.concatenate([w[..., None], v], axis=-1)


def quat_to_matrix(q):
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.empty(q.shape[:-1] + (3, 3))
    R[..., 0, 0] = 1 - 2 * (y * y + z * z)
    R[..., 0, 1] = 2 * (x * y - w * z)
    R[..., 0, 2] = 2 * (x * z + w * y)
    R[..., 1, 0] = 2 * (x * y + w * z)
    R[..., 1, 1] = 1 - 2 * (x * x + z * z)
    R[..., 1, 2] = 2 * (y * z - w * x)
    R[..., 2, 0] = 2 * (x * z - w * y)
    R[..., 2, 1] = 2 * (y * z + w * x)
    R[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def integrate(X, q, r_body, body, U, dt, comoving_gamma=0.0):
    """Euler-Maruyama rigid-body update: X += U dt (Eq. EM1);
    q <- normalise(q + dt/2 (0, Omega) (x) q) (Eq. EM2, quaternion product);
    x_b = X + R(q) r_body (Eq. EM3 read as reconstruction about the new X)."""
    Ut = U.copy()
    # disturbance motion only (U - U_inf, Omega - Omega_inf; the co-moving
    # flag of the library): no affine advection in a box without sheared images
    Ut[:, 0] -= comoving_gamma * X[:, 1]
    Ut[:, 5] += 0.5 * comoving_gamma
    X = X + Ut[:, 0:3] * dt
    om = np.concatenate([np.zeros((U.shape[0], 1)), Ut[:, 3:6]], axis=1)
    q = q + 0.5 * dt * quat_mul(om, q)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    R = quat_to_matrix(q)
    x = X[body] + np.einsum("bij,bj->bi", R[body], r_body)
    return X, q, x


# ---------------------------------------------------------------------------
# sampled rows (checks at sizes where the dense system does not fit)
# ---------------------------------------------------------------------------


def mobility_real_rows(pos, L, xi, rc, rows, F, a=1.0, eta=1.0):
    """Rows `rows` of the real-space Ewald part (incl. the self term) applied
    to F (Nt, 11): the same sum as mobility_real_dense, restricted to the
    requested target beads.  Returns (len(rows), 11)."""
    pos = np.asarray(pos, dtype=np.float64)
    F = np.asarray(F, dtype=np.float64)
    N = pos.shape[0]
    nimg = int(np.ceil(rc / L)) + 1
    shifts = _lattice(nimg).astype(np.float64) * L
    w0 = wave_blocks_free(np.zeros((1, 3)), xi, a, eta)[0]
    selfb = self_block(a, eta) - w0
    out = np.zeros((len(rows), 11))
    for k, i in enumerate(rows):
        d = pos[i][None, :] - pos
        x = (d[:, None, :] + shifts[None, :, :]).reshape(-1, 3)
        jj = np.repeat(np.arange(N), shifts.shape[0])
        r = np.linalg.norm(x, axis=1)
        keep = (r < rc) & (r > 0.0)
        if keep.any():
            blk = free_blocks(x[keep], a, eta) - wave_blocks_free(x[keep], xi, a, eta)
            out[k] = np.einsum("pst,pt->s", blk, F[jj[keep]])
        out[k] += selfb @ F[i]
    return out


def lubrication_rows(pos, body, L, bodies, dU, a=1.0, eta=1.0, rcut=3.0, hmin=1e-3):
    """(RR_FU^nf dU)_J for the aggregates J in `bodies`: the rows of
    Sigma R_FU Sigma^T, with every inter-body pair of a bead of J found by
    brute force (minimum image).  Returns (len(bodies), 6)."""
    pos = np.asarray(pos, dtype=np.float64)
    body = np.asarray(body)
    unw, X, r = body_geometry(pos, body, L)
    dU = np.asarray(dU, dtype=np.float64)

    def rigid(b):
        J = body[b]
        return np.concatenate([dU[J, 0:3] + np.cross(dU[J, 3:6], r[b]), dU[J, 3:6]])

    out = np.zeros((len(bodies), 6))
    for k, J in enumerate(bodies):
        for b in np.nonzero(body == J)[0]:
            d = unw - unw[b]
            d -= L * np.round(d / L)
            dist = np.linalg.norm(d, axis=1)
            f = np.zeros(6)
            for c in np.nonzero((dist < rcut) & (body != J))[0]:
                R = lub_pair_matrix(np.zeros(3), d[c], a, eta, rcut, hmin)
                f += R[0:6, 0:6] @ rigid(b) + R[0:6, 11:17] @ rigid(c)
            out[k, 0:3] += f[0:3]
            out[k, 3:6] += f[3:6] + np.cross(r[b], f[0:3])
    return out
