"""Brownian forcing of the rigid-aggregate saddle-point solve, as plain FP64
definitions.

TEST INFRASTRUCTURE ONLY: imported by tests/ (and nothing in the product
path).  It uses fsd_oracle for the mobility and resistance pieces and shares
no code with the CUDA library.

What it computes (paper: Sec. 2.2 "stochastic sampling", Eq. SP2, Eq. UBff;
Algorithm 1 step 3):

* far-field Brownian slip  u^B = sqrt(2 kT/dt) (u_w + u_r) per bead, 11
  components (velocity, rotation, strain):
  - u_r = (M_r)^(1/2) psi_r, with M_r the real-space Ewald part of the
    mobility and the square root from a dense symmetric eigendecomposition
    (M_r is positive definite for the Hasimoto split, Sec. 2.2);
  - u_w = (M_w)^(1/2) psi_w in the analytic form of the wave part: for a
    random field xi(k) on the wave vectors (complex standard Gaussian per
    component, Hermitian: xi(-k) = conj xi(k))
        u_w(x_i) = V^(-1/2) sum_k e^(i k.x_i) Q(k)^H sqrt(H(k)/(eta k^2)) (I - k k) xi(k),
    whose covariance over the field is exactly the wave-vector sum M_w
    (pinned in tests/test_oracle_brownian.py);
* near-field Brownian force  F^B_nf = sqrt(2 kT/dt) R_FU^nf^(1/2) psi_nf with
  the preconditioned square root of the "fast preconditioned Krylov" sampling
  (Sec. 2.2): per bead b, L_b L_b^T = D_b + 1e-6 (tr D_b / 6) I (Cholesky;
  D_b the 6x6 diagonal block of R; L_b = I when tr D_b = 0), G = blockdiag
  (L_b^-1), and R^(1/2) psi := L (G R G^T)^(1/2) psi, whose covariance is R
  for any invertible G (pinned); R_FU^nf is the bead-level near-field
  resistance;
* alternatively (a sampler this build adds beside the paper's Lanczos one),
  the near-field force by the pairwise decomposition of the pair model's
  dissipation form, R_FU^nf = sum_p K_p^T K_p with K_p = [G^(1/2) Ls;
  Gt^(1/2) Lt] (6 x 12): F^B_nf = sqrt(2 kT/dt) sum_p K_p^T psi_p, psi_p 6
  independent normals per pair; its covariance is exactly R_FU^nf (pinned);
* the saddle-point right-hand side with them (Eq. spm_agg): bead rows + u^B,
  body rows - Sigma F^B_nf.

Reading: u^B carries all 11 components of M^(1/2) psi (the strain rows get
their noise too).  Eliminating the force unknowns gives a body-velocity noise
of covariance 2 kT/dt (B^T M^-1 B + RR)^-1 only if the slip covariance is the
full M (Eq. spm_agg writes u^B in the velocity rows; the strain-row part is
the same sample's read-out).

Random numbers: tests pass them in.  For the generator inside the library the
oracle implements the same counter-based generator from its published
definition: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011) and the
Box-Muller transform, with this counter layout:
    key = (seed mod 2^32, seed div 2^32)
    counter = (index, stream * 256 + call, step mod 2^32, step div 2^32)
    stream 1: wave field, index = (kz * n + ky) * nh + kx of the canonical
              point, calls 0 and 1 give (re0, im0, re1, im1) and (re2, im2)
              (scaled by 1/sqrt 2); a point of the kx = 0 plane whose mirror
              (-ky, -kz) comes first in (kz, ky) order takes the conjugate of
              the mirror's value; Nyquist points and k = 0 are zero;
    stream 2: psi_r, index = bead (input order), calls 0..2 give 12 normals,
              the first 11 used;
    stream 3: psi_nf, index = bead (input order), calls 0..1 give 8 normals,
              the first 6 used;
    stream 5 (pairwise near-field sampler): counter (i, 5 * 256 + call, j,
              step mod 2^32) for the pair i < j, calls 0 and 1, the first 6
              of 8 normals.
    Box-Muller on one output (x0, x1, x2, x3): u_j = (x_j + 1) 2^-32,
    (z0, z1) = sqrt(-2 ln u0) (cos 2 pi u1, sin 2 pi u1), (z2, z3) likewise
    from (u2, u3).
"""

import numpy as np

from . import fsd_oracle as F

M32 = 0xFFFFFFFF


# --------------------------------------------------------------- generator
def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds: ctr = 4 words, key = 2 words (ints)."""
    c = [int(x) & M32 for x in ctr]
    k0, k1 = int(key[0]) & M32, int(key[1]) & M32
    for r in range(10):
        if r > 0:
            k0 = (k0 + 0x9E3779B9) & M32
            k1 = (k1 + 0xBB67AE85) & M32
        p0 = 0xD2511F53 * c[0]
        p1 = 0xCD9E8D57 * c[2]
        hi0, lo0 = (p0 >> 32) & M32, p0 & M32
        hi1, lo1 = (p1 >> 32) & M32, p1 & M32
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return c


def box_muller4(x):
    u = [(xi + 1) * 2.0 ** -32 for xi in x]
    r0 = np.sqrt(-2.0 * np.log(u[0]))
    r1 = np.sqrt(-2.0 * np.log(u[2]))
    return [r0 * np.cos(2 * np.pi * u[1]), r0 * np.sin(2 * np.pi * u[1]),
            r1 * np.cos(2 * np.pi * u[3]), r1 * np.sin(2 * np.pi * u[3])]


def _normals(seed, step, stream, index, ncalls):
    key = (seed & M32, (seed >> 32) & M32)
    out = []
    for call in range(ncalls):
        ctr = (index & M32, (stream << 8) | call, step & M32, (step >> 32) & M32)
        out += box_muller4(philox4x32_10(ctr, key))
    return out


def _is_nyq(i, n):
    return i == n // 2


def philox_wave_field(n, seed, step):
    """The library's wave random field: complex [3][n][n][n/2+1] ([c][kz][ky][kx])."""
    nh = n // 2 + 1
    xi = np.zeros((3, n, n, nh), dtype=np.complex128)
    s = 1.0 / np.sqrt(2.0)
    for kz in range(n):
        for ky in range(n):
            for kx in range(nh):
                if _is_nyq(kx, n) or _is_nyq(ky, n) or _is_nyq(kz, n) or (kx == 0 and ky == 0 and kz == 0):
                    continue
                cz, cy, conj = kz, ky, False
                if kx == 0:
                    mz, my = (n - kz) % n, (n - ky) % n
                    if (mz, my) < (kz, ky):
                        cz, cy, conj = mz, my, True
                z = _normals(seed, step, 1, (cz * n + cy) * nh + kx, 2)
                v = np.array([z[0] + 1j * z[1], z[2] + 1j * z[3], z[4] + 1j * z[5]]) * s
                xi[:, kz, ky, kx] = np.conj(v) if conj else v
    return xi


def philox_psi(n_beads, seed, step, stream, width):
    calls = (width + 3) // 4
    return np.array([_normals(seed, step, stream, b, calls)[:width] for b in range(n_beads)])


# --------------------------------------------------------------- sampling
def hermitian_field(n, rng):
    """A random field of the library's layout: complex standard Gaussian
    components, Hermitian in the kx = 0 plane, zero at Nyquist and k = 0."""
    nh = n // 2 + 1
    xi = (rng.normal(size=(3, n, n, nh)) + 1j * rng.normal(size=(3, n, n, nh))) / np.sqrt(2.0)
    for kz in range(n):
        for ky in range(n):
            mz, my = (n - kz) % n, (n - ky) % n
            if (mz, my) < (kz, ky):
                xi[:, kz, ky, 0] = np.conj(xi[:, mz, my, 0])
    idx = np.arange(n)
    nyq = idx == n // 2
    xi[:, nyq, :, :] = 0
    xi[:, :, nyq, :] = 0
    xi[:, :, :, n // 2] = 0
    xi[:, 0, 0, 0] = 0
    return xi


def _k_int(i, n):
    return i if i < n // 2 else i - n


def brownian_wave_slip(pos, L, xi, n, field, a=1.0, eta=1.0, tilt=0.0):
    """u_w per bead (N, 11) for the half-spectrum field [3][n][n][n/2+1]:
    V^-1/2 sum over k = 2 pi m / L, |m_i| < n/2, k != 0 (kx < 0 by
    conjugation) of e^(ik.x) Q(k)^H sqrt(H/(eta k^2)) (I - kk) xi(k).  In a
    Lees-Edwards box (tilt != 0) the field index m labels the reciprocal
    vector k = (2 pi / L)(m1, m2 - (tilt/L) m1, m3) of the sheared lattice."""
    pos = np.asarray(pos, dtype=np.float64)
    nh = n // 2 + 1
    ms, vals, wts = [], [], []
    for kz in range(n):
        for ky in range(n):
            for kx in range(nh):
                if _is_nyq(kx, n) or _is_nyq(ky, n) or _is_nyq(kz, n) or (kx == 0 and ky == 0 and kz == 0):
                    continue
                ms.append((kx, _k_int(ky, n), _k_int(kz, n)))
                vals.append(field[:, kz, ky, kx])
                wts.append(1.0 if kx == 0 else 2.0)  # kx > 0 also stands for -k
    m = np.array(ms, dtype=np.float64)
    m[:, 1] -= (tilt / L) * m[:, 0]
    v = np.array(vals)
    w = np.array(wts)
    k = 2.0 * np.pi * m / L
    kn = np.linalg.norm(k, axis=1)
    kh = k / kn[:, None]
    Pk = np.eye(3)[None] - np.einsum("pa,pb->pab", kh, kh)
    g = np.sqrt(F.hasimoto(kn, xi) / (eta * kn * kn))
    amp = np.einsum("pab,pb->pa", Pk, v) * g[:, None]        # sqrt(G) P xi
    Q = F.source_operator(k, a)                              # (K, 3, 11)
    QHa = np.einsum("pas,pa->ps", Q.conj(), amp)             # Q^H (...)
    ph = np.exp(1j * (k @ pos.T))                            # (K, N)
    u = np.einsum("p,pn,ps->ns", w, ph, QHa).real
    return u / np.sqrt(L ** 3)


def sqrtm_apply(A, v):
    """A^(1/2) v for a symmetric positive semidefinite A (eigendecomposition)."""
    lam, U = np.linalg.eigh(A)
    return U @ (np.sqrt(np.clip(lam, 0.0, None)) * (U.T @ v))


def block_precond_sqrt_apply(R, v, bs=6):
    """L (G R G^T)^(1/2) v with L = blockdiag(chol(D_b + 1e-6 tr(D_b)/6 I))
    over the bs x bs diagonal blocks D_b of the symmetric positive
    semidefinite R (L_b = I where tr D_b = 0) and G = L^-1."""
    nb = R.shape[0] // bs
    Lm = np.zeros_like(R)
    G = np.zeros_like(R)
    for b in range(nb):
        sl = slice(b * bs, (b + 1) * bs)
        D = 0.5 * (R[sl, sl] + R[sl, sl].T)
        tr = np.trace(D)
        if tr > 0:
            Lb = np.linalg.cholesky(D + 1e-6 * tr / bs * np.eye(bs))
        else:
            Lb = np.eye(bs)
        Lm[sl, sl] = Lb
        G[sl, sl] = np.linalg.inv(Lb)
    return Lm @ sqrtm_apply(G @ R @ G.T, v)


def pair_normals(seed, step, i, j):
    """6 standard normals of the bead pair (i < j, input order) for the
    pairwise near-field sampler: Philox4x32-10 with key = seed and counter
    (i, 5 * 256 + call, j, step mod 2^32), calls 0 and 1 (the first 6 of 8),
    Box-Muller."""
    key = (seed & M32, (seed >> 32) & M32)
    out = []
    for call in range(2):
        out += box_muller4(philox4x32_10((i & M32, (5 << 8) | call, j & M32, step & M32), key))
    return np.array(out[:6])


def pairwise_nf_apply(pos, body, L, psi_of_pair, rlub=3.0, a=1.0, eta=1.0, hmin=1e-3, tilt=0.0):
    """sum over inter-body pairs p = (i < j), r < rlub, of K_p^T psi_p, K_p
    (6 x 12) the pair's dissipation-form factor (K_p^T K_p = the pair's
    12 x 12 block of R_FU^nf on the velocities of i and j) and
    psi_p = psi_of_pair(i, j) (6 values); (N_tot, 6)."""
    pos = np.asarray(pos, dtype=np.float64)
    body = np.asarray(body)
    Nt = len(pos)
    out = np.zeros((Nt, 6))
    for i in range(Nt):
        for j in range(i + 1, Nt):
            if body[i] == body[j]:
                continue
            d = F.min_image(pos[j] - pos[i], L, tilt)
            if np.linalg.norm(d) >= rlub:
                continue
            K = F.lub_pair_factor(np.zeros(3), d, a, eta, rlub, hmin)
            v = K.T @ np.asarray(psi_of_pair(i, j), dtype=np.float64)
            out[i] += v[:6]
            out[j] += v[6:]
    return out


def pairwise_nf_force(pos, body, L, seed, step, rlub=3.0, a=1.0, eta=1.0, hmin=1e-3, tilt=0.0):
    """Near-field Brownian force (unscaled) by the pairwise decomposition
    R_FU^nf = sum_p K_p^T K_p: F = sum_p K_p^T psi_p with independent
    psi_p (pair_normals), whose covariance is exactly R_FU^nf."""
    return pairwise_nf_apply(pos, body, L, lambda i, j: pair_normals(seed, step, i, j), rlub, a, eta,
                             hmin, tilt)


def brownian_terms(pos, body, L, xi, n, field, psi_r, psi_nf, kT, dt, rlub=3.0, a=1.0, eta=1.0,
                   hmin=1e-3):
    """(u^B (N, 11), F^B_nf (N, 6)) of Eq. SP2 / Eq. UBff for the given random
    inputs; the real-space part uses the splitting xi with its converged
    cut-off (oracle_split's tail rule)."""
    pos = np.asarray(pos, dtype=np.float64)
    unw, X, r = F.body_geometry(pos, body, L)
    N = len(pos)
    rc = 2.0 + np.sqrt(46.0) / xi
    Mr = F.mobility_real_dense(unw, L, xi, rc, a, eta).reshape(11 * N, 11 * N)
    s = np.sqrt(2.0 * kT / dt)
    ur = sqrtm_apply(Mr, np.asarray(psi_r).reshape(-1)).reshape(N, 11)
    uw = brownian_wave_slip(unw, L, xi, n, field, a, eta)
    if rlub > 2.0 * a:
        Rg = F.lubrication_dense(unw, body, L, a, eta, rlub, hmin)
    else:
        Rg = np.zeros((11 * N, 11 * N))
    RFU = F.split_grand(Rg, N)[0]
    fnf = block_precond_sqrt_apply(RFU, np.asarray(psi_nf).reshape(-1)).reshape(N, 6)
    return s * (uw + ur), s * fnf


def solve_brownian(pos, body, L, uB, fnf, gamma=1.0, FT=None, rlub=3.0, a=1.0, eta=1.0,
                   hmin=1e-3, M=None):
    """Dense solve of Eq. spm_agg with the Brownian terms: bead rows + u^B,
    body rows - Sigma F^B_nf."""
    sys_ = F.assemble(pos, body, L, gamma, FT, a, eta, rlub, M, hmin)
    sys_["body"] = np.asarray(body)
    N = sys_["Nt"]
    b = sys_["b"].copy()
    b[:11 * N] += np.asarray(uB).reshape(-1)
    b[11 * N:] -= sys_["ST"].T @ np.asarray(fnf).reshape(-1)
    x = np.linalg.solve(sys_["A"], b)
    out = F.outputs(sys_, x)
    out["x"] = x
    return out
