"""Pins of the Brownian oracle (oracle/brownian_oracle.py) against what the
definitions and the paper fix (Sec. 2.2 stochastic sampling, Eq. SP2,
Eq. UBff):

* Philox4x32-10 reproduces the published known-answer vectors of its
  authors' reference implementation;
* the analytic wave-space sample has covariance exactly M_w: the sample is
  linear in the random field, so summing the outer products of its response
  to each independent field component gives the covariance, which must equal
  the wave-vector sum M_w of fsd_oracle (pinned elsewhere against closed forms
  and xi-independence);
* the dense square root applied twice is the operator; the block-Cholesky
  preconditioned square root L (G R G^T)^(1/2), G = L^-1, has covariance
  exactly R;
* a near-field Brownian force enters the body rows exactly like an applied
  aggregate force and torque (the same Sigma projection, the same sign);
* Box-Muller normals from Philox have zero mean, unit variance, no
  correlation between components;
* fluctuation-dissipation: over an orthonormal basis of all the noise the
  Brownian body velocities have covariance (2 kT/dt) N, N the body
  mobility (only with the strain rows of u^B);
* the pairwise near-field sampler has covariance R_FU^nf.
"""

import numpy as np
import pytest

import oracle as O
from oracle import brownian_oracle as B


def test_philox_known_answers():
    assert B.philox4x32_10((0, 0, 0, 0), (0, 0)) == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    f = 0xFFFFFFFF
    assert B.philox4x32_10((f, f, f, f), (f, f)) == [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]
    assert B.philox4x32_10((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344),
                           (0xA4093822, 0x299F31D0)) == [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def test_generators_follow_the_documented_counter_layout():
    # the library's documented layout for its own draws: key (seed mod 2^32,
    # seed / 2^32), counter (index, stream * 256 + call, step mod 2^32,
    # step / 2^32), four Box-Muller normals per call; a bead's psi takes the
    # first `width` normals of its calls, a wave-field point the six normals
    # of its canonical index (kz n + ky)(n/2 + 1) + kx, the mirror of a kx = 0
    # point their conjugate
    seed, step = 0x123456789ABC, (7 << 32) + 5
    key = (seed & 0xFFFFFFFF, seed >> 32)

    def normals(index, stream, call):
        ctr = (index, stream * 256 + call, step & 0xFFFFFFFF, step >> 32)
        return B.box_muller4(B.philox4x32_10(ctr, key))

    psi = B.philox_psi(3, seed, step, 2, 11)
    for b in range(3):
        z = normals(b, 2, 0) + normals(b, 2, 1) + normals(b, 2, 2)
        assert np.array_equal(psi[b], np.array(z[:11]))
    n = 6
    nh = n // 2 + 1
    f = B.philox_wave_field(n, seed, step)
    for kz, ky, kx in [(1, 2, 1), (4, 5, 2), (2, 1, 0)]:
        idx = (kz * n + ky) * nh + kx
        z = normals(idx, 1, 0) + normals(idx, 1, 1)
        v = np.array([z[0] + 1j * z[1], z[2] + 1j * z[3], z[4] + 1j * z[5]]) / np.sqrt(2.0)
        assert np.abs(f[:, kz, ky, kx] - v).max() < 1e-15
    # (2, 1, 0) comes before its mirror (4, 5, 0), which holds the conjugate
    assert np.abs(f[:, 4, 5, 0] - np.conj(f[:, 2, 1, 0])).max() == 0.0


def test_box_muller_moments():
    z = np.array([B._normals(7, 3, 2, i, 1) for i in range(20000)]).reshape(-1, 4)
    assert abs(z.mean()) < 0.02
    assert abs(z.var() - 1.0) < 0.03
    c = np.corrcoef(z.T)
    assert np.abs(c - np.eye(4)).max() < 0.03


def test_wave_sample_covariance_is_the_wave_mobility():
    # two beads, a grid whose k-cube contains the sphere the wave sum needs
    L, n, xi = 10.0, 12, 0.22
    pos = np.array([[1.0, 2.0, 3.0], [4.5, 2.5, 6.0]])
    nh = n // 2 + 1
    cov = np.zeros((22, 22))
    for c in range(3):
        for kz in range(n):
            for ky in range(n):
                for kx in range(nh):
                    if kx == n // 2 or ky == n // 2 or kz == n // 2 or (kx == ky == kz == 0):
                        continue
                    mz, my = (n - kz) % n, (n - ky) % n
                    if kx == 0 and (mz, my) < (kz, ky):
                        continue  # the mirror of a canonical point carries no new variable
                    for val in (1.0 / np.sqrt(2.0), 1j / np.sqrt(2.0)):
                        f = np.zeros((3, n, n, nh), dtype=np.complex128)
                        f[c, kz, ky, kx] = val
                        if kx == 0:
                            f[c, mz, my, 0] = np.conj(val)
                        u = B.brownian_wave_slip(pos, L, xi, n, f).reshape(-1)
                        cov += np.outer(u, u)
    kmax = 2.0 * xi * np.sqrt(46.0)
    assert kmax < 2 * np.pi * (n // 2 - 1) / L
    Mw = O.mobility_wave_dense(pos, L, xi, kmax).reshape(22, 22)
    assert np.abs(cov - Mw).max() < 1e-10 * np.abs(Mw).max()


def test_hermitian_field_gives_real_slip():
    rng = np.random.default_rng(3)
    n = 10
    f = B.hermitian_field(n, rng)
    pos = np.array([[1.0, 2.0, 3.0], [4.0, 5.0, 1.0]])
    u = B.brownian_wave_slip(pos, 9.0, 0.4, n, f)
    assert u.shape == (2, 11) and np.all(np.isfinite(u)) and np.abs(u).max() > 0
    # the library's generator fills the same layout with the same symmetry;
    # both fields are zero on the Nyquist planes and at k = 0 (a real field
    # has no independent Nyquist sine modes, and the k = 0 mode is excluded)
    g = B.philox_wave_field(n, seed=5, step=2)
    for fld in (f, g):
        assert np.abs(fld[:, n // 2, :, :]).max() == 0.0
        assert np.abs(fld[:, :, n // 2, :]).max() == 0.0
        assert np.abs(fld[:, :, :, n // 2]).max() == 0.0
        assert np.abs(fld[:, 0, 0, 0]).max() == 0.0
        for kz in range(n):
            for ky in range(n):
                mz, my = (n - kz) % n, (n - ky) % n
                assert np.allclose(fld[:, kz, ky, 0], np.conj(fld[:, mz, my, 0]))


def test_brownian_terms_have_the_fluctuation_dissipation_amplitude():
    # Eq. SP2: the real-space slip and the near-field force are
    # sqrt(2 kT/dt) times square roots of M_r and R_FU^nf, so that summed
    # over an orthonormal basis of their noise (psi_r, 11 per bead; psi_nf, 6
    # per bead) their second moments are (2 kT/dt) M_r and (2 kT/dt) R_FU^nf.
    # Two beads of different bodies 0.2a apart (one lubrication pair), a zero
    # wave field.
    L, xi, n, kT, dt = 8.0, 1.0, 4, 0.7, 0.02
    pos = np.array([[1.0, 1.5, 2.0], [3.2, 1.5, 2.0]])
    body = np.array([0, 1])
    field = np.zeros((3, n, n, n // 2 + 1), dtype=np.complex128)
    Nt = 2
    cu = np.zeros((11 * Nt, 11 * Nt))
    cf = np.zeros((6 * Nt, 6 * Nt))
    for k in range(11 * Nt):
        psi_r = np.eye(11 * Nt)[k].reshape(Nt, 11)
        u, f = B.brownian_terms(pos, body, L, xi, n, field, psi_r, np.zeros((Nt, 6)), kT, dt)
        assert np.abs(f).max() == 0.0
        cu += np.outer(u.reshape(-1), u.reshape(-1))
    for k in range(6 * Nt):
        psi_nf = np.eye(6 * Nt)[k].reshape(Nt, 6)
        u, f = B.brownian_terms(pos, body, L, xi, n, field, np.zeros((Nt, 11)), psi_nf, kT, dt)
        cf += np.outer(f.reshape(-1), f.reshape(-1))
    Mr = O.mobility_real_dense(pos, L, xi, 2.0 + np.sqrt(46.0) / xi).reshape(11 * Nt, 11 * Nt)
    R = O.split_grand(O.lubrication_dense(pos, body, L, rcut=3.0), Nt)[0]
    s2 = 2.0 * kT / dt
    assert np.abs(R).max() > 0
    assert np.abs(cu - s2 * Mr).max() < 1e-10 * np.abs(s2 * Mr).max()
    assert np.abs(cf - s2 * R).max() < 1e-10 * np.abs(s2 * R).max()


def test_sqrtm_apply():
    rng = np.random.default_rng(4)
    A = rng.normal(size=(9, 9))
    A = A @ A.T
    v = rng.normal(size=9)
    assert np.allclose(B.sqrtm_apply(A, B.sqrtm_apply(A, v)), A @ v, rtol=1e-10, atol=1e-10)


def test_near_field_noise_acts_like_an_aggregate_force():
    import synth

    pos, body, L = synth.config_doublets(3, 12.0, seed=4)
    rng = np.random.default_rng(5)
    f = rng.normal(size=(len(pos), 6))
    M = O.mobility_dense(pos, L)
    out = B.solve_brownian(pos, body, L, np.zeros((len(pos), 11)), f, gamma=0.5, rlub=0.0, M=M)
    unw, X, r = O.body_geometry(pos, body, L)
    FT = O.sigma_T(r, body, body.max() + 1).T @ f.reshape(-1)
    ref = O.solve(pos, body, L, gamma=0.5, FT=FT, rlub=0.0, M=M)
    assert np.allclose(out["U"], ref["U"], rtol=1e-12, atol=1e-14)


def test_zero_noise_is_the_deterministic_solve():
    import synth

    pos, body, L = synth.config_doublets(2, 12.0, seed=6)
    M = O.mobility_dense(pos, L)
    z = np.zeros((len(pos), 11))
    out = B.solve_brownian(pos, body, L, z, np.zeros((len(pos), 6)), gamma=1.0, rlub=0.0, M=M)
    ref = O.solve(pos, body, L, gamma=1.0, rlub=0.0, M=M)
    assert np.allclose(out["U"], ref["U"], rtol=1e-13, atol=1e-15)
    assert np.allclose(out["S"], ref["S"], rtol=1e-13, atol=1e-15)


def test_preconditioned_square_root_has_covariance_R():
    import synth

    rng = np.random.default_rng(3)
    shapes = [synth.random_attachment_aggregate(k, rng) for k in (2, 3, 4, 2, 3)]
    L = synth.box_for_phi(14, 0.15)
    pos, body = synth.pack_suspension(shapes, L, rng, h_gen=0.05)
    R = O.split_grand(O.lubrication_dense(pos, body, L, rcut=3.0), len(pos))[0]
    assert np.abs(R).max() > 0
    n = R.shape[0]
    S = np.column_stack([B.block_precond_sqrt_apply(R, e) for e in np.eye(n)])
    assert np.abs(S @ S.T - R).max() < 1e-9 * np.abs(R).max()


def test_wave_sample_covariance_with_tilt():
    # the same identity in a Lees-Edwards box: the index m of the field
    # labels the sheared reciprocal vector (2 pi/L)(m1, m2 - tau m1, m3)
    L, n, xi, tilt = 10.0, 12, 0.15, 3.0
    pos = np.array([[1.0, 2.0, 3.0], [4.5, 9.5, 6.0]])
    nh = n // 2 + 1
    cov = np.zeros((22, 22))
    for c in range(3):
        for kz in range(n):
            for ky in range(n):
                for kx in range(nh):
                    if kx == n // 2 or ky == n // 2 or kz == n // 2 or (kx == ky == kz == 0):
                        continue
                    mz, my = (n - kz) % n, (n - ky) % n
                    if kx == 0 and (mz, my) < (kz, ky):
                        continue
                    for val in (1.0 / np.sqrt(2.0), 1j / np.sqrt(2.0)):
                        f = np.zeros((3, n, n, nh), dtype=np.complex128)
                        f[c, kz, ky, kx] = val
                        if kx == 0:
                            f[c, mz, my, 0] = np.conj(val)
                        u = B.brownian_wave_slip(pos, L, xi, n, f, tilt=tilt).reshape(-1)
                        cov += np.outer(u, u)
    kmax = 2.0 * xi * np.sqrt(46.0)
    # every sheared reciprocal vector inside kmax has indices below Nyquist
    assert kmax * L / (2 * np.pi) * (1 + tilt / L) < n // 2 - 1
    Mw = O.mobility_wave_dense(pos, L, xi, kmax, tilt=tilt).reshape(22, 22)
    assert np.abs(cov - Mw).max() < 1e-10 * np.abs(Mw).max()
    Mw0 = O.mobility_wave_dense(pos, L, xi, kmax).reshape(22, 22)
    assert np.abs(Mw0 - Mw).max() > 1e-3 * np.abs(Mw).max()


def test_pairwise_near_field_sampler_has_covariance_R():
    # the map from the pair noises to the force is linear: summing the outer
    # products of its columns gives the covariance, which must be R_FU^nf
    import synth

    rng = np.random.default_rng(8)
    shapes = [synth.random_attachment_aggregate(k, rng) for k in (2, 3, 2, 3)]
    L = synth.box_for_phi(10, 0.15)
    pos, body = synth.pack_suspension(shapes, L, rng, h_gen=0.05)
    R = O.split_grand(O.lubrication_dense(pos, body, L, rcut=3.0), len(pos))[0]
    assert np.abs(R).max() > 0
    pairs = [(i, j) for i in range(len(pos)) for j in range(i + 1, len(pos))
             if body[i] != body[j]
             and np.linalg.norm(O.min_image(pos[j] - pos[i], L)) < 3.0]
    cov = np.zeros_like(R)
    for p in pairs:
        for k in range(6):
            col = B.pairwise_nf_apply(pos, body, L, lambda i, j: np.eye(6)[k] if (i, j) == p else np.zeros(6))
            cov += np.outer(col.reshape(-1), col.reshape(-1))
    assert np.abs(cov - R).max() < 1e-10 * np.abs(R).max()
    # and the factor of each pair reproduces that pair's block
    d = O.min_image(pos[pairs[0][1]] - pos[pairs[0][0]], L)
    K = O.lub_pair_factor(np.zeros(3), d)
    idx = np.r_[0:6, 11:17]
    Rp = O.lub_pair_matrix(np.zeros(3), d)[np.ix_(idx, idx)]
    assert np.abs(K.T @ K - Rp).max() < 1e-12 * np.abs(Rp).max()


def test_pair_normals_layout():
    z = B.pair_normals(11, 3, 2, 9)
    assert z.shape == (6,)
    assert np.allclose(z[:4], B.box_muller4(B.philox4x32_10((2, 5 << 8, 9, 3), (11, 0))))
    assert not np.allclose(B.pair_normals(11, 3, 2, 9), B.pair_normals(11, 3, 9, 2))


def test_brownian_velocity_covariance_is_the_body_mobility():
    # fluctuation-dissipation: with u^B = s M^(1/2) psi (all 11 components:
    # velocity, rotation and strain rows all carry noise, since eliminating
    # F from the saddle system mixes the strain rows into the body
    # velocities) and F^B = s R^(1/2) psi_nf, s^2 = 2 kT/dt, the body
    # velocities of the Brownian solve have covariance s^2 N, N the body
    # mobility (the solve's response to unit aggregate forces and torques).
    # Summed over an orthonormal basis of the noise the identity is exact.
    import synth

    rng = np.random.default_rng(3)
    shapes = [synth.random_attachment_aggregate(k, rng) for k in (2, 3, 4, 2, 3)]
    L = synth.box_for_phi(14, 0.15)
    pos, body = synth.pack_suspension(shapes, L, rng, h_gen=0.05)
    unw, X, r = O.body_geometry(pos, body, L)
    Nt, nb = len(pos), 5
    M = O.mobility_dense(unw, L)
    R = O.split_grand(O.lubrication_dense(unw, body, L, rcut=3.0), Nt)[0]
    assert np.abs(R).max() > 0  # near pairs: the near-field noise matters
    kT, dt = 0.8, 0.05
    s = np.sqrt(2.0 * kT / dt)
    Mh = np.linalg.cholesky(M)  # any square root gives the same covariance
    w, V = np.linalg.eigh(R)
    Rh = V @ np.diag(np.sqrt(np.clip(w, 0, None)))
    cov = np.zeros((6 * nb, 6 * nb))
    for k in range(11 * Nt + 6 * Nt):
        if k < 11 * Nt:
            uB, fB = s * Mh[:, k].reshape(Nt, 11), np.zeros((Nt, 6))
        else:
            uB, fB = np.zeros((Nt, 11)), s * Rh[:, k - 11 * Nt].reshape(Nt, 6)
        u = B.solve_brownian(pos, body, L, uB, fB, gamma=0.0, rlub=3.0, M=M)["U"].reshape(-1)
        cov += np.outer(u, u)
    Nm = np.column_stack([O.solve(pos, body, L, gamma=0.0, FT=np.eye(6 * nb)[j].reshape(nb, 6),
                                  rlub=3.0, M=M)["U"].reshape(-1) for j in range(6 * nb)])
    assert np.abs(Nm - Nm.T).max() < 1e-10 * np.abs(Nm).max()
    assert np.abs(cov - s * s * Nm).max() < 1e-9 * np.abs(s * s * Nm).max()
    # without the strain rows of u^B the far-field part of the identity
    # fails: the stresslet constraint couples them into the body velocities
    covf = np.zeros_like(cov)
    covf6 = np.zeros_like(cov)
    for k in range(11 * Nt):
        uB = s * Mh[:, k].reshape(Nt, 11)
        uB6 = uB.copy()
        uB6[:, 6:] = 0.0
        z6 = np.zeros((Nt, 6))
        u = B.solve_brownian(pos, body, L, uB, z6, gamma=0.0, rlub=3.0, M=M)["U"].reshape(-1)
        u6 = B.solve_brownian(pos, body, L, uB6, z6, gamma=0.0, rlub=3.0, M=M)["U"].reshape(-1)
        covf += np.outer(u, u)
        covf6 += np.outer(u6, u6)
    assert np.abs(covf6 - covf).max() > 1e-3 * np.abs(covf).max()
