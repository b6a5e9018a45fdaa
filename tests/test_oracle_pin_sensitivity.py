"""The oracle's pins catch plausible mistakes (CPU only).

Each case plants one mistake in a copy of one oracle module's source text (a
wrong sign, a dropped term, a wrong coefficient or exponent, a transposed
operand, a factor of two), executes the copy as a separate module, and runs
the pins expected to catch it with that module in place of the original: at
least one of them must fail.  The oracle package itself is never modified;
the same pins pass on it in their own files.  A planted text that no longer
occurs exactly once in its module makes the case fail, so an edit of the
oracle cannot silently retire a case.

The rolling coefficient of the lubrication pair model (8 pi eta a^3 (1/10)
ln(1/eps)) is the one value no pin fixes: it is this build's reading of
functions the paper does not print, and the published two-sphere functions
it stands in for are not of the pair model's form."""

import os
import types
import warnings

import numpy as np
import pytest

import synth
import test_oracle_brownian as TB
import test_oracle_contact as TC
import test_oracle_drift as TD
import test_oracle_ewald as TE
import test_oracle_lees_edwards as TL
import test_oracle_solve as TS
import test_oracle_tensors as TT

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
# the name under which the pin files hold each oracle module
HANDLE = {"fsd_oracle": "O", "brownian_oracle": "B", "drift_oracle": "D", "contact_oracle": "C"}
# the geometry of the drift pins' module fixture
DOUBLETS = synth.config_doublets(2, 9.0, seed=6)

# pin name -> (test module, test function, arguments)
PINS = {
    "reciprocity": (TS, "test_aggregate_reciprocity_of_velocity_and_stresslet", {}),
    "affine_strain": (TS, "test_lubrication_strain_columns_equal_affine_bead_motion", {"gap": 0.07}),
    "lub_asymptotics": (TS, "test_lubrication_coefficients_follow_equal_sphere_asymptotics", {}),
    "intrabody": (TS, "test_lubrication_cutoff_and_intrabody", {}),
    "sphere_in_shear": (TS, "test_single_sphere_in_periodic_shear", {"L": 10.0}),
    "doublet_in_shear": (TS, "test_doublet_in_shear_jeffery_form", {}),
    "precond_exact": (TS, "test_preconditioner_exact_for_scalar_mobility_without_lubrication", {}),
    "rigid_update": (TS, "test_integrator_keeps_bodies_rigid_and_quaternions_unit", {}),
    "lab_frame": (TS, "test_integrator_rotates_in_the_lab_frame", {}),
    "rpy": (TT, "test_translational_block_is_textbook_rpy", {"r": 2.7}),
    "faxen_DD": (TT, "test_free_phi_closed_form_matches_kspace_quadrature", {"kind": "DD"}),
    "symmetry": (TT, "test_blocks_reciprocal_symmetry", {}),
    "hasimoto_coefficient": (TE, "test_hasimoto_finite_size_coefficient", {}),
    "le_split": (TL, "test_split_independence_with_tilt", {}),
    "le_lattice": (TL, "test_lattice_translation_and_spd", {}),
    "le_solve": (TL, "test_solve_with_tilt_translation_invariant", {}),
    "le_minimum_image": (TL, "test_minimum_image_reduces_into_the_box", {}),
    "lub_lowers_mobility": (TS, "test_lubrication_lowers_the_body_mobility", {}),
    "precond_within_rp": (TS, "test_preconditioner_counts_only_pairs_within_rp", {}),
    "force_balance": (TS, "test_bead_forces_balance_each_body", {}),
    "comoving_update": (TS, "test_comoving_update_leaves_affine_motion_in_place", {}),
    "sampled_real_rows": (TS, "test_sampled_real_rows_equal_dense_rows", {}),
    "sampled_lub_rows": (TS, "test_sampled_lubrication_rows_equal_dense", {}),
    "lub_pair_psd": (TS, "test_lubrication_pair_symmetric_psd_and_rigid_invariant", {"gap": 0.05}),
    "rotation_blocks": (TT, "test_rotlet_and_rotation_blocks_are_textbook", {"r": 3.3}),
    "faxen_MM": (TT, "test_free_phi_closed_form_matches_kspace_quadrature", {"kind": "MM"}),
    "overlap_clamp": (TT, "test_overlapping_pairs_take_the_contact_blocks", {}),
    "split_independence": (TE, "test_mobility_independent_of_splitting", {}),
    "applied_wave_sum": (TE, "test_applied_wave_sum_equals_dense_wave_matrix", {}),
    "pair_factor": (TB, "test_pairwise_near_field_sampler_has_covariance_R", {}),
    "wave_point_limit": (TT, "test_wave_self_block_closed_form_in_the_point_limit", {}),
    "assembled_strain": (TS, "test_assembled_strain_blocks_equal_affine_bead_motion", {}),
    "philox_known_answers": (TB, "test_philox_known_answers", {}),
    "box_muller_moments": (TB, "test_box_muller_moments", {}),
    "wave_covariance": (TB, "test_wave_sample_covariance_is_the_wave_mobility", {}),
    "wave_covariance_tilt": (TB, "test_wave_sample_covariance_with_tilt", {}),
    "field_layout": (TB, "test_hermitian_field_gives_real_slip", {}),
    "fd_amplitude": (TB, "test_brownian_terms_have_the_fluctuation_dissipation_amplitude", {}),
    "nf_noise_as_force": (TB, "test_near_field_noise_acts_like_an_aggregate_force", {}),
    "precond_sqrt_covariance": (TB, "test_preconditioned_square_root_has_covariance_R", {}),
    "pairwise_covariance": (TB, "test_pairwise_near_field_sampler_has_covariance_R", {}),
    "pair_layout": (TB, "test_pair_normals_layout", {}),
    "generator_layout": (TB, "test_generators_follow_the_documented_counter_layout", {}),
    "rigid_displacement": (TD, "test_displacement_is_rigid_and_first_order_right", {"doublets": DOUBLETS}),
    "rfd_divergence": (TD, "test_rfd_basis_sum_is_the_mobility_divergence", {"doublets": DOUBLETS}),
    "fixman_derivative": (TD, "test_fixman_large_m_is_the_directional_derivative", {"doublets": DOUBLETS}),
    "hertz_closed_form": (TC, "test_single_pair_closed_form", {}),
    "hertz_in_pair_forces": (TC, "test_pair_forces_hertz_term_is_the_closed_form", {}),
    "hertz_rods_newton": (TC, "test_newton_third_law_for_rods", {}),
    "dlvo_minus_gradient": (TC, "test_dlvo_force_is_minus_the_potential_derivative", {}),
    "vdw_far_field": (TC, "test_van_der_waals_far_field_is_the_textbook_sphere_limit", {}),
    "double_layer": (TC, "test_double_layer_screening_and_contact_value", {}),
    "vdw_capped": (TC, "test_van_der_waals_attraction_capped_under_overlap_and_finite_at_contact", {}),
    "newton_cutoff_intrabody": (TC, "test_dlvo_and_hertz_newton_third_law_cutoff_and_intrabody", {}),
}

# (case, planted text, replacement, pins expected to catch it): fsd_oracle
MUTATIONS = [
    ("constraint stresslet factor 1/2 doubled",
     "SC[J] += 0.5 * (np.outer", "SC[J] += 1.0 * (np.outer", ["reciprocity"]),
    ("near-field force left out of the constraint stresslet",
     "Ft = Fm[bb, 0:3] + Fnf[bb, 0:3]", "Ft = Fm[bb, 0:3]", ["reciprocity"]),
    ("near-field stresslet sign",
     'Snf = -(sys_["RSU"] @ dv) + sys_["RSE"] @ sys_["Erep"]',
     'Snf = (sys_["RSU"] @ dv) + sys_["RSE"] @ sys_["Erep"]', ["reciprocity"]),
    ("R_FE strain term dropped from the body rows",
     "RRFE_E = ST.T @ (RFU @ Er + RFE @ Erep)", "RRFE_E = ST.T @ (RFU @ Er)", ["reciprocity"]),
    ("bead right-hand side E.(X - x) (the Table 1 sign)",
     "        b[11 * bb:11 * bb + 3] = E @ r[bb]", "        b[11 * bb:11 * bb + 3] = -E @ r[bb]",
     ["reciprocity", "doublet_in_shear"]),
    ("strain columns of the pair model negated for bead i",
     'Ls[:, 6:11] = 0.5 * r * np.einsum("mab,b->am", EB, n)\n    Ls[:, 11:14]',
     'Ls[:, 6:11] = -0.5 * r * np.einsum("mab,b->am", EB, n)\n    Ls[:, 11:14]', ["affine_strain"]),
    ("squeeze coefficient 1/4 -> 1/2",
     "return 1.0 / (4.0 * x) + (9.0 / 40.0)", "return 1.0 / (2.0 * x) + (9.0 / 40.0)",
     ["lub_asymptotics"]),
    ("squeeze logarithm 9/40 -> 9/20",
     "(9.0 / 40.0) * np.log(1.0 / x)", "(9.0 / 20.0) * np.log(1.0 / x)", ["lub_asymptotics"]),
    ("sliding coefficient 1/6 -> 1/3",
     "B = 6 * PI * eta * a * (1.0 / 6.0)", "B = 6 * PI * eta * a * (1.0 / 3.0)", ["lub_asymptotics"]),
    ("intra-body pairs kept in the near field",
     "            if body[i] == body[j]:\n                continue\n            d = pos[j] - pos[i]\n"
     "            d = min_image(d, L, tilt)\n            if np.linalg.norm(d) >= rcut:",
     "            d = pos[j] - pos[i]\n"
     "            d = min_image(d, L, tilt)\n            if np.linalg.norm(d) >= rcut:", ["intrabody"]),
    ("imposed rotation sign",
     "Om = np.array([0.0, 0.0, -0.5 * gamma])", "Om = np.array([0.0, 0.0, 0.5 * gamma])",
     ["sphere_in_shear"]),
    ("imposed velocity at X read from x instead of y",
     'U[:, 0] += sys_["gamma"] * X[:, 1]', 'U[:, 0] += sys_["gamma"] * X[:, 0]', ["sphere_in_shear"]),
    ("lever-arm sign of Sigma^T",
     '= -np.einsum("abc,b->ac", EPS, r[b])', '= np.einsum("abc,b->ac", EPS, r[b])',
     ["doublet_in_shear"]),
    ("body position the first bead instead of the centroid",
     "X[J] = unw[idx].mean(axis=0)", "X[J] = unw[idx][0]", ["rigid_update"]),
    ("monopole Faxen coefficient 1/6 -> 1/8",
     'FAXEN_C = {"M": 1.0 / 6.0', 'FAXEN_C = {"M": 1.0 / 8.0', ["rpy"]),
    ("dipole Faxen coefficient 1/10 -> 1/6",
     '"D": 1.0 / 10.0}', '"D": 1.0 / 6.0}', ["faxen_DD"]),
    ("rotation-force block factor 1/2 dropped",
     'M[:, 3:6, 0:3] = 0.5 * np.einsum("aef,pfbe->pab"',
     'M[:, 3:6, 0:3] = 1.0 * np.einsum("aef,pfbe->pab"', ["symmetry"]),
    ("Hasimoto factor (1 + k^2/4xi^2) dropped",
     "return (1.0 + x) * np.exp(-x)", "return np.exp(-x)", ["hasimoto_coefficient"]),
    ("wave sum without its -k half",
     "w = 2.0 * hasimoto(kn, xi) / (eta * kn * kn) / L ** 3  # x2: +k and -k",
     "w = 1.0 * hasimoto(kn, xi) / (eta * kn * kn) / L ** 3  # x2: +k and -k", ["sphere_in_shear"]),
    ("torque source sign in wave space",
     "Q[:, :, 3:6] = 0.5j * fD", "Q[:, :, 3:6] = -0.5j * fD", ["le_split"]),
    ("stresslet source sign in wave space",
     "Q[:, :, 6:11] = -1j * fD", "Q[:, :, 6:11] = 1j * fD", ["le_split"]),
    ("Lees-Edwards offset sign in the minimum image",
     "d[..., 0] -= ny * tilt", "d[..., 0] += ny * tilt", ["le_solve"]),
    ("Lees-Edwards offset sign in the reciprocal lattice",
     "n[:, 1] -= tau * n[:, 0]", "n[:, 1] += tau * n[:, 0]", ["le_lattice"]),
    ("Lees-Edwards offset sign in the real-space images",
     "shifts[:, 0] += lat[:, 1] * tilt", "shifts[:, 0] -= lat[:, 1] * tilt", ["le_lattice"]),
    ("quaternion update in the body frame",
     "q = q + 0.5 * dt * quat_mul(om, q)", "q = q + 0.5 * dt * quat_mul(q, om)", ["lab_frame"]),
    ("rotation matrix element with a flipped sign",
     "R[..., 0, 1] = 2 * (x * y - w * z)", "R[..., 0, 1] = 2 * (x * y + w * z)", ["rigid_update"]),
    ("preconditioner scalar zeta0 -> 1/zeta0",
     "Mid[:n1, :n1] = z0 * np.eye(n1)", "Mid[:n1, :n1] = np.eye(n1) / z0", ["precond_exact"]),
    ("near-field block of the saddle matrix with the wrong sign",
     "A[n1:, n1:] = -RRFU", "A[n1:, n1:] = RRFU", ["lub_lowers_mobility"]),
    ("constraint rows of the saddle matrix negated",
     "A[n1:, :n1] = BST.T", "A[n1:, :n1] = -BST.T", ["precond_exact"]),
    ("preconditioner's upper factor sign",
     "Upper[:n1, n1:] = -z0 * BST", "Upper[:n1, n1:] = z0 * BST", ["precond_exact"]),
    ("preconditioner's lower factor sign",
     "Lower[n1:, :n1] = -z0 * BST.T", "Lower[n1:, :n1] = z0 * BST.T", ["precond_exact"]),
    ("preconditioner's Schur blocks without their minus sign",
     "Sinv[6 * J:6 * J + 6, 6 * J:6 * J + 6] = -np.linalg.inv(blk)",
     "Sinv[6 * J:6 * J + 6, 6 * J:6 * J + 6] = np.linalg.inv(blk)", ["precond_exact"]),
    ("preconditioner pairs up to the lubrication cut-off instead of r_p",
     "if np.linalg.norm(d) >= min(rpair, rlub):", "if np.linalg.norm(d) >= max(rpair, rlub):",
     ["precond_within_rp"]),
    ("near-field force taken at u - u_inf + 2 E.r",
     'dv = sys_["ST"] @ sol[n1:] - sys_["Er"]', 'dv = sys_["ST"] @ sol[n1:] + sys_["Er"]',
     ["force_balance"]),
    ("near-field force sign in the outputs",
     'Fnf = -(sys_["RFU"] @ dv) + sys_["RFE"] @ sys_["Erep"]',
     'Fnf = (sys_["RFU"] @ dv) + sys_["RFE"] @ sys_["Erep"]', ["force_balance"]),
    ("imposed rotation added with the wrong sign to Omega",
     'U[:, 3:6] += sys_["Om"]', 'U[:, 3:6] -= sys_["Om"]', ["sphere_in_shear"]),
    ("velocity gradient instead of the rate of strain",
     "E[0, 1] = E[1, 0] = 0.5 * gamma", "E[0, 1] = gamma", ["doublet_in_shear"]),
    ("z component left out of the minimum image",
     "d[..., 2] -= L * np.round(d[..., 2] / L)", "d[..., 2] -= 0.0 * np.round(d[..., 2] / L)",
     ["sampled_lub_rows"]),
    ("co-moving update with the imposed rotation's sign flipped",
     "Ut[:, 5] += 0.5 * comoving_gamma", "Ut[:, 5] -= 0.5 * comoving_gamma", ["comoving_update"]),
    ("co-moving update with the imposed velocity read from x",
     "Ut[:, 0] -= comoving_gamma * X[:, 1]", "Ut[:, 0] -= comoving_gamma * X[:, 0]", ["comoving_update"]),
    ("strain basis element (2zz - xx - yy)/sqrt6 with zz halved",
     "E[1, 0, 0], E[1, 1, 1], E[1, 2, 2] = -1 / s6, -1 / s6, 2 / s6",
     "E[1, 0, 0], E[1, 1, 1], E[1, 2, 2] = -1 / s6, -1 / s6, 1 / s6", ["affine_strain"]),
    ("strain basis element sqrt2 xy normalised to 1/2",
     "E[2, 0, 1] = E[2, 1, 0] = 1 / s2", "E[2, 0, 1] = E[2, 1, 0] = 1 / 2", ["sphere_in_shear"]),
    ("one delta-delta term of the fourth derivative dropped",
     '+ np.einsum("ad,bc->abcd", d, d))', ")", ["rotation_blocks"]),
    ("sign of the Bessel series recursion",
     "term = term * (-(zs * zs) / 2.0) / (k * (2 * n + 2 * k + 1))",
     "term = term * ((zs * zs) / 2.0) / (k * (2 * n + 2 * k + 1))", ["faxen_MM"]),
    ("wave-part quadrature truncated early",
     "K = 2.0 * xi * np.sqrt(46.0)", "K = 2.0 * xi * np.sqrt(8.0)", ["hasimoto_coefficient"]),
    ("strain self mobility 1/(20 pi) instead of 3/(20 pi)",
     "3.0 / (20 * PI * eta * a ** 3)", "1.0 / (20 * PI * eta * a ** 3)", ["sphere_in_shear"]),
    ("real-space self term without the wave part removed",
     "selfb = self_block(a, eta) - w0\n    for i in range(N):", "selfb = self_block(a, eta)\n    for i in range(N):",
     ["sphere_in_shear"]),
    ("rotlet block factor 1/2 dropped",
     "M[:, 0:3, 3:6] = 0.5 * np.einsum", "M[:, 0:3, 3:6] = 1.0 * np.einsum", ["symmetry"]),
    ("relative rotation of the pair with bead j's sign flipped",
     "Lt[:, 14:17] = I3", "Lt[:, 14:17] = -I3", ["lub_pair_psd"]),
    ("lever of bead i's rotation in the surface velocity negated",
     "Ls[:, 3:6] = -0.5 * r * nx      # (r/2) n x dw_i with dw_i = -nu",
     "Ls[:, 3:6] = 0.5 * r * nx      # (r/2) n x dw_i with dw_i = -nu", ["lub_pair_psd"]),
    ("pair factor with bead j's rotation lever negated",
     "Ls[:, 9:12] = -0.5 * r * nx\n    Lt = np.zeros((3, 12))", "Ls[:, 9:12] = 0.5 * r * nx\n    Lt = np.zeros((3, 12))",
     ["pair_factor"]),
    ("free-space blocks of overlapping pairs not clamped to 2a",
     "reff = np.maximum(r, 2.0 * a)", "reff = r", ["overlap_clamp"]),
    ("oracle's own real-space cut-off too short",
     "rc = 2.0 + np.sqrt(46.0) / xi\n    kmax = 2.0 * xi * np.sqrt(46.0)\n    return",
     "rc = 2.0 + np.sqrt(9.0) / xi\n    kmax = 2.0 * xi * np.sqrt(46.0)\n    return", ["split_independence"]),
    ("matrix-free wave sum without the projection I - kk",
     'g = g - kh * np.einsum("pa,pa->p", kh, g)[:, None]  # (I - kk) g', "g = g  # (I - kk) g",
     ["applied_wave_sum"]),
    ("sampled real-space rows without the self term",
     "        out[k] += selfb @ F[i]\n", "        out[k] += 0.0 * selfb @ F[i]\n", ["sampled_real_rows"]),
    ("odd permutations of the Levi-Civita symbol positive",
     "e[0, 2, 1] = e[2, 1, 0] = e[1, 0, 2] = -1.0", "e[0, 2, 1] = e[2, 1, 0] = e[1, 0, 2] = 1.0", ["symmetry"]),
    ("radial derivative (1/r d/dr) r^p with the factor p - 1",
     "return {p - 2: p * c for p, c in poly.items() if p != 0 and c != 0.0}",
     "return {p - 2: (p - 1) * c for p, c in poly.items() if p != 0 and c != 0.0}", ["rpy"]),
    ("sign of the wave part's radial integrals",
     "out[:, n - 1] = (-1.0) ** (n + 1) / (2 * PI * PI * eta) * (integrand @ w)",
     "out[:, n - 1] = (-1.0) ** n / (2 * PI * PI * eta) * (integrand @ w)", ["wave_point_limit"]),
    ("wave part's radial integrals over 2 pi instead of 2 pi^2",
     "out[:, n - 1] = (-1.0) ** (n + 1) / (2 * PI * PI * eta) * (integrand @ w)",
     "out[:, n - 1] = (-1.0) ** (n + 1) / (2 * PI * eta) * (integrand @ w)", ["wave_point_limit"]),
    ("Hasimoto exponent k^2/(2 xi^2) (a consistent change of the splitting)",
     "x = k * k / (4.0 * xi * xi)", "x = k * k / (2.0 * xi * xi)", ["wave_point_limit"]),
    ("monopole and dipole form factors swapped in wave space",
     'fM = form_factor("M", kn * a)\n    fD = form_factor("D", kn * a)',
     'fM = form_factor("D", kn * a)\n    fD = form_factor("M", kn * a)', ["split_independence"]),
    ("dipole form factor j1(z)/z without its 3",
     "return 3.0 * jn_over_zn(1, z)", "return jn_over_zn(1, z)", ["faxen_DD"]),
    ("lever block of Sigma^T transposed",
     '= -np.einsum("abc,b->ac", EPS, r[b])', '= -np.einsum("abc,b->ca", EPS, r[b])', ["force_balance"]),
    ("strain rows picked one place early from the grand resistance",
     "e = np.concatenate([np.arange(11 * b + 6, 11 * b + 11) for b in range(Nt)])",
     "e = np.concatenate([np.arange(11 * b + 5, 11 * b + 10) for b in range(Nt)])", ["assembled_strain"]),
    ("squeeze and sliding coefficients exchanged in the pair matrix",
     'G = A * nn + B * (I3 - nn)\n    Gt = D * (I3 - nn)\n    nx = np.einsum("abc,b->ac", EPS, n)  # n x v = [n]x v',
     'G = B * nn + A * (I3 - nn)\n    Gt = D * (I3 - nn)\n    nx = np.einsum("abc,b->ac", EPS, n)  # n x v = [n]x v',
     ["lub_pair_psd"]),
    ("real-space image sum stored with the wrong transpose",
     "M[i] += acc.transpose(1, 0, 2)", "M[i] += acc.transpose(2, 0, 1)", ["sampled_real_rows"]),
    ("wave vectors with zero first component counted twice",
     "n = n[first > 0]", "n = n[first >= 0]", ["hasimoto_coefficient"]),
    ("sign of the imaginary terms of the wave sum",
     "- (S * ai[:, None]).T @ C + (C * ai[:, None]).T @ S)", "+ (S * ai[:, None]).T @ C - (C * ai[:, None]).T @ S)",
     ["applied_wave_sum"]),
    ("body rows of the right-hand side with the wrong sign",
     "b[n1:] = -(FP + RRFE_E)", "b[n1:] = (FP + RRFE_E)", ["force_balance"]),
    ("squeeze coefficient not shifted to vanish at the cut-off",
     "A = 6 * PI * eta * a * (sq(e) - sq(ec))", "A = 6 * PI * eta * a * sq(e)", ["intrabody"]),
    ("Lees-Edwards minimum image wrapping x before the offset shift",
     "    ny = np.round(d[..., 1] / L)\n    d[..., 0] -= ny * tilt\n    d[..., 1] -= ny * L\n"
     "    d[..., 0] -= L * np.round(d[..., 0] / L)",
     "    ny = np.round(d[..., 1] / L)\n    d[..., 0] -= L * np.round(d[..., 0] / L)\n"
     "    d[..., 0] -= ny * tilt\n    d[..., 1] -= ny * L", ["le_minimum_image"]),
    ("sampled lubrication rows with the torque lever negated",
     "out[k, 3:6] += f[3:6] + np.cross(r[b], f[0:3])", "out[k, 3:6] += f[3:6] - np.cross(r[b], f[0:3])",
     ["sampled_lub_rows"]),
]
CASES = [("fsd_oracle",) + m for m in MUTATIONS]

# brownian_oracle, drift_oracle, contact_oracle
CASES += [
    ("brownian_oracle", "Philox key schedule constant",
     "k0 = (k0 + 0x9E3779B9) & M32", "k0 = (k0 + 0x9E3779B8) & M32", ["philox_known_answers"]),
    ("brownian_oracle", "Box-Muller radius without the factor 2",
     "r0 = np.sqrt(-2.0 * np.log(u[0]))", "r0 = np.sqrt(-np.log(u[0]))", ["box_muller_moments"]),
    ("brownian_oracle", "wave sample without its -k half",
     "wts.append(1.0 if kx == 0 else 2.0)", "wts.append(1.0 if kx == 0 else 1.0)", ["wave_covariance"]),
    ("brownian_oracle", "wave sample on the sheared lattice with the offset sign flipped",
     "m[:, 1] -= (tilt / L) * m[:, 0]", "m[:, 1] += (tilt / L) * m[:, 0]", ["wave_covariance_tilt"]),
    ("brownian_oracle", "conjugate mirror of the kx = 0 plane dropped",
     "xi[:, kz, ky, kx] = np.conj(v) if conj else v", "xi[:, kz, ky, kx] = v", ["field_layout"]),
    ("brownian_oracle", "Nyquist plane of the random field kept",
     "xi[:, :, :, n // 2] = 0", "xi[:, :, :, n // 2] *= 1", ["field_layout"]),
    ("brownian_oracle", "Brownian amplitude sqrt(kT/dt) instead of sqrt(2 kT/dt)",
     "s = np.sqrt(2.0 * kT / dt)", "s = np.sqrt(kT / dt)", ["fd_amplitude"]),
    ("brownian_oracle", "near-field Brownian force added with the wrong sign",
     'b[11 * N:] -= sys_["ST"].T', 'b[11 * N:] += sys_["ST"].T', ["nf_noise_as_force"]),
    ("brownian_oracle", "preconditioned square root with the transposed factor",
     "return Lm @ sqrtm_apply(G @ R @ G.T, v)", "return Lm.T @ sqrtm_apply(G @ R @ G.T, v)",
     ["precond_sqrt_covariance"]),
    ("brownian_oracle", "pair noise scattered to bead j with the wrong sign",
     "out[j] += v[6:]", "out[j] -= v[6:]", ["pairwise_covariance"]),
    ("brownian_oracle", "pair counter on another generator stream",
     "(i & M32, (5 << 8) | call, j & M32, step & M32)", "(i & M32, (4 << 8) | call, j & M32, step & M32)",
     ["pair_layout"]),
    ("drift_oracle", "random displacement rotated by twice the angle",
     "0.5 * h * v[:, 3:6]", "h * v[:, 3:6]", ["rigid_displacement"]),
    ("drift_oracle", "RFD with the full step on each side",
     "p = displaced(pos, body, L, dq, 0.5 * s * eps, tilt)", "p = displaced(pos, body, L, dq, s * eps, tilt)",
     ["rfd_divergence"]),
    ("drift_oracle", "modified Fixman factor m instead of m/2",
     '0.5 * m * (o1["U"] - o0["U"])', 'm * (o1["U"] - o0["U"])', ["fixman_derivative"]),
    ("drift_oracle", "modified Fixman stresslet sign",
     '-0.5 * m * (o1["SH"] - o0["SH"])', '0.5 * m * (o1["SH"] - o0["SH"])', ["fixman_derivative"]),
    ("contact_oracle", "Hertz exponent 1 instead of 3/2",
     "f = kn * delta ** 1.5 * d / dist", "f = kn * delta ** 1.0 * d / dist", ["hertz_closed_form"]),
    ("contact_oracle", "Hertz exponent 1 in the combined force routine",
     "f += kn * (2.0 * a - dist) ** 1.5", "f += kn * (2.0 * a - dist) ** 1.0", ["hertz_in_pair_forces"]),
    ("contact_oracle", "sign of the van der Waals logarithm",
     "+ np.log((rv * rv - s2) / (rv * rv)))", "- np.log((rv * rv - s2) / (rv * rv)))",
     ["dlvo_minus_gradient", "vdw_far_field"]),
    ("contact_oracle", "van der Waals prefactor A/3 instead of A/6",
     "vdw = -A_H / 6.0 * (2.0 * a * a / (rv * rv - s2)", "vdw = -A_H / 3.0 * (2.0 * a * a / (rv * rv - s2)",
     ["vdw_far_field"]),
    ("contact_oracle", "double layer screened twice as fast",
     "el = a * a / r * Z * np.exp(-kappa * (r - 2.0 * a))",
     "el = a * a / r * Z * np.exp(-2 * kappa * (r - 2.0 * a))", ["double_layer"]),
    ("contact_oracle", "power of one van der Waals force term",
     "d2 = -2.0 * a * a * 2.0 / rv ** 3", "d2 = -2.0 * a * a * 2.0 / rv ** 2", ["dlvo_minus_gradient"]),
    ("contact_oracle", "sign of the double-layer force's screening term",
     "del_ = a * a * Z * e * (-1.0 / (r * r) - kappa / r)", "del_ = a * a * Z * e * (-1.0 / (r * r) + kappa / r)",
     ["dlvo_minus_gradient"]),
    ("contact_oracle", "van der Waals attraction not capped under overlap",
     "rv = max(r, 2.0 * a) + h_c", "rv = r + h_c", ["vdw_capped"]),
    ("contact_oracle", "Newton's third law broken for bead j",
     "fb[j] -= f * d / dist", "fb[j] += f * d / dist", ["newton_cutoff_intrabody"]),
    ("brownian_oracle", "slip added to the bead rows with the wrong sign",
     "b[:11 * N] += np.asarray(uB).reshape(-1)", "b[:11 * N] -= np.asarray(uB).reshape(-1)",
     ["fixman_derivative"]),
    ("brownian_oracle", "the two words of the step swapped in the counter",
     "ctr = (index & M32, (stream << 8) | call, step & M32, (step >> 32) & M32)",
     "ctr = (index & M32, (stream << 8) | call, (step >> 32) & M32, step & M32)", ["generator_layout"]),
    ("brownian_oracle", "a bead's noise from the last normals of its calls",
     "_normals(seed, step, stream, b, calls)[:width]", "_normals(seed, step, stream, b, calls)[-width:]",
     ["generator_layout"]),
    ("brownian_oracle", "wave-field draw index with kz and ky transposed",
     "(cz * n + cy) * nh + kx, 2)", "(cy * n + cz) * nh + kx, 2)", ["generator_layout"]),
    ("brownian_oracle", "real-space square root on a cut-off too short",
     "    rc = 2.0 + np.sqrt(46.0) / xi\n    Mr", "    rc = 2.0 + np.sqrt(9.0) / xi\n    Mr", ["fd_amplitude"]),
    ("drift_oracle", "random displacement translated backwards",
     "Xn = X + h * v[:, 0:3]", "Xn = X - h * v[:, 0:3]", ["rigid_displacement"]),
    ("contact_oracle", "Hertz force pointing from i to j (attraction)",
     "            d = F.min_image(unw[i] - unw[j], L, tilt)\n            dist = np.linalg.norm(d)\n            delta",
     "            d = F.min_image(unw[j] - unw[i], L, tilt)\n            dist = np.linalg.norm(d)\n            delta",
     ["hertz_closed_form"]),
    ("contact_oracle", "DLVO forces beyond their cut-off",
     "if dist < r_cut and (A_H", "if dist < 2 * r_cut and (A_H", ["newton_cutoff_intrabody"]),
    ("contact_oracle", "double-layer potential a/r instead of a^2/r",
     "el = a * a / r * Z * np.exp", "el = a / r * Z * np.exp", ["double_layer"]),
    ("contact_oracle", "Hertz contact acting beyond touching",
     "if kn > 0.0 and dist < 2.0 * a:", "if kn > 0.0 and dist < 2.0 * a + 0.2:", ["newton_cutoff_intrabody"]),
    ("contact_oracle", "Hertz torque as F x r",
     "                fb[j] -= f\n    nb = int(body.max()) + 1\n    out = np.zeros((nb, 6))\n    for b in range(Nt):\n"
     "        out[body[b], :3] += fb[b]\n        out[body[b], 3:] += np.cross(r[b], fb[b])",
     "                fb[j] -= f\n    nb = int(body.max()) + 1\n    out = np.zeros((nb, 6))\n    for b in range(Nt):\n"
     "        out[body[b], :3] += fb[b]\n        out[body[b], 3:] += np.cross(fb[b], r[b])", ["hertz_rods_newton"]),
    ("contact_oracle", "aggregate torque as F x r",
     "fb[j] -= f * d / dist\n    nb = int(body.max()) + 1\n    out = np.zeros((nb, 6))\n    for b in range(Nt):\n"
     "        out[body[b], :3] += fb[b]\n        out[body[b], 3:] += np.cross(r[b], fb[b])",
     "fb[j] -= f * d / dist\n    nb = int(body.max()) + 1\n    out = np.zeros((nb, 6))\n    for b in range(Nt):\n"
     "        out[body[b], :3] += fb[b]\n        out[body[b], 3:] += np.cross(fb[b], r[b])",
     ["newton_cutoff_intrabody"]),
]


def _mutant(module, old, new):
    src = os.path.join(ROOT, "oracle", module + ".py")
    with open(src) as f:
        text = f.read()
    assert text.count(old) == 1, "planted text no longer occurs exactly once in " + module
    mod = types.ModuleType("oracle." + module + "_mutant")
    mod.__file__ = src
    mod.__package__ = "oracle"  # its relative imports resolve to the real oracle modules
    exec(compile(text.replace(old, new), src + " (mutant)", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("module,case,old,new,pins", CASES, ids=[c[1] for c in CASES])
def test_planted_mistake_fails_a_pin(module, case, old, new, pins, monkeypatch):
    mod = _mutant(module, old, new)
    failed = []
    for name in pins:
        tmod, fn, kw = PINS[name]
        monkeypatch.setattr(tmod, HANDLE[module], mod)
        try:
            # a mutant may divide by zero or take the log of a negative
            # number on its way to failing a pin
            with np.errstate(all="ignore"), warnings.catch_warnings():
                warnings.simplefilter("ignore", RuntimeWarning)
                getattr(tmod, fn)(**kw)
        except AssertionError:
            failed.append(name)
    assert failed, "no pin caught: " + case
