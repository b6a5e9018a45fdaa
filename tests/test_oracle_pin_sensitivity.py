"""The oracle's pins catch plausible mistakes (CPU only).

Each case plants one mistake in a copy of the oracle's source text (a wrong
sign, a dropped term, a wrong coefficient, a transposed operand, a factor of
two), executes the copy as a separate module, and runs the pins expected to
catch it with that module in place of the oracle: at least one of them must
fail.  The oracle package itself is never modified; the same pins pass on it
in their own files.  A planted text that no longer occurs exactly once in the
oracle makes its case fail, so an edit of the oracle cannot silently retire a
case.

The rolling coefficient of the lubrication pair model (8 pi eta a^3 (1/10)
ln(1/eps)) is the one value no pin fixes: it is this build's reading of
functions the paper does not print, and the published two-sphere functions
it stands in for are not of the pair model's form."""

import os
import types

import pytest

import test_oracle_ewald as TE
import test_oracle_lees_edwards as TL
import test_oracle_solve as TS
import test_oracle_tensors as TT

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "fsd_oracle.py")

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
}

# (case, planted text, replacement, pins expected to catch it)
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
]


def _mutant(old, new):
    with open(SRC) as f:
        text = f.read()
    assert text.count(old) == 1, "planted text no longer occurs exactly once in the oracle"
    mod = types.ModuleType("fsd_oracle_mutant")
    mod.__file__ = SRC
    exec(compile(text.replace(old, new), SRC + " (mutant)", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("case,old,new,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(case, old, new, pins, monkeypatch):
    mod = _mutant(old, new)
    failed = []
    for name in pins:
        tmod, fn, kw = PINS[name]
        monkeypatch.setattr(tmod, "O", mod)
        try:
            getattr(tmod, fn)(**kw)
        except AssertionError:
            failed.append(name)
    assert failed, "no pin caught: " + case
