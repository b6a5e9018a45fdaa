"""Write the stored oracle solution of the accuracy sub-box.

The step benchmark's suspension (8-bead random-attachment aggregates, bead
volume fraction 0.2, simple shear of rate 1, lubrication cut-off 3a) is too
large for the dense FP64 oracle (Eq. spm_agg as one dense system), so its
accuracy is measured on a sub-box built by the same generator: 48 aggregates,
384 beads, the smallest such box whose side exceeds twice the real-space
cut-off 2a + sqrt(-ln 1e-6)/xi at xi = 0.5 (Sec. 3.2 accuracy rules).  The
dense oracle takes several minutes here, so this script runs it once and
stores the bead positions, aggregate ids, the applied forces and the oracle's
U, Omega and stresslet for two right-hand sides: shear alone (the benchmark's
step), and shear plus random aggregate forces and torques.

Only oracle/ and synth/ are called.  Output: subbox_384_phi02.txt beside this
script.  Run from the repository root:  python tests/golden/make_subbox_reference.py
"""

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import synth  # noqa: E402

N_AGG, N_B, PHI, SEED = 48, 8, 0.2, 2
SHEAR, RLUB = 1.0, 3.0


def main(path=os.path.join(HERE, "subbox_384_phi02.txt")):
    pos, body, L = synth.suspension(N_AGG, N_B, PHI, SEED)
    body = np.asarray(body)
    nb = int(body.max()) + 1
    ft = synth.random_forces(nb, SEED)
    unw = O.body_geometry(pos, body, L)[0]
    M = O.mobility_dense(unw, L)
    cases = []
    for name, FT in (("shear", None), ("shear+forces", ft)):
        out = O.solve(pos, body, L, gamma=SHEAR, FT=FT, rlub=RLUB, M=M)
        cases.append((name, out))
    with open(path, "w") as f:
        f.write("# oracle solution of Eq. spm_agg (dense FP64 Ewald mobility, dense lubrication,\n")
        f.write("# LAPACK solve) for a 384-bead sub-box of the step benchmark's suspension;\n")
        f.write("# written by make_subbox_reference.py (oracle/ and synth/ only)\n")
        f.write("# generator synth.suspension(%d, %d, %g, %d); shear %g; lubrication %ga\n"
                % (N_AGG, N_B, PHI, SEED, SHEAR, RLUB))
        f.write("L %.17g\n" % L)
        f.write("beads %d aggregates %d\n" % (len(pos), nb))
        for p, b in zip(pos, body):
            f.write("x %.17g %.17g %.17g %d\n" % (p[0], p[1], p[2], b))
        for J in range(nb):
            f.write("ft " + " ".join("%.17g" % v for v in ft[J]) + "\n")
        for name, out in cases:
            f.write("case %s residual %.3e\n" % (name, out["rel_residual"]))
            for J in range(nb):
                f.write("U " + " ".join("%.17g" % v for v in out["U"][J]) + "\n")
            for J in range(nb):
                f.write("S " + " ".join("%.17g" % v for v in out["S"][J].reshape(-1)) + "\n")
    return path


def load(path=os.path.join(HERE, "subbox_384_phi02.txt")):
    """Parse the stored file: dict(L, pos, body, ft, cases={name: (U, S)})."""
    pos, body, ft, cases = [], [], [], {}
    cur = None
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            t = line.split()
            if t[0] == "L":
                L = float(t[1])
            elif t[0] == "x":
                pos.append([float(v) for v in t[1:4]])
                body.append(int(t[4]))
            elif t[0] == "ft":
                ft.append([float(v) for v in t[1:]])
            elif t[0] == "case":
                cur = t[1]
                cases[cur] = ([], [])
            elif t[0] == "U":
                cases[cur][0].append([float(v) for v in t[1:]])
            elif t[0] == "S":
                cases[cur][1].append([float(v) for v in t[1:]])
    cases = {k: (np.array(u), np.array(s).reshape(-1, 3, 3)) for k, (u, s) in cases.items()}
    return dict(L=L, pos=np.array(pos), body=np.array(body, dtype=np.int32), ft=np.array(ft),
                cases=cases)


if __name__ == "__main__":
    print(main())
