"""Writes tests/golden/oracle_direct8.txt from the oracle alone.

The paper prints no worked example of the force path, so this fixture is a
regression record of the FP64 oracle (direct summation with exact Ewald
images, no table): the periodic acceleration a_E of a unit source at a few
separations, and the direct-sum accelerations of eight fixed particles.  It
is regenerated only when the oracle's arithmetic changes for a reason that
names the passage or reading behind it.

    python tests/golden/make_oracle_fixture.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

SEPARATIONS = [(0.1, 0.0, 0.0), (0.25, 0.0, 0.0), (0.2, 0.3, -0.1), (0.45, -0.35, 0.25), (0.01, 0.02, -0.015)]
POSITIONS = [(0.10, 0.20, 0.30), (0.70, 0.25, 0.28), (0.55, 0.90, 0.05), (0.33, 0.61, 0.72),
             (0.95, 0.05, 0.50), (0.12, 0.48, 0.97), (0.81, 0.77, 0.66), (0.40, 0.02, 0.18)]
MASSES = [0.10, 0.15, 0.05, 0.20, 0.12, 0.08, 0.18, 0.12]
EPS = 0.02


def main():
    lines = ["# Regression fixture of the FP64 oracle (exact Ewald sums, alpha = 2, no table).",
             "# Written by tests/golden/make_oracle_fixture.py, which calls only oracle/.",
             "# section ewald: rx ry rz ax ay az  (a_E of a unit source with neutralising background)"]
    for r in SEPARATIONS:
        a = oracle.ewald_acc(np.array(r))
        lines.append("ewald %s" % " ".join("%.17g" % v for v in (*r, *a)))
    acc = oracle.direct_forces(np.array(POSITIONS), np.array(MASSES), EPS, table_n1=None)
    lines.append("# section direct: eps %.17g; per particle: m x y z ax ay az" % EPS)
    for (x, m, a) in zip(POSITIONS, MASSES, acc):
        lines.append("direct %s" % " ".join("%.17g" % v for v in (m, *x, *a)))
    with open(os.path.join(HERE, "oracle_direct8.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
