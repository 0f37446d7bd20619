"""Writes the stored expected values of tests/golden/ from the FP64 oracle
alone (test infrastructure; nothing here touches the CUDA path).

The paper prints no worked numerical example of the solver (its tables are
parallel efficiencies of its CPU machines, Sec. 4), so these fixtures are
oracle outputs kept as regression values: a later change to the oracle's
arithmetic must reproduce them or say, in its commit message, which passage
of the paper justifies the change.

Fixtures (plain text, one value per line after a header):
* config1_32.txt: configuration 1 (32^3, nu = 0.01, dt = 1e-3, ABC plus a
  seeded perturbation on 2 <= |k| <= 4 at rms 0.1, seed 1): energy and
  enstrophy after each of 10 RK2 steps, and the final coefficients of a few
  modes (Sec. 2, Eqs. 1-2; the diagnostics of Sec. 3).
* box_12x18x24.txt: a forced, rotating run on the 12 x 18 x 24 grid of the
  box of sides 2 pi (1, 1.5, 2) (Sec. 5's domains of other aspect ratios),
  5 steps: energy, enstrophy, helicity per step.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1003_4322_gb300 import inputs  # noqa: E402

MODES = [(0, 0, 0, 1), (1, 0, 1, 0), (2, 1, 0, 0), (0, 2, 3, 1), (1, 31, 2, 4), (2, 3, 30, 2)]


def config1():
    p = oracle.Params(n=32, nu=0.01, dt=1e-3)
    a = inputs.config1_state(32, seed=1)
    rows = []
    for _ in range(10):
        a = oracle.step(a, p, 1)
        e, om, _ = oracle.diagnostics(a)
        rows.append(f"{e:.17e} {om:.17e}")
    modes = [f"{c} {x} {y} {z} {a[c, x, y, z].real:.17e} {a[c, x, y, z].imag:.17e}" for c, x, y, z in MODES]
    return ("# config 1, 32^3, nu=0.01, dt=1e-3, seed 1: step-by-step 'energy enstrophy' (10 lines),\n"
            "# then 'component ix iy kz re im' of the state after 10 steps (6 lines)\n"
            + "\n".join(rows + modes) + "\n")


def box():
    kw = dict(n=12, ny=18, nz=24, lx=1.0, ly=1.5, lz=2.0, nu=0.02, dt=2e-3, force_amp=0.5,
              force_k=2, rot=0.8)
    p = oracle.Params(**kw)
    a = inputs.random_solenoidal_grid((12, 18, 24), (1.0, 1.5, 2.0), 0.5, 3.0, 1.0, seed=9)
    rows = []
    for _ in range(5):
        a = oracle.step(a, p, 1)
        e, om, _ = oracle.diagnostics(a, p)
        h, _ = oracle.helicity(a, p)
        rows.append(f"{e:.17e} {om:.17e} {h:.17e}")
    return ("# 12x18x24 grid, box 2pi (1, 1.5, 2), nu=0.02, dt=2e-3, ABC k=2 F=0.5, rot=0.8, start\n"
            "# random_solenoidal_grid(0.5 <= |k| <= 3, rms 1, seed 9): 'energy enstrophy helicity' per step\n"
            + "\n".join(rows) + "\n")


def main():
    with open(os.path.join(HERE, "config1_32.txt"), "w") as f:
        f.write(config1())
    with open(os.path.join(HERE, "box_12x18x24.txt"), "w") as f:
        f.write(box())


if __name__ == "__main__":
    main()
