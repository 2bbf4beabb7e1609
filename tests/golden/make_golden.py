"""Writes the regression fixtures of this folder from the FP64 oracle only.

The paper prints no worked numerical example for the pressure solve (its
tables hold grid sizes and Nusselt numbers of DNS runs), so these fixtures are
not paper values: they freeze the oracle's results on tiny seeded grids, so
that a change to the oracle's arithmetic shows up as a failing test and has to
name the passage that justifies it.  Run from the repository root:

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import grid, operator, mg, direct  # noqa: E402

CASES = {
    # Section 3.2 steps 1-5 (Eqs. jacobi, skewness) and step 3 (cell volume)
    "metric_triaxial_4x4x8": dict(nr=4, nth=4, nph=8, mapping=2, flattening=0.1, e2=0.05, stretch=2.0),
    # the full sphere with the shell cut (Sections 3.5, 3.7)
    "metric_full_sphere_4x4x8": dict(nr=4, nth=4, nph=8, th0=0.0, th1=float(np.pi), cut=True),
}
SOLVE = ("solution_oblate_4x6x8", dict(nr=4, nth=6, nph=8, mapping=1, flattening=0.1, r_out=1 / 0.6), 19)


def metric_rows(d):
    fm = grid.face_metrics(grid.shell(d))
    return np.concatenate([fm["G0"].ravel(), fm["G1"].ravel(), fm["G2"].ravel(), fm["J"].ravel()])


def solution(d, stencil):
    """Eqs. PC_6 / PC_8: the discrete solution (bordered direct solve, zero
    J-weighted mean) for a seeded right side."""
    sh = grid.shell(d)
    fm = grid.face_metrics(sh)
    A = operator.assemble(sh, fm, stencil)
    f = np.random.default_rng(2024).standard_normal(sh.n)
    b, _ = mg.prepare_rhs(fm["J"], f)
    x, _ = direct.bordered_solve(A, b, fm["J"].ravel())
    return mg.gauge(fm["J"], x)


def write(name, values, header):
    with open(os.path.join(HERE, name + ".txt"), "w") as fh:
        fh.write("# " + header + "\n")
        fh.write("# written by tests/golden/make_golden.py from the FP64 oracle (regression fixture)\n")
        for v in values:
            fh.write(f"{v:.17e}\n")


def main():
    for name, d in CASES.items():
        write(name, metric_rows(d), f"{name}: {d}; G0, G1, G2 face rows then cell |J^-1|, "
                                    "Section 3.2 steps 1-5")
    name, d, st = SOLVE
    write(name, solution(d, st), f"{name}: {d}, {st}-point; x of Eq. PC_8 for f ~ N(0,1) seed 2024, "
                                 "zero J-weighted mean")


if __name__ == "__main__":
    main()
