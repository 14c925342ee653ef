"""Writes tests/golden/box3d_rk4_step.txt: one classical RK4 step (Sec. 3.4, dt = 0.01) of the full
48^3 periodic box (dG degree 2, l_max = 5, N = 107,495,424) from its seeded initial condition, at a
few sampled cells, computed by the FP64 oracle.

The full box is too large to assemble, but its coefficients are constant and one RK4 step couples a
cell only to cells at most four cells away (four stages, each reaching the face neighbours).  So the
step at a sampled cell equals the step at the centre of a 9 x 9 x 9 sub-box of the same cells with
the same initial data: whatever the sub-box's own boundary does reaches at most four cells inward
and never the centre.  The oracle assembles that sub-box (oracle/dg.py) and steps it
(oracle/steppers.py).

Calls only the oracle and the seeded input definitions (paper_2501_05110_gb300/workloads.py).
Run:  python tests/golden/make_box3d_rk4_step.py   (a few minutes per cell, ~20 GB RAM)
"""
import copy
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import dg, steppers  # noqa: E402
from paper_2501_05110_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "box3d_rk4_step.txt")
CENTRES = [(24, 24, 24), (7, 40, 13), (47, 0, 31)]  # (ix, iy, iz) of the full 48^3 box
R = 4


def main():
    prob = W.box3d()
    nc = 48
    e = prob.edges[0]
    h = e[1] - e[0]
    lines = []
    for ctr in CENTRES:
        t0 = time.time()
        sub = copy.copy(prob)
        # cells ctr-R .. ctr+R along each axis; past the box ends the edges continue (the initial
        # condition is periodic, the coefficients constant)
        sub.edges = [e[0] + h * np.arange(c - R, c + R + 2, dtype=float) for c in ctr]
        d = dg.Discretisation(sub)
        pts = d.gauss_points().reshape(-1, 3)  # (ncell * 27, 3), cell-major
        f0 = sub.f0(pts).reshape(d.mesh.ncell, d.mesh.nloc, d.n)  # values at the Gauss points
        y0 = f0.transpose(0, 2, 1).reshape(-1)                     # canonical nodal layout
        z1 = steppers.rk4(d.M, d.D, d.h, d.from_gauss_nodal(y0), sub.dt, 1)
        y1 = d.to_gauss_nodal(z1).reshape(d.mesh.ncell, -1)
        mid = R + (2 * R + 1) * R + (2 * R + 1) ** 2 * R
        gcell = ctr[0] % nc + nc * (ctr[1] % nc) + nc * nc * (ctr[2] % nc)
        lines.append(f"S {gcell} " + " ".join(f"{v:.17e}" for v in y1[mid]))
        print(f"cell {ctr}: {time.time() - t0:.0f} s", flush=True)
    with open(OUT, "w") as fh:
        fh.write("# FP64 oracle: one RK4 step (dt = 0.01) of the 48^3 box (k = 2, l_max = 5) from its\n")
        fh.write("# initial condition, at sampled cells (9^3 sub-box argument; Sec. 3.4).\n")
        fh.write("# Written by tests/golden/make_box3d_rk4_step.py from oracle/ only.\n")
        fh.write("# S <global cell> <972 nodal values in canonical order (j, node)>\n")
        fh.write("\n".join(lines) + "\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
