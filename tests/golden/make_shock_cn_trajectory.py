"""Writes tests/golden/shock_cn_trajectory.txt: the FP64 oracle's Crank--Nicolson trajectory of the
full parallel-shock workload (256 x 64 cells in (x, ln p), dG degree 1, l_max = 3, dt = 1, 2000
steps; N = 1,048,576), solved exactly by sparse LU (Eq. theta-method with theta = 1/2, Eq.
system-matrix-rhs).

Calls only the oracle (oracle/dg.py, oracle/steppers.py) and the seeded input definitions
(paper_2501_05110_gb300/workloads.py).  Stored per checkpoint step:
  * the nodal values (at the tensor Gauss points, the library's canonical layout) of a fixed set of
    sampled cells;
  * two aggregates over every DoF: the particle number int int f_000 dx d(ln p) (Gauss weights times
    cell size) and the Euclidean norm of the whole nodal vector.
Run:  python tests/golden/make_shock_cn_trajectory.py   (about 40 minutes on one core, ~8 GB RAM)
"""
import os
import sys
import time

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import dg  # noqa: E402
from paper_2501_05110_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "shock_cn_trajectory.txt")
CHECKPOINTS = (1, 10, 100, 500, 1000, 2000)   # aggregates
SAMPLED_AT = (10, 100, 2000)                   # sampled nodal values


def sample_cells(nx=256, npc=64):
    """Cells around the source (x = 0, ln p = 1) and the shock, the domain corners and seeded ones."""
    fixed = [(127, 6), (128, 6), (128, 7), (126, 9), (131, 20), (140, 30), (200, 12), (60, 8),
             (0, 0), (nx - 1, npc - 1), (255, 6)]
    rng = np.random.default_rng(8)
    extra = [(int(i), int(j)) for i, j in zip(rng.integers(0, nx, 5), rng.integers(0, npc, 5))]
    return sorted({ix + nx * ip for ix, ip in fixed + extra})


def main():
    prob = W.shock()
    t0 = time.time()
    d = dg.Discretisation(prob)
    n, nloc = d.n, d.mesh.nloc
    lhs = spla.splu(sp.csc_matrix(d.M + 0.5 * prob.dt * d.D))
    rhs_op = (d.M - 0.5 * prob.dt * d.D).tocsr()
    print(f"assembly + LU: {time.time() - t0:.0f} s", flush=True)
    cells = sample_cells()
    # particle-number weights: Gauss weights on [0,1]^2 times the cell size, on the f_000 rows
    xg, wg = dg.gauss_rule(d.mesh.q)
    wq = np.outer(wg, wg).ravel()  # axis 0 fastest is irrelevant: the rule is symmetric
    hx = np.diff(prob.edges[0])
    hp = np.diff(prob.edges[1])
    area = (hp[:, None] * hx[None, :]).ravel()  # cell index = ix + nx * ip
    z = np.zeros(d.N)
    lines = []
    for step in range(1, 2001):
        z = lhs.solve(rhs_op @ z + prob.dt * d.h)
        if step in CHECKPOINTS:
            y = d.to_gauss_nodal(z)
            f000 = y.reshape(-1, n, nloc)[:, 0, :]
            mass = float((f000 * wq[None, :] * area[:, None]).sum())
            lines.append(f"A {step} {mass:.17e} {np.linalg.norm(y):.17e}")
            if step in SAMPLED_AT:
                yc = y.reshape(-1, n * nloc)
                for c in cells:
                    vals = " ".join(f"{v:.17e}" for v in yc[c])
                    lines.append(f"S {step} {c} {vals}")
            print(f"step {step}: {time.time() - t0:.0f} s", flush=True)
    with open(OUT, "w") as fh:
        fh.write("# FP64 oracle CN trajectory of the 256 x 64 parallel shock (k = 1, l_max = 3, dt = 1),\n")
        fh.write("# exact sparse-LU solves (Eq. theta-method, theta = 1/2; Eq. system-matrix-rhs).\n")
        fh.write("# Written by tests/golden/make_shock_cn_trajectory.py from oracle/ only.\n")
        fh.write("# A <step> <int f_000 dx dlnp> <||nodal vector||_2>\n")
        fh.write(f"# S <step> <cell> <{n * nloc} nodal values in canonical order (j, node)>\n")
        fh.write("\n".join(lines) + "\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
