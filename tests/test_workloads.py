"""The seeded synthetic workloads have the stated shapes and recipes: the 1-D periodic, shock and
3-D box sizes, the batched-shock parameter ranges and total size, the per-cell log-normal nu, and
determinism under their seeds."""
import math

import numpy as np

from paper_2501_05110_gb300 import workloads as W


def test_workload_sizes():
    assert W.periodic_1d().ndofs == 64 * 16 * 3          # 64 cells, l_max 3, k 2
    assert W.shock().ndofs == 256 * 64 * 16 * 4 == 1_048_576
    assert W.box3d().ndofs == 48 ** 3 * 36 * 27 == 107_495_424


def test_batched_shocks_recipe():
    probs = W.batched_shocks()
    assert len(probs) == 512
    nx = np.array([len(p.edges[0]) - 1 for p in probs])
    npc = {len(p.edges[1]) - 1 for p in probs}
    lmax = np.array([p.lmax for p in probs])
    assert npc == {64} and nx.min() >= 64 and nx.max() <= 512
    assert set(lmax.tolist()) == {1, 3, 5, 7}
    for l in (1, 3, 5, 7):  # uniform over the four orders: each within 5 sigma of 128
        assert abs((lmax == l).sum() - 128) < 5 * math.sqrt(512 * 0.25 * 0.75)
    total = sum(p.ndofs for p in probs)
    assert 1.0e9 < total < 1.3e9                        # about 1.13e9 DoFs in all
    again = W.batched_shocks()
    assert [(p.lmax, len(p.edges[0]), p.ndofs) for p in probs] == \
           [(p.lmax, len(p.edges[0]), p.ndofs) for p in again]


def test_lognormal_cell_nu_recipe():
    base = W.shock()
    xe, pe = base.edges
    nu, z = W.lognormal_cell_nu(xe, pe, seed=6)
    assert z.shape == (64, 256)
    assert abs(z.mean()) < 0.02 and abs(z.std() - 1.0) < 0.02
    # at a cell centre nu = p_c exp(0.3 z_c)
    ix, ip = 17, 40
    xc, lnpc = 0.5 * (xe[ix] + xe[ix + 1]), 0.5 * (pe[ip] + pe[ip + 1])
    got = nu(np.array([[xc]]), np.array([math.exp(lnpc)]))[0]
    assert math.isclose(got, math.exp(lnpc) * math.exp(0.3 * z[ip, ix]), rel_tol=1e-14)
    nu2, z2 = W.lognormal_cell_nu(xe, pe, seed=6)
    assert np.array_equal(z, z2)
