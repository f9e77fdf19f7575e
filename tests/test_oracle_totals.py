"""Pins of the oracle's conservation totals: a level's total is the exactly
rounded sum of U dx^3 over its leaf cells (math.fsum) within the rounding
bound of a sequential sum, and the levels' totals add up to the mesh total."""
import math

import numpy as np

from paper_2607_20704_gb300 import inputs

U = 2.0 ** -53


def _leaf(o, l):
    _, Uo = o.read(l)
    sp = o.read_split(l).ravel()
    return Uo[:, sp == 0] * 2.0 ** (-3 * l)


def test_level_totals_are_the_leaf_sums():
    import oracle
    prob = inputs.random_mesh(3, 6, seed=21)
    o = oracle.Mesh(*prob.mesh_args(), **prob.params())
    o.advance(1)
    total = np.zeros(5)
    for l in o.levels():
        x = _leaf(o, l)
        got = o.level_totals(l)
        K = x.shape[1]
        for v in range(5):
            exact = math.fsum(x[v].tolist())
            assert abs(got[v] - exact) <= K * U * math.fsum(np.abs(x[v]).tolist()) + 1e-300
        total += got
    t = o.totals()
    K = prob.leaf_cells()
    scale = sum(np.abs(_leaf(o, l)).sum(axis=1) for l in o.levels())
    assert np.all(np.abs(total - t) <= 2 * K * U * scale)


def test_split_cells_are_left_out_and_empty_levels_give_zero():
    import oracle
    prob = inputs.sod(4, 5)
    o = oracle.Mesh(*prob.mesh_args(), **prob.params())
    # a level above levelmax and an unpopulated level sum to zero
    assert np.all(o.level_totals(7) == 0.0)
    # Sod at rest: mass = 0.5 * 1 + 0.5 * 0.125 exactly (the refined slab
    # holds the same states as the cells it replaces)
    m = o.level_totals(4)[0] + o.level_totals(5)[0]
    assert abs(m - 0.5625) <= 1e-15
