"""The test-side threshold band of the regrid parity tests (tests/regrid_band.py):
a density jump planted exactly at the threshold is found, jumps clearly
on either side are not, and the reach of an ambiguous flag covers the
neighbourhood that expansion and grading can change."""
import dataclasses

import numpy as np

import regrid_band
from paper_2607_20704_gb300 import inputs


def _slab_problem(b_over_a, level=3):
    """One level (levelmax one above) with rho = 1 for x < 1/2 and b_over_a
    beyond, at rest, uniform pressure."""
    def fn(x, y, z):
        rho = np.where(x < 0.5, 1.0, b_over_a)
        zero = np.zeros_like(rho)
        return rho, zero, zero.copy(), zero.copy(), np.ones_like(rho)
    prob = inputs.uniform_grid(level, fn)
    return dataclasses.replace(prob, levelmax=level + 1)


def _amb(prob, thr):
    import oracle
    o = oracle.Mesh(*prob.mesh_args(), **prob.params())
    return o, regrid_band.ambiguous(o, prob.gamma, prob.levelmax, grad_rho=thr, grad_p=0.0)


def test_jump_at_the_threshold_is_ambiguous():
    # 2 (b - 1) / (1 + b) = 0.1 exactly for b = 2.1 / 1.9 (up to rounding of b)
    prob = _slab_problem(2.1 / 1.9)
    o, amb = _amb(prob, 0.1)
    a = amb[prob.levelmin]
    # the two cell columns on each side of the interfaces at x = 1/2 and x = 0
    n = 1 << prob.levelmin
    assert a.sum() == 4 * n * n, int(a.sum())
    reach = regrid_band.influence(o, amb)[prob.levelmin]
    assert reach.all()  # +-2 cells around every interface column of an 8^3 grid


def test_clear_jumps_are_not():
    for b in (1.2, 1.05):  # J = 0.18 and 0.049 against 0.1
        prob = _slab_problem(b)
        _, amb = _amb(prob, 0.1)
        assert not amb[prob.levelmin].any(), b


def test_reach_is_local():
    """A single ambiguous cell on a 16^3 grid reaches +-2 cells (5^3) at
    its level."""
    prob = _slab_problem(1.5, level=4)
    import oracle
    o = oracle.Mesh(*prob.mesh_args(), **prob.params())
    keys, _ = o.read(4)
    amb = {4: np.zeros(8 * keys.size, bool)}
    amb[4][8 * 37 + 5] = True
    reach = regrid_band.influence(o, amb)[4]
    assert reach.sum() == 125
