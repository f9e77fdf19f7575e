"""FP64 conservation totals on the device (amr_totals) against the oracle and
against exact host sums, in both precisions.

Bounds: a sum of K terms evaluated in any order is within (K - 1) u of
sum |x| of the exact sum (u = 2^-53), so two evaluations in different orders
differ by at most 2 K u sum |x|, and one evaluation differs from the
correctly rounded sum (math.fsum) by at most K u sum |x|."""
import math

import numpy as np
import pytest

from paper_2607_20704_gb300 import inputs

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_20704_gb300 import amr, build
    build.build()
    amr.load()


def _leaf(g, l):
    """U dx^3 of the leaf cells of level l of a GPU mesh (host copy)."""
    _, Um = g.read(l)
    sp = g.read_index(l)[1].ravel()
    return Um[:, sp == 0] * 2.0 ** (-3 * l)


def test_fresh_mesh_totals_match_the_oracle():
    """Identical states on both sides: per level and over all levels."""
    import oracle
    from paper_2607_20704_gb300 import amr
    for prob in (inputs.random_mesh(3, 6, seed=51), inputs.sedov(4, 6, radii={5: 0.15, 6: 0.08})):
        g = amr.Mesh(*prob.mesh_args(), **prob.params())
        o = oracle.Mesh(*prob.mesh_args(), **prob.params())
        scale_all = np.zeros(5)
        for l in o.levels():
            x = _leaf(g, l)
            scale = np.abs(x).sum(axis=1)
            scale_all += scale
            K = x.shape[1]
            assert np.all(np.abs(g.totals(l) - o.level_totals(l)) <= 2 * K * U * scale), l
        K = prob.leaf_cells()
        assert np.all(np.abs(g.totals(0) - o.totals()) <= 2 * K * U * scale_all)
        g.close()


@pytest.mark.parametrize("precision", [8, 4])
def test_totals_after_steps_are_the_exact_leaf_sums(precision):
    """After coarse steps: each level's device total against the correctly
    rounded sum of the state as read back (FP32 states widened exactly);
    calls repeat bit for bit."""
    from paper_2607_20704_gb300 import amr
    prob = inputs.random_mesh(3, 6, seed=52)
    g = amr.Mesh(*prob.mesh_args(), **prob.params(), precision=precision)
    g.advance(2, sync=True)
    for l in g.levels():
        x = _leaf(g, l)
        got = g.totals(l)
        assert np.array_equal(got, g.totals(l))
        for v in range(5):
            exact = math.fsum(x[v].tolist())
            assert abs(got[v] - exact) <= x.shape[1] * U * np.abs(x[v]).sum() + 1e-300, (l, v)
    g.close()


def test_totals_of_a_batch_member_and_of_an_empty_level():
    from paper_2607_20704_gb300 import amr
    probs = [inputs.sod(3, 5), inputs.random_mesh(3, 5, seed=53)]
    b = amr.Mesh.batch(probs)
    for q, pr in enumerate(probs):
        a = amr.Mesh(*pr.mesh_args(), **pr.params())
        b.select(q)
        for l in [0] + a.levels():
            assert np.array_equal(b.totals(l), a.totals(l)), (q, l)
        assert np.all(b.totals(9) == 0.0)
        a.close()
    b.close()


def test_periodic_refluxed_mesh_conserves_on_the_device():
    """Mass, momentum and energy over leaf cells stay constant to round-off
    over W-cycles with reflux (the oracle's pinned property), read by the
    device reduction."""
    from paper_2607_20704_gb300 import amr
    prob = inputs.random_mesh(3, 6, seed=54)
    g = amr.Mesh(*prob.mesh_args(), **prob.params())
    t0 = g.totals(0)
    g.advance(3, sync=True)
    t1 = g.totals(0)
    sc = np.array([abs(t0[0])] * 4 + [abs(t0[4])])
    assert np.all(np.abs(t1 - t0) <= 1e-13 * sc), np.abs(t1 - t0) / sc
    g.close()
