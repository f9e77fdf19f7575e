"""The five workload configurations at full size, each in the way the oracle
can check it: the whole state where the oracle finishes in seconds, sampled
members or the finest level where it does not, and conservation where only
a property that holds at any size is affordable."""
import numpy as np
import pytest

from paper_2607_20704_gb300 import inputs
from parity import compare_all

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_20704_gb300 import amr, build
    build.build()
    amr.load()


def _l1(Ug, Uo):
    """L1 error of rho and E relative to the L1 norm of the oracle's."""
    d = np.abs(Ug - Uo).sum(axis=1)
    n = np.maximum(np.abs(Uo).sum(axis=1), 1e-300)
    return d[0] / n[0], d[4] / n[4]


def _leaf_terms(m, l, v):
    """U_v dx^3 of the leaf cells of level l (host copy of the state)."""
    _, U = m.read(l)
    _, sp = m.read_index(l)
    return (U[v, sp == 0] * 2.0 ** (-3 * l)).tolist()


def _leaf_totals(m):
    """Correctly rounded host sums of U dx^3 over the leaf cells (fsum)."""
    import math
    return np.array([math.fsum(x for l in m.levels() for x in _leaf_terms(m, l, v))
                     for v in range(5)])


def test_sod_ten_coarse_steps():
    """Sod tube, 32^3 base octs plus the refined slab, ten coarse W-cycle
    steps (30 level steps): every cell against the oracle, FP64."""
    import oracle
    from paper_2607_20704_gb300 import amr
    prob = inputs.sod()
    g = amr.Mesh(*prob.mesh_args(), **prob.params())
    o = oracle.Mesh(*prob.mesh_args(), **prob.params())
    for _ in range(10):
        dtg = g.advance(1, sync=True)
        dto = o.advance(1)
        assert abs(dtg - dto) <= 1e-11 * dto
    worst = compare_all(g, o, 1e-11)
    print(f"sod 10 coarse steps: worst scaled error {worst:.2e}")
    g.close()


@pytest.mark.parametrize("precision", [8, 4])
def test_sedov_fifty_coarse_steps_conserve(precision):
    """Sedov, levels 7-10, fifty coarse steps (750 level steps): the oracle
    would need minutes, so the run is checked by its conserved totals (mass,
    momentum, energy over leaf cells, periodic box with refluxing).  The
    update conserves exactly in real arithmetic; what drifts is round-off,
    about 1e-14 of the total per level step in FP64 (energy, whose fluxes
    are largest, measured 1.6e-12 after the 750 level steps).  The totals
    are the device's FP64 fixed-order reduction (amr_totals) in both
    precisions, checked once against an exact host sum of the state."""
    import math
    from paper_2607_20704_gb300 import amr
    prob = inputs.sedov()
    g = amr.Mesh(*prob.mesh_args(), **prob.params(), precision=precision)
    t0 = g.totals(0)
    g.advance(50, sync=True)
    t1 = g.totals(0)
    host = _leaf_totals(g)
    n_leaf = prob.leaf_cells()
    for v in range(5):
        absum = math.fsum(abs(x) for l in g.levels() for x in _leaf_terms(g, l, v))
        assert abs(t1[v] - host[v]) <= 2 * n_leaf * 2.0 ** -53 * absum, (v, t1[v], host[v])
    sc = np.array([abs(t0[0])] * 4 + [abs(t0[4])])
    rel = np.abs(t1 - t0) / sc
    print(f"sedov 50 coarse steps, precision {precision}: relative drift {rel}")
    assert np.all(rel <= (1e-11 if precision == 8 else 1e-6)), rel
    for l in g.levels():
        _, U = g.read(l)
        assert np.isfinite(U).all() and U[0].min() > 0
    g.close()


def test_lognormal_five_finest_level_steps():
    """Cosmology-shaped mesh (256^3 base cells, refinement up to level 11):
    five steps of the finest level from the initial state, all finest octs
    against the oracle; FP64 within the chained-step tolerance, FP32 by its
    L1 error."""
    import oracle
    from paper_2607_20704_gb300 import amr
    prob = inputs.lognormal()
    o = oracle.Mesh(*prob.mesh_args(), **prob.params())
    lf = o.levels()[-1]
    dt = o.cfl_dt() * 0.5 ** (lf - prob.levelmin)
    g8 = amr.Mesh(*prob.mesh_args(), **prob.params())
    g4 = amr.Mesh(*prob.mesh_args(), **prob.params(), precision=4)
    for _ in range(5):
        o.step_level(lf, dt)
        g8.step_level(lf, dt)
        g4.step_level(lf, dt)
    worst = compare_all(g8, o, 1e-11, levels=[lf], reflux=False)
    _, Uo = o.read(lf)
    l1 = _l1(g4.read(lf)[1], Uo)
    print(f"lognormal level {lf} x5: FP64 worst {worst:.2e}; FP32 L1 rho {l1[0]:.2e} E {l1[1]:.2e}")
    assert max(l1) < 1e-5, l1
    g8.close()
    g4.close()


def test_batched_ensemble_sampled_members():
    """The 512-mesh ensemble (11.3 M octs) advanced as one batched handle,
    one coarse step in each precision; eight members (the smallest, the
    largest and six drawn at random) against their own oracles."""
    import oracle
    from paper_2607_20704_gb300 import amr
    probs = inputs.batched()
    n = np.array([p.n_oct for p in probs])
    rng = np.random.default_rng(5)
    pick = sorted({int(n.argmin()), int(n.argmax())} |
                  set(int(q) for q in rng.choice(len(probs), 6, replace=False)))
    want = {}
    for q in pick:
        o = oracle.Mesh(*probs[q].mesh_args(), **probs[q].params())
        o.advance(1)
        want[q] = o
    for precision in (8, 4):
        b = amr.Mesh.batch(probs, precision=precision)
        b.advance(1, sync=True)
        for q in pick:
            b.select(q)
            if precision == 8:
                compare_all(b, want[q], 1e-11)
            else:
                for l in want[q].levels():
                    l1 = _l1(b.read(l)[1], want[q].read(l)[1])
                    assert max(l1) < 5e-6, (q, l, l1)
        b.close()
