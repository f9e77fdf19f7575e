"""Pins of the oracle's Poisson solve on a refined level (Sec. 5: the
potential built level by level; Dirichlet values at the level's boundary
through an adjusted diagonal).  The discrete problem is assembled here
independently -- unknowns at the level's cells, the 7-point operator, and
at a face to a cell outside the level the ghost 2 phi_b - phi with phi_b the
mean of the coarse potential of the cell's father and of the coarse cell
across the face -- and solved directly; the oracle's V-cycles must converge
to that solution.  On a level that covers the whole box there is no
boundary and the problem is the periodic one of the base solver."""
import numpy as np

import oracle
from paper_2607_20704_gb300 import inputs


def _cells(keys):
    k = keys.astype(np.int64)
    oi, oj, ok = (k >> 40) & 0xFFFFF, (k >> 20) & 0xFFFFF, k & 0xFFFFF
    c = np.arange(8)
    return np.stack([(2 * oi[:, None] + (c & 1)).ravel(), (2 * oj[:, None] + ((c >> 1) & 1)).ravel(),
                     (2 * ok[:, None] + ((c >> 2) & 1)).ravel()], axis=1)


def _dense_solution(o, L, phic, fourpiG, rho_bar):
    keys, U = o.read(L)
    cells = _cells(keys)
    index = {tuple(c): t for t, c in enumerate(cells)}
    ckeys, _ = o.read(L - 1)
    ccells = _cells(ckeys)
    cindex = {tuple(c): t for t, c in enumerate(ccells)}
    n = len(cells)
    side, cside = 1 << L, 1 << (L - 1)
    A = np.zeros((n, n))
    b = fourpiG * (U[0] - rho_bar) * (2.0 ** -L) ** 2
    for t, (x, y, z) in enumerate(cells):
        pf = phic[cindex[(x // 2, y // 2, z // 2)]]
        for d in range(3):
            for s in (-1, 1):
                q = [x, y, z]
                q[d] = (q[d] + s) % side
                if tuple(q) in index:
                    A[t, index[tuple(q)]] += 1.0
                    A[t, t] -= 1.0
                else:
                    pc = phic[cindex[(q[0] // 2 % cside, q[1] // 2 % cside, q[2] // 2 % cside)]]
                    phib = 0.5 * (pf + pc)
                    A[t, t] -= 2.0  # ghost 2 phi_b - phi, minus the diagonal's phi
                    b[t] -= 2.0 * phib
    return np.linalg.solve(A, b)


def test_refined_level_converges_to_the_direct_solution():
    prob = inputs.sedov(3, 5, radii={4: 0.22, 5: 0.1})
    o = oracle.Mesh(*prob.mesh_args(), **prob.params())
    rng = np.random.default_rng(3)
    for L in (4, 5):
        nc = o.num_octs(L - 1)
        ccells = _cells(o.read(L - 1)[0])
        # a smooth coarse potential with a random component
        phic = np.sin(2 * np.pi * (ccells[:, 0] + 0.5) / (1 << (L - 1))) + 0.1 * rng.standard_normal(8 * nc)
        want = _dense_solution(o, L, phic, 2.0, 0.7)
        phi, res = o.mg_level(L, phic, fourpiG=2.0, rho_bar=0.7, ncycles=40)
        assert np.max(np.abs(phi - want)) <= 1e-10 * np.max(np.abs(want)), L
        assert res[-1] < 1e-8 * res[0]


def test_v_cycles_reduce_the_residual():
    prob = inputs.random_mesh(3, 6, seed=14)
    o = oracle.Mesh(*prob.mesh_args(), **prob.params())
    for L in o.levels()[1:]:
        phic = np.zeros(8 * o.num_octs(L - 1))
        _, res = o.mg_level(L, phic, fourpiG=1.0, rho_bar=0.8, ncycles=6)
        rates = res[1:] / res[:-1]
        assert np.all(rates < 0.35), (L, rates)


def test_complete_level_is_the_periodic_problem():
    """A level that covers the box has no boundary faces: its solution is
    the base solver's at that resolution (both up to a constant)."""
    rng = np.random.default_rng(5)
    lv = [3] * 64 + [4] * 512
    prob = inputs.uniform_grid(3, lambda x, y, z: (1 + 0 * x, 0 * x, 0 * x, 0 * x, 1 + 0 * x))
    # level 4 complete: every base cell split
    from paper_2607_20704_gb300.inputs import graded_octs, cells_of_level
    codes, _, _, _ = cells_of_level(3)
    lvl, i, j, k = graded_octs(3, {3: codes})
    n8 = 8 * lvl.size
    U = np.zeros((5, n8))
    U[0] = 1.0 + 0.3 * rng.standard_normal(n8)
    U[4] = 1.0
    p = inputs.Problem("full", 3, 4, 1.4, 0.8, lvl, i, j, k, U)
    o = oracle.Mesh(*p.mesh_args(), **p.params())
    keys, U4 = o.read(4)
    cells = _cells(keys)
    rho = np.zeros((16, 16, 16))
    rho[cells[:, 0], cells[:, 1], cells[:, 2]] = U4[0]
    rho_bar = rho.mean()
    want, _ = oracle.mg_solve(rho, 1.0 / 16, fourpiG=1.0, ncycles=40)
    phic = np.zeros(8 * o.num_octs(3))
    phi, _ = o.mg_level(4, phic, fourpiG=1.0, rho_bar=rho_bar, ncycles=40)
    got = phi - phi.mean()
    w = want[cells[:, 0], cells[:, 1], cells[:, 2]]
    w = w - w.mean()
    assert np.max(np.abs(got - w)) <= 1e-9 * np.max(np.abs(w))
