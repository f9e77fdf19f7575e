"""Pins of the oracle's level step against invariants and special cases:
HLLC special solutions, prolongation, exact preservation of a uniform flow,
conservation with refluxing (and its failure without), identity with the
independent uniform-grid and 1-D solvers, mirror symmetry."""
import numpy as np
import pytest

from paper_2607_20704_gb300 import inputs

G = 1.4


def _cons(r, u, p, v=0.0, w=0.0, g=G):
    return np.array([r, r * u, r * v, r * w, p / (g - 1) + 0.5 * r * (u * u + v * v + w * w)])


def _phys_flux(r, u, p, v=0.0, w=0.0, g=G):
    E = p / (g - 1) + 0.5 * r * (u * u + v * v + w * w)
    return np.array([r * u, r * u * u + p, r * u * v, r * u * w, (E + p) * u])


def _interface_flux(orc, left, right, n=16, dt=1e-3):
    """HLLC flux at the jump x = 1/2 of a piecewise-constant 1-D state, read
    back from one step: with constant data on each side every limited slope
    is zero, so the step is a first-order Godunov step and the cell right of
    the jump changes by dt/dx (F_jump - F_phys(right))."""
    U = np.zeros((5, n))
    U[:, : n // 2] = _cons(*left)[:, None]
    U[:, n // 2:] = _cons(*right)[:, None]
    U1 = orc.step_1d(U.copy(), G, dt)
    dtdx = dt * n
    return (U1[:, n // 2] - U[:, n // 2]) / dtdx + _phys_flux(*right)


def test_hllc_consistency(orc):
    s = (1.3, 0.4, 2.0, 0.3, -0.2)
    F = _interface_flux(orc, s, s)
    np.testing.assert_allclose(F, _phys_flux(*s), rtol=1e-12, atol=1e-12)


def test_hllc_resolves_a_stationary_contact_exactly(orc):
    F = _interface_flux(orc, (1.0, 0.0, 1.0), (0.125, 0.0, 1.0))
    np.testing.assert_allclose(F, [0.0, 1.0, 0.0, 0.0, 0.0], atol=1e-12)


@pytest.mark.parametrize("u", [3.0, -3.0])
def test_hllc_is_upwind_for_supersonic_flow(orc, u):
    L, R = (1.0, u, 1.0), (0.5, u * 1.1, 0.8)
    F = _interface_flux(orc, L, R)
    np.testing.assert_allclose(F, _phys_flux(*(L if u > 0 else R)), rtol=1e-12, atol=1e-12)


def test_hllc_mirror_symmetry(orc):
    L, R = (1.0, 0.3, 1.0), (0.4, -0.2, 0.5)
    F = _interface_flux(orc, L, R)
    Fm = _interface_flux(orc, (R[0], -R[1], R[2]), (L[0], -L[1], L[2]))
    # reflection x -> -x: mass and energy fluxes change sign, momentum flux does not
    np.testing.assert_allclose(Fm, [-F[0], F[1], -F[2], -F[3], -F[4]], rtol=1e-12, atol=1e-13)


def test_prolongation_is_exact_for_linear_data_and_conservative(orc):
    """Ghost children of a father cell sitting in a linear field take the
    linear field's values at their centres; their mean is the father's value."""
    prob = inputs.random_mesh(3, 4, seed=2, n_seeds=1, radius=0.25)
    x, y, z = inputs.cell_centres(prob.level, prob.i, prob.j, prob.k)
    a = np.array([2.0, 0.1, -0.2, 0.3, 5.0])
    b = np.array([[0.5, -0.3, 0.2], [0.1, 0.2, -0.1], [0.0, 0.3, 0.1], [-0.2, 0.1, 0.4], [1.0, -0.5, 0.7]])
    # linear in a window away from the periodic seam: use the father level only
    U = np.stack([(a[v] + b[v, 0] * x + b[v, 1] * y + b[v, 2] * z).ravel() for v in range(5)])
    prob.U = U
    m = orc.Mesh(*prob.mesh_args(), **prob.params())
    keys = m.read_cache(4)
    Ug = m.ghost(4)
    ok = 0
    for s, k in enumerate(keys.tolist()):
        gi, gj, gk = (k >> 40) & 0xFFFFF, (k >> 20) & 0xFFFFF, k & 0xFFFFF
        # fathers at least two coarse cells from the seam see a linear field
        if min(gi, gj, gk) < 2 or max(gi, gj, gk) > 5:
            continue
        for c in range(8):
            xc = (2 * gi + (c & 1) + 0.5) / 16
            yc = (2 * gj + ((c >> 1) & 1) + 0.5) / 16
            zc = (2 * gk + ((c >> 2) & 1) + 0.5) / 16
            np.testing.assert_allclose(Ug[:, 8 * s + c], a + b @ [xc, yc, zc], rtol=1e-13, atol=1e-13)
        ok += 1
    assert ok > 10
    # conservative for any data: mean of children == father
    prob2 = inputs.random_mesh(3, 5, seed=4)
    m2 = orc.Mesh(*prob2.mesh_args(), **prob2.params())
    for l in (4, 5):
        keys = m2.read_cache(l)
        Ug = m2.ghost(l)
        kk, Uc = m2.read(l - 1)
        idx = {kq: t for t, kq in enumerate(kk.tolist())}
        for s, k in enumerate(keys.tolist()):
            gi, gj, gk = (k >> 40) & 0xFFFFF, (k >> 20) & 0xFFFFF, k & 0xFFFFF
            f = idx[orc.pack_key(l - 1, gi >> 1, gj >> 1, gk >> 1)]
            c = (gi & 1) + 2 * (gj & 1) + 4 * (gk & 1)
            np.testing.assert_allclose(Ug[:, 8 * s:8 * s + 8].mean(axis=1), Uc[:, 8 * f + c],
                                       rtol=1e-14, atol=1e-14)


def test_uniform_moving_state_is_preserved(orc):
    """All fluxes are equal: bitwise on one level; with refluxing and
    restriction, to a few ulps (sums of equal terms round)."""
    prob = inputs.uniform_state(3, 5, seed=7)
    m = orc.Mesh(*prob.mesh_args(), **prob.params())
    ref = prob.U[:, 0].copy()
    for _ in range(3):
        m.advance(1)
    for l in m.levels():
        _, U = m.read(l)
        err = np.abs(U - ref[:, None]) / np.abs(ref).max()
        assert err.max() <= 1e-14, err.max()
        assert np.abs(m.read_R(l)).max() <= 1e-14
    one = inputs.uniform_grid(3, lambda x, y, z: tuple(np.full(x.shape, q) for q in (1.3, 0.7, -0.4, 0.25, 2.0)))
    m1 = orc.Mesh(*one.mesh_args(), **one.params())
    ref = one.U[:, 0].copy()
    for _ in range(3):
        m1.advance(1)
    _, U = m1.read(3)
    assert np.array_equal(U, np.repeat(ref[:, None], U.shape[1], axis=1))


@pytest.mark.parametrize("seed", [11, 12])
def test_conservation_with_reflux(orc, seed):
    prob = inputs.random_mesh(3, 5, seed=seed)
    m = orc.Mesh(*prob.mesh_args(), **prob.params())
    t0 = m.totals()
    for _ in range(3):
        m.advance(1)
    t1 = m.totals()
    scale = np.array([abs(t0[0]), abs(t0[0]), abs(t0[0]), abs(t0[0]), abs(t0[4])])
    assert np.all(np.abs(t1 - t0) <= 1e-13 * scale), (t1 - t0) / scale


def test_deepest_hierarchy_conserves_and_keeps_the_coarse_levels_at_rest(orc):
    """Levels 2..15 (the deepest hierarchy), one coarse step = 16,383 level
    steps: mass and energy conserved to round-off, and the coarse levels,
    which the blast cannot reach in one step, keep momenta at round-off
    against the energy present (the scale of the parity tolerance)."""
    prob = inputs.sedov(2, 15, radii={l: 3 * 2.0 ** -l for l in range(3, 16)}, centre=(0.3, 0.7, 0.55))
    m = orc.Mesh(*prob.mesh_args(), **prob.params())
    t0 = m.totals()
    m.advance(1)
    t1 = m.totals()
    assert np.all(np.abs(t1 - t0)[[0, 4]] <= 1e-13 * np.abs(t0[[0, 4]]))
    for l in (2, 3, 4):
        _, U = m.read(l)
        scale = np.sqrt(2.0 * U[0] * U[4]).max()
        assert np.abs(U[1:4]).max() <= 1e-15 * scale, (l, np.abs(U[1:4]).max(), scale)


def test_conservation_fails_without_reflux(orc):
    """Negative control: without refluxing, coarse-fine faces leak."""
    prob = inputs.random_mesh(3, 5, seed=11)
    m = orc.Mesh(*prob.mesh_args(), **prob.params(), reflux=False)
    t0 = m.totals()
    for _ in range(3):
        m.advance(1)
    t1 = m.totals()
    assert np.max(np.abs(t1 - t0)[[0, 4]] / np.abs(t0[[0, 4]])) > 1e-8


def test_single_level_mesh_equals_uniform_grid_solver(orc):
    def fn(x, y, z):
        rho = 1 + 0.3 * np.sin(2 * np.pi * x) * np.cos(4 * np.pi * y) + 0.1 * np.sin(2 * np.pi * z)
        u = 0.5 * np.sin(2 * np.pi * y)
        v = -0.3 * np.cos(2 * np.pi * z)
        w = 0.2 * np.sin(2 * np.pi * x)
        p = 1 + 0.4 * np.cos(2 * np.pi * (x + y))
        return rho, u, v, w, p
    prob = inputs.uniform_grid(4, fn).shuffled(3)
    m = orc.Mesh(*prob.mesh_args(), **prob.params())
    A = inputs.to_array(inputs.uniform_grid(4, fn))
    for _ in range(3):
        dt = m.cfl_dt()
        assert dt == orc.uniform_cfl_dt(A, G, 0.8)
        m.step_level(4, dt)
        orc.uniform_step(A, G, dt)
    kk, U = m.read(4)
    n = 16
    c = np.arange(8)
    I = ((kk >> np.uint64(40)) & np.uint64(0xFFFFF)).astype(np.int64)
    J = ((kk >> np.uint64(20)) & np.uint64(0xFFFFF)).astype(np.int64)
    K = (kk & np.uint64(0xFFFFF)).astype(np.int64)
    gx = (2 * I[:, None] + (c & 1)).ravel()
    gy = (2 * J[:, None] + ((c >> 1) & 1)).ravel()
    gz = (2 * K[:, None] + ((c >> 2) & 1)).ravel()
    assert np.array_equal(U, A[:, gx + n * (gy + n * gz)])


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_3d_sod_equals_1d_solver(orc, axis):
    prob = inputs.sod(4, 4, axis=axis)
    m = orc.Mesh(*prob.mesh_args(), **prob.params())
    n = 16
    xs = (np.arange(n) + 0.5) / n
    U1 = np.zeros((5, n))
    left = xs < 0.5
    U1[0] = np.where(left, 1.0, 0.125)
    U1[4] = np.where(left, 1.0, 0.1) / 0.4
    for _ in range(5):
        dt = m.cfl_dt()
        m.step_level(4, dt)
        orc.step_1d(U1, G, dt)
    kk, U = m.read(4)
    c = np.arange(8)
    coord = [((kk >> np.uint64(s)) & np.uint64(0xFFFFF)).astype(np.int64) for s in (40, 20, 0)]
    g = (2 * coord[axis][:, None] + ((c >> axis) & 1)).ravel()
    perm = [0, 1 + axis, *(1 + a for a in range(3) if a != axis), 4]
    for v in range(5):
        src = U1[{0: 0, 4: 4}.get(v, 1)] if v in (0, 4) or v == 1 + axis else np.zeros(n)
        np.testing.assert_allclose(U[v], src[g], rtol=1e-14, atol=1e-14)
    del perm


def test_mirror_symmetry_of_a_centred_blast(orc):
    prob = inputs.sedov(3, 5, radii={5: 0.1, 4: 0.2}, gamma=5.0 / 3.0)
    m = orc.Mesh(*prob.mesh_args(), **prob.params())
    for _ in range(4):
        m.advance(1)
    for l in m.levels():
        kk, U = m.read(l)
        side = 1 << l
        idx = {}
        cells = []
        for t, k in enumerate(kk.tolist()):
            a, b, c0 = (k >> 40) & 0xFFFFF, (k >> 20) & 0xFFFFF, k & 0xFFFFF
            for c in range(8):
                cells.append((2 * a + (c & 1), 2 * b + ((c >> 1) & 1), 2 * c0 + ((c >> 2) & 1)))
                idx[cells[-1]] = 8 * t + c
        scale = np.abs(U).max(axis=1)
        for (x, y, z), s in idx.items():
            for ax in range(3):
                mc = [x, y, z]
                mc[ax] = side - 1 - mc[ax]
                t = idx[tuple(mc)]
                sign = np.ones(5)
                sign[1 + ax] = -1
                assert np.all(np.abs(U[:, t] - sign * U[:, s]) <= 1e-13 * scale)
