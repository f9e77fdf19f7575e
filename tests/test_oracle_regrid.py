"""Pins of the oracle's regrid (Sec. 2.2: refinement, de-refinement, level
and Hilbert order) against facts independent of the oracle: closed-form flag
sets of planar jumps, brute-force flag sets and grading closures computed
here with numpy and Python sets on small meshes, conservation of the
conserved totals, and refine/de-refine round trips."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2607_20704_gb300 import inputs

GAMMA = 1.4


def _grid(level, fn, extra=2):
    """Complete base level `level` only, allowed to refine `extra` levels."""
    lv, i, j, k = inputs.graded_octs(level, {})
    U = inputs._state(GAMMA, lv, i, j, k, fn)
    return inputs.Problem("grid", level, level + extra, GAMMA, 0.8, lv, i, j, k, U)


def _mesh(prob):
    return oracle.Mesh(*prob.mesh_args(), **prob.params())


def _cells(o, level):
    """(x, y, z) cell coordinates of a level's cells in mesh order, [8n, 3]."""
    keys, _ = o.read(level)
    keys = keys.astype(np.int64)
    oi, oj, ok = (keys >> 40) & 0xFFFFF, (keys >> 20) & 0xFFFFF, keys & 0xFFFFF
    c = np.arange(8)
    x = (2 * oi[:, None] + (c & 1)).ravel()
    y = (2 * oj[:, None] + ((c >> 1) & 1)).ravel()
    z = (2 * ok[:, None] + ((c >> 2) & 1)).ravel()
    return np.stack([x, y, z], axis=1)


def _step_x(x, y, z):
    rho = np.where((x > 0.5), 0.125, 1.0) + 0.0 * y
    p = np.where((x > 0.5), 0.1, 1.0) + 0.0 * z
    zero = 0.0 * x
    return rho, zero, zero, zero, p


def test_planar_jump_flags_the_columns_next_to_it():
    """Jumps at x = 1/2 and (periodic) x = 0: the two cell columns on each
    side of each jump are flagged, and with expansion one more on each
    side; nothing else (the states are piecewise constant)."""
    level = 4
    n = 1 << level
    o = _mesh(_grid(level, _step_x))
    xyz = _cells(o, level)
    for expand, cols in ((0, {n // 2 - 1, n // 2, 0, n - 1}),
                         (1, {n // 2 - 2, n // 2 - 1, n // 2, n // 2 + 1, n - 2, n - 1, 0, 1})):
        f = o.level_flags(level, grad_rho=0.1, grad_p=0.1, expand=expand)
        want = np.isin(xyz[:, 0], sorted(cols))
        assert np.array_equal(f.astype(bool), want), expand


def test_thresholds_decide_on_the_relative_jump():
    """rho jumps by a factor 1.3 (relative jump 2*0.3/2.3 = 0.26): flagged
    at threshold 0.2, not at 0.3; pressure is uniform, so grad_p alone
    flags nothing."""
    def fn(x, y, z):
        rho = np.where(x > 0.5, 1.3, 1.0) + 0.0 * y
        zero = 0.0 * x
        return rho, zero, zero, zero, 1.0 + zero
    o = _mesh(_grid(3, fn))
    assert o.level_flags(3, grad_rho=0.2, grad_p=0, expand=0).any()
    assert not o.level_flags(3, grad_rho=0.3, grad_p=0, expand=0).any()
    assert not o.level_flags(3, grad_rho=0, grad_p=0.01, expand=0).any()


def _blob(x, y, z):
    r2 = (x - 0.4) ** 2 + (y - 0.55) ** 2 + (z - 0.5) ** 2
    rho = np.where(r2 < 0.04, 3.0, 1.0)
    zero = 0.0 * x
    return rho, zero, zero, zero, 1.0 + zero


def test_blob_flags_match_a_brute_force_stencil():
    """Spherical density jump on a 32^3 grid: raw flags are the cells with a
    face neighbour on the other side; expansion is a periodic 3x3x3 dilation
    (computed here with numpy on the cell array)."""
    level = 5
    n = 1 << level
    o = _mesh(_grid(level, _blob))
    xyz = _cells(o, level)
    c = (np.arange(n) + 0.5) / n
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    rho = _blob(X, Y, Z)[0]
    raw = np.zeros_like(rho, bool)
    for ax in range(3):
        for s in (-1, 1):
            raw |= np.roll(rho, s, axis=ax) != rho
    dil = np.zeros_like(raw)
    for dx, dy, dz in itertools.product((-1, 0, 1), repeat=3):
        dil |= np.roll(raw, (dx, dy, dz), axis=(0, 1, 2))
    for expand, want in ((0, raw), (1, dil)):
        f = o.level_flags(level, grad_rho=0.1, grad_p=0.1, expand=expand)
        assert np.array_equal(f.astype(bool), want[xyz[:, 0], xyz[:, 1], xyz[:, 2]]), expand


def test_mass_criterion():
    """rho dx^3 above the threshold, nothing else (no gradients)."""
    level = 4
    o = _mesh(_grid(level, _blob))
    xyz = _cells(o, level)
    _, U = o.read(level)
    m = 2.0 * 2.0 ** (-3 * level)  # between 1 dx^3 and 3 dx^3
    f = o.level_flags(level, grad_rho=0, grad_p=0, mass=m, expand=0)
    assert np.array_equal(f.astype(bool), U[0] * 2.0 ** (-3 * level) > m)


def _closure(o, raw_sets, lmin, lmax):
    """Grading closure of per-level flagged cell sets (brute force): finest
    level first, a flagged cell X of level l flags the level-(l-1) cells
    covering the 27 level-l cells around X."""
    flags = {l: set(raw_sets.get(l, ())) for l in range(lmin, lmax)}
    for l in range(lmax - 1, lmin, -1):
        side = 1 << l
        for (x, y, z) in list(flags[l]):
            for dx, dy, dz in itertools.product((-1, 0, 1), repeat=3):
                flags[l - 1].add((((x + dx) % side) >> 1, ((y + dy) % side) >> 1,
                                  ((z + dz) % side) >> 1))
    return flags


def test_grading_closure_matches_brute_force():
    """Mass-flagged cells on a three-level mesh (a dense ball): the oracle's
    final flags equal the brute-force closure of the raw flags, the new mesh
    is exactly the children of the flagged cells, and it is graded (the
    rebuild validates it)."""
    prob = inputs.random_mesh(3, 6, seed=8)
    c = inputs.cell_centres(prob.level, prob.i, prob.j, prob.k)
    r2 = (c[0] - 0.3) ** 2 + (c[1] - 0.6) ** 2 + (c[2] - 0.45) ** 2
    rho = np.where(r2 < 0.02, 5.0, 1.0)
    zero = np.zeros_like(rho)
    prob.U = inputs.prim_to_cons(prob.gamma, rho, zero, zero, zero, 1.0 + zero)
    o = _mesh(prob)
    m = 3.0 * 2.0 ** (-3 * 5)  # 5 dx^3 at level 5 and coarser: the ball at levels <= 5
    kw = dict(grad_rho=0, grad_p=0, mass=m, expand=0)
    allf = o.flags(**kw)
    raw = {}
    for l in o.levels():
        if l >= prob.levelmax:
            continue
        xyz = _cells(o, l)
        _, U = o.read(l)
        raw[l] = {tuple(v) for v in xyz[U[0] * 2.0 ** (-3 * l) > m]}
    want = _closure(o, raw, prob.levelmin, prob.levelmax)
    for l in o.levels():
        a = o.level_offset(l)
        got = allf[8 * a: 8 * (a + o.num_octs(l))].astype(bool)
        xyz = _cells(o, l)
        exp = np.array([tuple(v) in want.get(l, set()) for v in xyz], bool)
        assert np.array_equal(got, exp), l
    o.regrid(**kw)
    for l in range(prob.levelmin + 1, prob.levelmax + 1):
        keys, _ = o.read(l)
        keys = keys.astype(np.int64)
        got = {((k >> 40) & 0xFFFFF, (k >> 20) & 0xFFFFF, k & 0xFFFFF) for k in keys}
        assert got == want.get(l - 1, set()), l


def _leaf_totals(o):
    t = np.zeros(5)
    for l in o.levels():
        _, U = o.read(l)
        sp = o.read_split(l)
        t += U[:, sp == 0].sum(axis=1) * 2.0 ** (-3 * l)
    return t


@pytest.mark.parametrize("seed", [3, 4])
def test_regrid_conserves_the_totals(seed):
    """New children are conservative prolongations and removed octs leave
    their restricted father: leaf totals are unchanged to round-off."""
    prob = inputs.random_mesh(3, 6, seed=seed)
    o = _mesh(prob)
    t0 = _leaf_totals(o)
    cr, rm = o.regrid(grad_rho=0.05, grad_p=0.05)
    assert cr > 0
    t1 = _leaf_totals(o)
    sc = np.array([abs(t0[0])] * 4 + [abs(t0[4])])
    assert np.all(np.abs(t1 - t0) <= 1e-14 * sc)


def test_refine_then_coarsen_round_trip():
    """Refine everything that the criterion flags, then regrid with every
    criterion off: all octs above the base level go, and the base cells get
    back their values (father = mean of its prolonged children)."""
    prob = _grid(4, _blob, extra=2)
    o = _mesh(prob)
    k0, U0 = o.read(4)
    cr, rm = o.regrid(grad_rho=0.1, grad_p=0.1)
    assert cr > 0 and rm == 0 and o.num_octs(5) == cr
    cr2, rm2 = o.regrid(grad_rho=0, grad_p=0, mass=0)
    assert cr2 == 0 and rm2 == cr and o.levels() == [4]
    k1, U1 = o.read(4)
    assert np.array_equal(k0, k1)
    assert np.max(np.abs(U1 - U0)) <= 1e-15 * np.abs(U0).max()


def test_uniform_state_coarsens_everything_and_refines_nothing():
    prob = inputs.uniform_state(3, 6, seed=9)
    o = _mesh(prob)
    assert not o.flags().any()
    n_above = sum(o.num_octs(l) for l in o.levels() if l > 3)
    cr, rm = o.regrid()
    assert (cr, rm) == (0, n_above) and o.levels() == [3]


def test_refinement_advances_one_level_per_regrid():
    prob = _grid(3, _blob, extra=3)
    o = _mesh(prob)
    for want in (4, 5, 6, 6):
        o.regrid(grad_rho=0.1, grad_p=0.1)
        assert max(o.levels()) == want


def test_new_children_interpolate_linear_data():
    """Density linear in x (slope 0.1): the children created in flagged
    cells away from the periodic seam equal the linear field at their own
    centres (minmod of two equal differences is that difference), which a
    wrong sign or a dropped slope would break."""
    def fn(x, y, z):
        zero = 0.0 * x
        return 1.0 + 0.1 * x + zero, zero, zero, zero, 1.0 + zero
    level = 4
    o = _mesh(_grid(level, fn))
    m = 1.05 * 2.0 ** (-3 * level)  # flags the cells with rho > 1.05, i.e. x > 1/2
    o.regrid(grad_rho=0, grad_p=0, mass=m, expand=0)
    keys, U = o.read(level + 1)
    assert len(keys)
    xyz = _cells(o, level + 1)
    xc = (xyz[:, 0] + 0.5) / (1 << (level + 1))
    interior = (xc > 0.5) & (xc < 0.93)  # fathers not next to the seam at x = 1
    assert interior.sum() > 0
    want = 1.0 + 0.1 * xc[interior]
    assert np.max(np.abs(U[0, interior] - want)) <= 1e-14


@pytest.mark.parametrize("seed,pre,thr", [(3, None, 0.05), (4, None, 0.05), (5, 0.05, 0.3), (7, 0.03, 0.3)])
def test_new_order_from_the_old_one(seed, pre, thr):
    """The regridded mesh's order (level, then Hilbert index) is the old order
    of the kept octs merged by rank with the new octs taken by father (in the
    old order) and sorted within each father's group, because an oct's
    Hilbert index is its father's followed by one octal digit.  The kept and
    new octs are derived here from the oracle's flags and split masks; the
    merge is compared with the order of the oracle's regridded mesh."""
    import bisect
    prob = inputs.random_mesh(3, 6, seed=seed)
    o = _mesh(prob)
    if pre is not None:  # a refined mesh first, so that this regrid also removes octs
        o.regrid(grad_rho=pre, grad_p=pre)
    crit = dict(grad_rho=thr, grad_p=thr)
    F = o.flags(**crit)

    def coords(k):
        k = int(k)
        return (k >> 40) & 0xFFFFF, (k >> 20) & 0xFFFFF, k & 0xFFFFF

    def hkey(l, x, y, z):
        return l, oracle.hilbert3(x, y, z, l - 1)

    old = []  # (level, x, y, z, flags[8], split[8]) in mesh order
    for l in o.levels():
        keys, _ = o.read(l)
        off = o.level_offset(l)
        fl = F[8 * off: 8 * (off + len(keys))].reshape(-1, 8)
        sp = o.read_split(l).reshape(-1, 8)
        old += [(l, *coords(k), fl[q], sp[q]) for q, k in enumerate(keys)]
    where = {(l, x, y, z): q for q, (l, x, y, z, _, _) in enumerate(old)}
    kept, groups = [], []
    for l, x, y, z, fl, sp in old:
        if l == o.levelmin:
            keep = True
        else:
            father = old[where[(l - 1, x >> 1, y >> 1, z >> 1)]]
            keep = bool(father[4][(x & 1) | ((y & 1) << 1) | ((z & 1) << 2)])
        if keep:
            kept.append(hkey(l, x, y, z))
        groups.append(sorted(hkey(l + 1, 2 * x + (c & 1), 2 * y + ((c >> 1) & 1), 2 * z + ((c >> 2) & 1))
                             for c in range(8) if fl[c] and not sp[c]))
    new = [k for g in groups for k in g]
    assert new == sorted(new) and kept == sorted(kept)
    merged = [None] * (len(kept) + len(new))
    for i, k in enumerate(kept):
        merged[i + bisect.bisect_left(new, k)] = k
    for i, k in enumerate(new):
        merged[i + bisect.bisect_left(kept, k)] = k
    created, removed = o.regrid(**crit)
    assert (created, removed) == (len(new), len(old) - len(kept))
    assert created > 0 and (pre is None or removed > 0), (created, removed)
    want = []
    for l in o.levels():
        keys, _ = o.read(l)
        want += [hkey(l, *coords(k)) for k in keys]
    assert merged == want
