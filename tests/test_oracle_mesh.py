"""Pins of the oracle's mesh machinery against brute force on tiny meshes:
level/Hilbert order (Sec. 2.2), hash_get lookups (Sec. 2.1), the 27-entry
neighbour array and ghost (cache) octs (Sec. 2.3), split flags, validation."""
import numpy as np
import pytest

from paper_2607_20704_gb300 import inputs


def _mesh(orc, prob, **kw):
    return orc.Mesh(*prob.mesh_args(), **prob.params(), **kw)


def _keys_by_input(orc, prob):
    return [orc.pack_key(l, a, b, c) for l, a, b, c in
            zip(prob.level.tolist(), prob.i.tolist(), prob.j.tolist(), prob.k.tolist())]


@pytest.fixture(scope="module")
def small(orc):
    prob = inputs.random_mesh(2, 4, seed=3, n_seeds=2, radius=0.3).shuffled(5)
    return prob, _mesh(orc, prob)


def test_order_is_level_then_hilbert(orc, small):
    prob, m = small
    expect = []
    for idx, (l, a, b, c) in enumerate(zip(prob.level.tolist(), prob.i.tolist(),
                                           prob.j.tolist(), prob.k.tolist())):
        expect.append((l, orc.hilbert3(a, b, c, l - 1), idx, orc.pack_key(l, a, b, c)))
    expect.sort()
    got = np.concatenate([m.read(l)[0] for l in range(prob.levelmin, prob.levelmax + 1)])
    assert [e[3] for e in expect] == got.tolist()
    off = 0
    for l in range(prob.levelmin, prob.levelmax + 1):
        assert m.level_offset(l) == off
        off += m.num_octs(l)


def test_state_follows_its_oct(orc, small):
    prob, m = small
    keys = _keys_by_input(orc, prob)
    where = {k: t for t, k in enumerate(keys)}
    for l in range(prob.levelmin, prob.levelmax + 1):
        kk, U = m.read(l)
        split = m.read_split(l)
        for t, k in enumerate(kk.tolist()):
            s = where[k]
            for c in range(8):
                if not split[8 * t + c]:
                    assert np.array_equal(U[:, 8 * t + c], prob.U[:, 8 * s + c])


def test_lookup_matches_dictionary(orc, small):
    prob, m = small
    sorted_keys = np.concatenate([m.read(l)[0] for l in range(prob.levelmin, prob.levelmax + 1)])
    for idx, k in enumerate(sorted_keys.tolist()):
        assert m.lookup(k) == idx
    rng = np.random.default_rng(0)
    present = set(sorted_keys.tolist())
    for _ in range(500):
        l = int(rng.integers(prob.levelmin, prob.levelmax + 2))
        side = 1 << (l - 1)
        k = orc.pack_key(l, *rng.integers(0, side, 3).tolist())
        assert m.lookup(k) == (sorted_keys.tolist().index(k) if k in present else -1)


def test_neighbours_and_cache_by_brute_force(orc, small):
    prob, m = small
    allkeys = [(l, a, b, c) for l, a, b, c in zip(prob.level.tolist(), prob.i.tolist(),
                                                  prob.j.tolist(), prob.k.tolist())]
    sorted_keys = np.concatenate([m.read(l)[0] for l in range(prob.levelmin, prob.levelmax + 1)]).tolist()
    missing = set()
    expect = {}
    for l in range(prob.levelmin, prob.levelmax + 1):
        side = 1 << (l - 1)
        for k in m.read(l)[0].tolist():
            a, b, c = (k >> 40) & 0xFFFFF, (k >> 20) & 0xFFFFF, k & 0xFFFFF
            row = []
            for dz in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        t = (l, (a + dx) % side, (b + dy) % side, (c + dz) % side)
                        # O(N) scan of the raw input list
                        found = [s for s, q in enumerate(allkeys) if q == t]
                        pk = orc.pack_key(*t)
                        if found:
                            row.append(("real", sorted_keys.index(pk)))
                        else:
                            row.append(("miss", pk))
                            missing.add(pk)
            expect[k] = row
    cache = sorted(missing)
    got_cache = np.concatenate([m.read_cache(l) for l in range(0, prob.levelmax + 1)]).tolist()
    assert got_cache == cache
    for l in range(prob.levelmin, prob.levelmax + 1):
        nb = m.read_nbr(l)
        for t, k in enumerate(m.read(l)[0].tolist()):
            for e, (kind, val) in enumerate(expect[k]):
                if kind == "real":
                    assert nb[t, e] == val
                else:
                    assert nb[t, e] == -(1 + cache.index(val))
            assert nb[t, 13] == m.level_offset(l) + t


def test_split_flags_by_brute_force(orc, small):
    prob, m = small
    present = set(zip(prob.level.tolist(), prob.i.tolist(), prob.j.tolist(), prob.k.tolist()))
    for l in range(prob.levelmin, prob.levelmax + 1):
        split = m.read_split(l)
        for t, k in enumerate(m.read(l)[0].tolist()):
            a, b, c = (k >> 40) & 0xFFFFF, (k >> 20) & 0xFFFFF, k & 0xFFFFF
            for q in range(8):
                child = (l + 1, 2 * a + (q & 1), 2 * b + ((q >> 1) & 1), 2 * c + ((q >> 2) & 1))
                assert bool(split[8 * t + q]) == (child in present)


def test_split_cells_hold_the_mean_of_their_children(orc, small):
    prob, m = small
    for l in range(prob.levelmin, prob.levelmax):
        kk, U = m.read(l)
        split = m.read_split(l)
        kf, Uf = m.read(l + 1)
        idx = {k: t for t, k in enumerate(kf.tolist())}
        for t, k in enumerate(kk.tolist()):
            a, b, c = (k >> 40) & 0xFFFFF, (k >> 20) & 0xFFFFF, k & 0xFFFFF
            for q in range(8):
                if split[8 * t + q]:
                    ck = orc.pack_key(l + 1, 2 * a + (q & 1), 2 * b + ((q >> 1) & 1), 2 * c + ((q >> 2) & 1))
                    s = idx[ck]
                    mean = Uf[:, 8 * s:8 * s + 8].mean(axis=1)
                    np.testing.assert_allclose(U[:, 8 * t + q], mean, rtol=1e-14, atol=1e-15)


def test_rejects_duplicates(orc):
    prob = inputs.random_mesh(2, 3, seed=1)
    lv = np.concatenate([prob.level, prob.level[-1:]])
    i = np.concatenate([prob.i, prob.i[-1:]])
    j = np.concatenate([prob.j, prob.j[-1:]])
    k = np.concatenate([prob.k, prob.k[-1:]])
    U = np.concatenate([prob.U, prob.U[:, -8:]], axis=1)
    with pytest.raises(orc.OracleError) as e:
        orc.Mesh(lv, i, j, k, U, **prob.params())
    assert e.value.code == 4


def test_rejects_grading_violation(orc):
    # a level-4 oct whose father's neighbourhood at level 3 is missing
    prob = inputs.uniform_grid(2, lambda x, y, z: (1 + 0 * x, 0 * x, 0 * x, 0 * x, 1 + 0 * x))
    lv = np.concatenate([prob.level, [3, 4]]).astype(np.uint8)
    i = np.concatenate([prob.i, [0, 0]]).astype(np.uint32)
    j = np.concatenate([prob.j, [0, 0]]).astype(np.uint32)
    k = np.concatenate([prob.k, [0, 0]]).astype(np.uint32)
    U = np.concatenate([prob.U, np.ones((5, 16))], axis=1)
    with pytest.raises(orc.OracleError) as e:
        orc.Mesh(lv, i, j, k, U, levelmin=2, levelmax=4, gamma=1.4)
    assert e.value.code == 3


def test_rejects_incomplete_base_and_bad_levels(orc):
    prob = inputs.uniform_grid(3, lambda x, y, z: (1 + 0 * x, 0 * x, 0 * x, 0 * x, 1 + 0 * x))
    with pytest.raises(orc.OracleError) as e:
        orc.Mesh(prob.level[1:], prob.i[1:], prob.j[1:], prob.k[1:], prob.U[:, 8:], **prob.params())
    assert e.value.code == 3
    bad = prob.level.copy()
    bad[0] = 5
    with pytest.raises(orc.OracleError) as e:
        orc.Mesh(bad, prob.i, prob.j, prob.k, prob.U, **prob.params())
    assert e.value.code == 1
    badi = prob.i.copy()
    badi[0] = 4
    with pytest.raises(orc.OracleError) as e:
        orc.Mesh(prob.level, badi, prob.j, prob.k, prob.U, **prob.params())
    assert e.value.code == 1


def test_generator_meshes_are_graded(orc):
    """The input generators only emit meshes the oracle accepts."""
    for prob in (inputs.sod(4, 5), inputs.sedov(3, 6), inputs.random_mesh(2, 5, seed=9),
                 inputs.lognormal(4, 2, seed=7)):
        m = _mesh(orc, prob)
        assert sum(m.num_octs(l) for l in range(16)) == prob.n_oct
