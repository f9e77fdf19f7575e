"""Batched handles: many independent meshes advanced by the same launches.
Each member must equal the same mesh in a handle of its own, bit for bit,
and match its FP64 oracle within the W-cycle tolerance."""
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


def _mixed(seed):
    """Members with different levelmin, depth, gamma and level ranges."""
    return [inputs.random_mesh(3, 5, seed=seed).shuffled(1),
            inputs.sedov(3, 5, radii={5: 0.1, 4: 0.2}),
            inputs.random_mesh(4, 4, seed=seed + 1),
            inputs.sod(3, 4),
            inputs.random_mesh(2, 5, seed=seed + 2, gamma=5.0 / 3.0),
            inputs.random_mesh(3, 6, seed=seed + 3)]


@pytest.mark.parametrize("precision", [8, 4])
def test_members_equal_the_same_mesh_alone(precision):
    from paper_2607_20704_gb300 import amr
    probs = _mixed(31)
    b = amr.Mesh.batch(probs, precision=precision)
    assert b.info()["n_members"] == len(probs)
    b.advance(3, sync=True)
    dts = b.member_dt()
    for q, pr in enumerate(probs):
        alone = amr.Mesh(*pr.mesh_args(), **pr.params(), precision=precision)
        dt = alone.advance(3, sync=True)
        assert dts[q] == dt, (q, dts[q], dt)
        b.select(q)
        for l in alone.levels():
            ka, Ua = alone.read(l)
            kb, Ub = b.read(l)
            assert np.array_equal(ka, kb)
            assert np.array_equal(Ua, Ub), (q, l)
        alone.close()


def test_members_match_their_oracles():
    import oracle
    from paper_2607_20704_gb300 import amr
    probs = _mixed(41)
    b = amr.Mesh.batch(probs)
    orcs = [oracle.Mesh(*pr.mesh_args(), **pr.params()) for pr in probs]
    for _ in range(2):
        b.advance(1, sync=True)
        for o in orcs:
            o.advance(1)
    for q, o in enumerate(orcs):
        b.select(q)
        compare_all(b, o, 1e-11)
        # index of each member against its own oracle, bit for bit
        for l in o.levels():
            nbg, spg = b.read_index(l)
            assert np.array_equal(nbg, o.read_nbr(l))
            assert np.array_equal(spg, o.read_split(l))
            assert np.array_equal(b.read_cache(l)[0], o.read_cache(l))


def test_member_level_steps_match():
    """amr_step_level advances the level of every member with one dt."""
    import oracle
    from paper_2607_20704_gb300 import amr
    probs = [inputs.random_mesh(3, 5, seed=51), inputs.random_mesh(3, 4, seed=52)]
    b = amr.Mesh.batch(probs)
    orcs = [oracle.Mesh(*pr.mesh_args(), **pr.params()) for pr in probs]
    dt = min(o.cfl_dt() for o in orcs) * 0.25
    for l in (5, 4, 3):
        b.step_level(l, dt)
        for o in orcs:
            if o.num_octs(l):
                o.step_level(l, dt)
    for q, o in enumerate(orcs):
        b.select(q)
        compare_all(b, o, 1e-11)


def test_ensemble_shape_and_lookup():
    """The seeded ensemble generator's meshes load as one batch; lookups
    resolve within the selected member only."""
    from paper_2607_20704_gb300 import amr
    probs = inputs.batched(24, seed=11, max_extra=2)
    b = amr.Mesh.batch(probs)
    inf = b.info()
    assert inf["n_members"] == 24
    assert inf["n_oct"] == sum(p.n_oct for p in probs)
    b.advance(2, sync=True)
    for q in (0, 7, 23):
        b.select(q)
        keys = np.concatenate([b.read(l)[0] for l in b.levels()])
        idx = b.lookup(keys)
        assert np.array_equal(idx, np.arange(len(keys)))


def test_tile_size_and_schedule_do_not_change_results():
    """The autotuner's choices (tile size, persistent or one-tile-per-block
    grids) and its snapshot/restore leave every result bit-identical."""
    from paper_2607_20704_gb300 import amr
    probs = _mixed(61)
    outs = []
    for tile, sched in ((64, 1), (128, 0), (512, 1), (0, -1)):
        b = amr.Mesh.batch(probs, tile=tile, schedule=sched)
        b.advance(2, sync=True)
        inf = b.info()
        if tile:
            assert (inf["tile"], inf["schedule"]) == (tile, sched)
        else:
            assert inf["tile"] in (64, 128, 256, 512) and inf["schedule"] in (0, 1)
        res = []
        for q in range(len(probs)):
            b.select(q)
            res += [b.read(l)[1] for l in b.levels()]
        outs.append(res)
        b.close()
    for other in outs[1:]:
        for a, c in zip(outs[0], other):
            assert np.array_equal(a, c)


@pytest.mark.parametrize("precision", [8, 4])
def test_repack_keeps_members_bit_for_bit(precision):
    """A batch repacked between coarse steps (one finished member dropped, a
    new mesh added): every member's state equals the same mesh advanced
    alone, bit for bit, and step counts carry over."""
    from paper_2607_20704_gb300 import amr
    kw = dict(precision=precision, tile=128, schedule=0)
    probs = [inputs.sod(3, 5), inputs.random_mesh(3, 5, seed=71), inputs.sedov(4, 5, radii={5: 0.15})]
    new = inputs.random_mesh(3, 4, seed=72)
    b = amr.Mesh.batch(probs, **kw)
    b.set_member_steps([5, 2, -1])
    b.advance(2, sync=True)
    b.repack([0, 2], [new], [3])
    assert b.n_members == 3
    b.advance(3, sync=True)
    for q, (pr, n) in enumerate([(probs[0], 5), (probs[2], 5), (new, 3)]):
        a = amr.Mesh(*pr.mesh_args(), **pr.params(), **kw)
        a.advance(n, sync=True)
        b.select(q)
        assert b.levels() == a.levels(), q
        for l in a.levels():
            ka, Ua = a.read(l)
            kb, Ub = b.read(l)
            assert np.array_equal(ka, kb) and np.array_equal(Ua, Ub), (q, l)
        a.close()
    # a repack that only drops members, then one that only adds
    b.repack([1])
    b.repack([0], [probs[1]], [-1])
    assert b.n_members == 2
    b.close()


def test_repack_rejects_bad_arguments_and_keeps_the_handle():
    from paper_2607_20704_gb300 import amr
    probs = [inputs.sod(3, 4), inputs.random_mesh(3, 4, seed=73)]
    b = amr.Mesh.batch(probs)
    before = [b.select(q).read(3)[1].copy() for q in range(2)]
    for keep in ([1, 0], [0, 0], [2], []):
        with pytest.raises(amr.AmrError) as e:
            b.repack(keep)
        assert e.value.status == amr.AMR_EINVAL
    bad = inputs.sod(3, 4)
    bad.level[0] = 7  # a level-7 oct in a levelmax-4 mesh
    with pytest.raises(amr.AmrError):
        b.repack([0], [bad], [1])
    for q in range(2):
        assert np.array_equal(b.select(q).read(3)[1], before[q])
    b.close()
