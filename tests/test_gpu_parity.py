"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

Integer work (order, hash lookups, neighbour array, split flags, ghost
keys) must match bit for bit; FP64 states within the tolerance stated in
tests/parity.py."""
import numpy as np
import pytest

from paper_2607_20704_gb300 import inputs
from parity import close, compare_all, pair

pytestmark = pytest.mark.gpu

SEEDS = [1, 2, 3]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_20704_gb300 import amr, build
    build.build()
    amr.load()


def _random(seed, lmin=3, lmax=5, **kw):
    return inputs.random_mesh(lmin, lmax, seed=seed, **kw).shuffled(seed + 100)


@pytest.mark.parametrize("seed", SEEDS)
def test_index_matches_oracle_bit_for_bit(seed):
    prob = _random(seed, 3, 6)
    g, o = pair(prob)
    total = 0
    for l in range(prob.levelmin, prob.levelmax + 1):
        kg, _ = g.read(l)
        ko, _ = o.read(l)
        assert np.array_equal(kg, ko), f"order at level {l}"
        nbg, spg = g.read_index(l)
        assert np.array_equal(nbg, o.read_nbr(l)), f"neighbours at level {l}"
        assert np.array_equal(spg, o.read_split(l)), f"split flags at level {l}"
        ckg, _, first = g.read_cache(l)
        assert np.array_equal(ckg, o.read_cache(l)), f"ghost keys at level {l}"
        total += len(kg)
    assert total == prob.n_oct
    # hash_get on every key, plus absent keys (neighbours outside the mesh)
    allk = np.concatenate([o.read(l)[0] for l in o.levels()])
    rng = np.random.default_rng(seed)
    extra = []
    for _ in range(2000):
        l = int(rng.integers(1, prob.levelmax + 2))
        side = 1 << (l - 1)
        a, b, c = rng.integers(0, side, 3)
        extra.append((l << 60) | (int(a) << 40) | (int(b) << 20) | int(c))
    keys = np.concatenate([allk, np.array(extra, np.uint64)])
    got = g.lookup(keys)
    want = np.array([o.lookup(int(k)) for k in keys.tolist()])
    assert np.array_equal(got, want)


def test_caller_supplied_sort_keys_set_the_order():
    prob = _random(4, 3, 4)
    keys = np.arange(prob.n_oct, dtype=np.uint64)[::-1].copy()
    from paper_2607_20704_gb300 import amr
    g = amr.Mesh(*prob.mesh_args(), **prob.params(), hilbert_key=keys)
    for l in range(prob.levelmin, prob.levelmax + 1):
        kg, _ = g.read(l)
        sel = np.nonzero(prob.level == l)[0][::-1]
        expect = [(int(prob.level[t]) << 60) | (int(prob.i[t]) << 40) | (int(prob.j[t]) << 20) | int(prob.k[t]) for t in sel]
        assert kg.tolist() == expect


@pytest.mark.parametrize("seed", SEEDS)
def test_ghost_prolongation_matches(seed):
    prob = _random(seed, 3, 5)
    g, o = pair(prob)
    for l in range(prob.levelmin + 1, prob.levelmax + 1):
        g.fill_ghosts(l)
        _, Ug, _ = g.read_cache(l)
        close(Ug, o.ghost(l), 1e-14, f"ghosts level {l}")


@pytest.mark.parametrize("seed", SEEDS)
def test_cfl_dt_matches(seed):
    prob = _random(seed, 3, 5)
    g, o = pair(prob)
    assert abs(g.cfl_dt() - o.cfl_dt()) <= 1e-14 * o.cfl_dt()


@pytest.mark.parametrize("seed", SEEDS)
def test_each_level_step_matches(seed):
    prob = _random(seed, 3, 6)
    for l in range(prob.levelmin, prob.levelmax + 1):
        g, o = pair(prob)
        dt = o.cfl_dt() * 0.5 ** (l - prob.levelmin)
        g.step_level(l, dt)
        o.step_level(l, dt)
        compare_all(g, o, 1e-12)


@pytest.mark.parametrize("graphs,reindex", [(True, True), (False, False), (True, False)])
def test_w_cycle_matches(graphs, reindex):
    prob = _random(7, 3, 6)
    g, o = pair(prob, gpu_kw=dict(use_graphs=graphs, reindex_every_step=reindex))
    for _ in range(2):
        dtg = g.advance(1, sync=True)
        dto = o.advance(1)
        assert abs(dtg - dto) <= 1e-12 * dto
    compare_all(g, o, 1e-11)


@pytest.mark.parametrize("precision", [8, 4])
def test_reindex_only_on_change_equals_reindex_every_step(precision):
    """Skipping the per-step index rebuild on an unchanged mesh changes
    nothing: states and pending reflux equal the per-step rebuild bit for
    bit after several coarse steps, a batch too, with and without graphs."""
    from paper_2607_20704_gb300 import amr
    probs = [_random(12, 3, 6), inputs.sedov(4, 6, radii={5: 0.15, 6: 0.08})]
    for graphs in (True, False):
        outs = []
        for every in (True, False):
            g = amr.Mesh.batch(probs, precision=precision, use_graphs=graphs,
                               reindex_every_step=every, tile=128, schedule=0)
            g.advance(3, sync=True)
            o = []
            for q in range(len(probs)):
                g.select(q)
                o += [g.read(l)[1] for l in g.levels()] + [g.read_reflux(l) for l in g.levels()]
            outs.append(o)
            g.close()
        for a, b in zip(*outs):
            assert np.array_equal(a, b)


def test_runs_repeat_bit_for_bit():
    prob = _random(8, 3, 6)
    from paper_2607_20704_gb300 import amr
    outs = []
    for _ in range(2):
        g = amr.Mesh(*prob.mesh_args(), **prob.params())
        g.advance(3)
        outs.append([g.read(l)[1] for l in g.levels()] + [g.read_reflux(l) for l in g.levels()])
        g.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_uniform_moving_state_is_preserved():
    prob = inputs.uniform_state(3, 6, seed=9)
    from paper_2607_20704_gb300 import amr
    g = amr.Mesh(*prob.mesh_args(), **prob.params())
    ref = prob.U[:, 0].copy()
    g.advance(3, sync=True)
    for l in g.levels():
        _, U = g.read(l)
        assert np.max(np.abs(U - ref[:, None])) <= 1e-14 * np.abs(ref).max()


def test_conservation_on_the_gpu():
    prob = _random(11, 3, 6)
    from paper_2607_20704_gb300 import amr
    g = amr.Mesh(*prob.mesh_args(), **prob.params())

    def totals():
        t = np.zeros(5)
        for l in g.levels():
            _, U = g.read(l)
            _, sp = g.read_index(l)
            t += (U[:, sp == 0]).sum(axis=1) * 2.0 ** (-3 * l)
        return t
    t0 = totals()
    g.advance(3, sync=True)
    t1 = totals()
    sc = np.array([abs(t0[0])] * 4 + [abs(t0[4])])
    assert np.all(np.abs(t1 - t0) <= 1e-13 * sc)


def test_fp32_state_path_against_fp64_oracle():
    prob = _random(12, 3, 5)
    g, o = pair(prob, gpu_kw=dict(precision=4))
    for _ in range(2):
        dt = o.advance(1)
        g.advance(1, sync=True)
    for l in o.levels():
        _, Ug = g.read(l)
        _, Uo = o.read(l)
        l1 = np.abs(Ug - Uo).sum(axis=1) / np.maximum(np.abs(Uo).sum(axis=1), 1e-300)
        assert l1[0] < 2e-6 and l1[4] < 2e-6, l1


def test_write_read_roundtrip_and_restart():
    prob = _random(13, 3, 5)
    from paper_2607_20704_gb300 import amr
    g = amr.Mesh(*prob.mesh_args(), **prob.params())
    g.advance(1)
    saved = {l: g.read(l)[1] for l in g.levels()}
    g.advance(2)
    after = {l: g.read(l)[1] for l in g.levels()}
    h = amr.Mesh(*prob.mesh_args(), **prob.params())
    for l, U in saved.items():
        h.write(l, U)
    h.advance(2)
    for l in g.levels():
        assert np.array_equal(h.read(l)[1], after[l])


def test_single_oct_and_single_level_meshes():
    import oracle
    from paper_2607_20704_gb300 import amr
    for lev in (1, 3):
        prob = inputs.uniform_grid(lev, lambda x, y, z: (1 + 0.2 * np.sin(2 * np.pi * x), 0.3 + 0 * x,
                                                         0 * x, 0 * x, 1 + 0.1 * np.cos(2 * np.pi * y)))
        g = amr.Mesh(*prob.mesh_args(), **prob.params())
        o = oracle.Mesh(*prob.mesh_args(), **prob.params())
        g.advance(2, sync=True)
        o.advance(2)
        compare_all(g, o, 1e-12)


def _expect_status(code, fn):
    from paper_2607_20704_gb300 import amr
    with pytest.raises(amr.AmrError) as e:
        fn()
    assert e.value.status == code, str(e.value)


def test_error_statuses():
    from paper_2607_20704_gb300 import amr
    prob = inputs.random_mesh(2, 3, seed=1)
    # duplicate oct
    lv = np.concatenate([prob.level, prob.level[-1:]])
    i, j, k = (np.concatenate([a, a[-1:]]) for a in (prob.i, prob.j, prob.k))
    U = np.concatenate([prob.U, prob.U[:, -8:]], axis=1)
    _expect_status(amr.AMR_EDUP, lambda: amr.Mesh(lv, i, j, k, U, **prob.params()))
    # grading violation: a level-4 oct far from any level-3 oct
    base = inputs.uniform_grid(2, lambda x, y, z: (1 + 0 * x, 0 * x, 0 * x, 0 * x, 1 + 0 * x))
    lv = np.concatenate([base.level, [3, 4]]).astype(np.uint8)
    i = np.concatenate([base.i, [0, 0]]).astype(np.uint32)
    j = np.concatenate([base.j, [0, 0]]).astype(np.uint32)
    k = np.concatenate([base.k, [0, 0]]).astype(np.uint32)
    U = np.concatenate([base.U, np.ones((5, 16))], axis=1)
    _expect_status(amr.AMR_EGRADING, lambda: amr.Mesh(lv, i, j, k, U, levelmin=2, levelmax=4, gamma=1.4))
    # incomplete base level
    _expect_status(amr.AMR_EGRADING, lambda: amr.Mesh(base.level[1:], base.i[1:], base.j[1:], base.k[1:],
                                                      base.U[:, 8:], **base.params()))
    # coordinate out of range
    bi = base.i.copy()
    bi[0] = 9
    _expect_status(amr.AMR_EINVAL, lambda: amr.Mesh(base.level, bi, base.j, base.k, base.U, **base.params()))
    # HBM budget
    _expect_status(amr.AMR_ENOMEM, lambda: amr.Mesh(*prob.mesh_args(), **prob.params(), hbm_budget_bytes=4096))
    # bad level / dt on a live mesh
    g = amr.Mesh(*prob.mesh_args(), **prob.params())
    _expect_status(amr.AMR_EINVAL, lambda: g.step_level(9, 0.1))
    _expect_status(amr.AMR_EINVAL, lambda: g.step_level(2, -1.0))
    # non-finite state is reported by the time-step reduction
    U = prob.U.copy()
    leaf = int(np.nonzero(prob.level == prob.level.max())[0][-1])
    U[0, 8 * leaf + 3] = np.nan
    h = amr.Mesh(prob.level, prob.i, prob.j, prob.k, U, **prob.params())
    _expect_status(amr.AMR_ENAN, lambda: h.cfl_dt())


def test_level_steps_in_sequence_match():
    """Chained steps of different levels on one mesh (pending reflux,
    restricted fathers and scratch reuse carry over between calls)."""
    prob = _random(14, 3, 6)
    g, o = pair(prob)
    dt = o.cfl_dt()
    order = [6, 6, 5, 6, 6, 5, 4, 3]
    for l in order:
        dl = dt * 0.5 ** (l - 3)
        g.step_level(l, dl)
        o.step_level(l, dl)
    compare_all(g, o, 1e-11)


@pytest.mark.parametrize("cfg", ["sod", "sedov"])
def test_full_size_coarse_step(cfg):
    """Full-size Sod (32^3 base octs + refined slab) and Sedov (levels 7-10,
    about 2.4 M leaf cells): one coarse W-cycle step, every cell compared."""
    prob = inputs.sod() if cfg == "sod" else inputs.sedov()
    g, o = pair(prob)
    dtg = g.advance(1, sync=True)
    dto = o.advance(1)
    assert abs(dtg - dto) <= 1e-13 * dto
    compare_all(g, o, 1e-11)


def test_full_size_lognormal_sampled_level_steps():
    """Cosmology-shaped mesh (256^3 base cells plus clustered refinement):
    one step of the finest and of the base level, compared on 3000 sampled
    octs per level (the oracle computes those octs one by one)."""
    import oracle
    from paper_2607_20704_gb300 import amr
    prob = inputs.lognormal()
    o = oracle.Mesh(*prob.mesh_args(), **prob.params())
    levels = o.levels()
    rng = np.random.default_rng(0)
    dt0 = o.cfl_dt()
    for l in (levels[-1], levels[0]):
        g = amr.Mesh(*prob.mesh_args(), **prob.params())
        dt = dt0 * 0.5 ** (l - prob.levelmin)
        n = o.num_octs(l)
        pick = np.sort(rng.choice(n, size=min(3000, n), replace=False))
        want = o.step_sample(l, dt, o.level_offset(l) + pick)
        g.step_level(l, dt)
        _, Ug = g.read(l)
        cells = (8 * pick[:, None] + np.arange(8)[None, :]).ravel()
        close(Ug[:, cells], want, 1e-12, f"lognormal level {l}")
        g.close()


@pytest.mark.parametrize("cfg", ["random", "sod", "sedov"])
def test_fp32_l1_error_per_config(cfg):
    """FP32 state path against the FP64 oracle, one coarse W-cycle step:
    L1 relative error of rho and E per level (reported with -s)."""
    import oracle
    from paper_2607_20704_gb300 import amr
    prob = {"random": lambda: _random(21, 3, 6), "sod": inputs.sod, "sedov": inputs.sedov}[cfg]()
    g = amr.Mesh(*prob.mesh_args(), **prob.params(), precision=4)
    o = oracle.Mesh(*prob.mesh_args(), **prob.params())
    o.advance(1)
    g.advance(1, sync=True)
    worst = 0.0
    for l in o.levels():
        _, Ug = g.read(l)
        _, Uo = o.read(l)
        l1 = np.abs(Ug - Uo).sum(axis=1) / np.maximum(np.abs(Uo).sum(axis=1), 1e-300)
        print(f"FP32 L1 {cfg} level {l}: rho {l1[0]:.2e} E {l1[4]:.2e}")
        worst = max(worst, l1[0], l1[4])
    assert worst < 5e-6, worst


def test_fp32_runs_repeat_bit_for_bit():
    prob = _random(22, 3, 6)
    from paper_2607_20704_gb300 import amr
    outs = []
    for _ in range(2):
        g = amr.Mesh(*prob.mesh_args(), **prob.params(), precision=4)
        g.advance(3)
        outs.append([g.read(l)[1] for l in g.levels()])
        g.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def _deepest():
    # levels 2..15 (the deepest a handle holds: 4-bit level, 14-bit
    # coordinates), 27 octs per level around an off-centre point
    return inputs.sedov(2, 15, radii={l: 3 * 2.0 ** -l for l in range(3, 16)}, centre=(0.3, 0.7, 0.55))


def test_deepest_hierarchy_index_and_level_steps():
    prob = _deepest()
    assert prob.levelmax == 15
    g, o = pair(prob)
    for l in range(prob.levelmin, prob.levelmax + 1):
        kg, _ = g.read(l)
        assert np.array_equal(kg, o.read(l)[0]), f"order at level {l}"
        nbg, spg = g.read_index(l)
        assert np.array_equal(nbg, o.read_nbr(l)), f"neighbours at level {l}"
        assert np.array_equal(spg, o.read_split(l)), f"split flags at level {l}"
        assert np.array_equal(g.read_cache(l)[0], o.read_cache(l)), f"ghost keys at level {l}"
    allk = np.concatenate([o.read(l)[0] for l in o.levels()])
    rng = np.random.default_rng(15)
    extra = []
    for _ in range(2000):
        l = int(rng.integers(1, 16))
        a, b, c = rng.integers(0, 1 << (l - 1), 3)
        extra.append((l << 60) | (int(a) << 40) | (int(b) << 20) | int(c))
    keys = np.concatenate([allk, np.array(extra, np.uint64)])
    assert np.array_equal(g.lookup(keys), np.array([o.lookup(int(k)) for k in keys.tolist()]))
    for l in range(prob.levelmin, prob.levelmax + 1):
        g, o = pair(prob)
        dt = o.cfl_dt() * 0.5 ** (l - prob.levelmin)
        g.step_level(l, dt)
        o.step_level(l, dt)
        compare_all(g, o, 1e-12)


@pytest.mark.parametrize("graphs", [True, False])
def test_deepest_hierarchy_w_cycle(graphs):
    """One coarse step of the 14-level hierarchy: 16,383 level steps."""
    prob = _deepest()
    g, o = pair(prob, gpu_kw=dict(use_graphs=graphs, tile=128, schedule=0, nsubgrid=0))
    dtg = g.advance(1, sync=True)
    dto = o.advance(1)
    assert abs(dtg - dto) <= 1e-12 * dto
    compare_all(g, o, 1e-11)
