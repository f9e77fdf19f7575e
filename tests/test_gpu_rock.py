"""The fused shared-memory level steps (the paper's rock kernel, Sec. 3, and
its planar "paper" kernel, each with nsubgrid 1, 2 and 4) against the per-cell passes: states, pending reflux and
ghost values equal bit for bit in FP64 and FP32, for single level steps,
W-cycles, batches and regrids, also with caller-given sort keys that split
the aligned oct groups into several blocks; and against the oracle."""
import numpy as np
import pytest

from paper_2607_20704_gb300 import inputs
from parity import compare_all, pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_20704_gb300 import amr, build
    build.build()
    amr.load()


def _state(m):
    out = []
    for l in m.levels():
        out.append(m.read(l)[1])
        out.append(m.read_reflux(l))
    return out


def _same(a, b, what):
    sa, sb = _state(a), _state(b)
    assert len(sa) == len(sb), what
    for t, (x, y) in enumerate(zip(sa, sb)):
        assert np.array_equal(x, y), (what, t, float(np.nanmax(np.abs(x - y))) if x.size else 0.0)


def _problems():
    return [inputs.random_mesh(3, 6, seed=41), inputs.sedov(4, 6, radii={5: 0.15, 6: 0.08}),
            inputs.sod(4, 6), inputs.random_mesh(4, 6, seed=42).shuffled(5)]


def _mesh(prob, **kw):
    from paper_2607_20704_gb300 import amr
    return amr.Mesh(*prob.mesh_args(), **prob.params(), **kw)


@pytest.mark.parametrize("precision,ns,planar", [(8, 1, 0), (8, 2, 0), (8, 4, 0), (4, 1, 0), (4, 2, 0), (4, 4, 0),
                                                (8, 1, 1), (8, 2, 1), (8, 4, 1), (4, 2, 1), (4, 4, 1)])
def test_level_steps_equal_the_per_cell_passes(ns, planar, precision):
    for prob in _problems():
        for l in range(prob.levelmin, prob.levelmax + 1):
            ref = _mesh(prob, precision=precision, nsubgrid=0, tile=128, schedule=0)
            rk = _mesh(prob, precision=precision, nsubgrid=ns, planar=planar, tile=128, schedule=0)
            assert rk.info()["nsubgrid"] == ns and ref.info()["nsubgrid"] == 0
            assert rk.info()["planar"] == planar
            dt = ref.cfl_dt() * 0.5 ** (l - prob.levelmin)
            ref.step_level(l, dt)
            rk.step_level(l, dt)
            _same(ref, rk, (prob.name, l, ns, planar, precision))
            ref.close()
            rk.close()


@pytest.mark.parametrize("precision,ns,schedule,planar", [
    (8, 1, 0, 0), (8, 2, 1, 0), (8, 2, 0, 0), (8, 4, 1, 0), (4, 1, 0, 0), (4, 2, 1, 0), (4, 4, 1, 0),
    (4, 4, 0, 0),
    (8, 1, 1, 1), (8, 2, 0, 1), (8, 4, 1, 1), (4, 2, 1, 1), (4, 4, 0, 1)])
def test_w_cycles_equal_the_per_cell_passes(ns, schedule, planar, precision):
    for prob in _problems()[:3]:
        ref = _mesh(prob, precision=precision, nsubgrid=0, tile=128, schedule=schedule)
        rk = _mesh(prob, precision=precision, nsubgrid=ns, planar=planar, tile=128, schedule=schedule)
        ref.advance(3, sync=True)
        rk.advance(3, sync=True)
        _same(ref, rk, (prob.name, ns, schedule, planar, precision))
        ref.close()
        rk.close()


@pytest.mark.parametrize("ns,precision,planar", [(1, 8, 0), (2, 8, 0), (4, 4, 0), (4, 8, 0), (2, 8, 1),
                                                 (4, 8, 1)])
def test_split_oct_groups_with_caller_keys(ns, precision, planar):
    """Random sort keys scatter each aligned oct group over several runs, so
    one group forms several blocks; each updates only its own octs."""
    prob = inputs.random_mesh(3, 6, seed=43)
    keys = np.random.default_rng(3).permutation(prob.n_oct).astype(np.uint64)
    ref = _mesh(prob, nsubgrid=0, tile=128, schedule=0, hilbert_key=keys, precision=precision)
    rk = _mesh(prob, nsubgrid=ns, planar=planar, tile=128, schedule=0, hilbert_key=keys, precision=precision)
    ref.advance(2, sync=True)
    rk.advance(2, sync=True)
    _same(ref, rk, ("caller keys", ns))


@pytest.mark.parametrize("ns,planar", [(1, 0), (2, 0), (4, 0), (2, 1)])
def test_batched_and_regridded_meshes(ns, planar):
    from paper_2607_20704_gb300 import amr
    probs = [inputs.sod(3, 5), inputs.random_mesh(3, 5, seed=44), inputs.sedov(4, 5, radii={5: 0.15})]
    out = []
    for nsub in (0, ns):
        b = amr.Mesh.batch(probs, nsubgrid=nsub, planar=planar if nsub else -1, tile=128, schedule=0,
                           refine_grad_rho=0.1, refine_grad_p=0.1)
        b.advance(1)
        b.regrid()
        b.advance(2, sync=True)
        assert b.info()["nsubgrid"] == nsub
        out.append(b)
    for q in range(len(probs)):
        out[0].select(q)
        out[1].select(q)
        _same(out[0], out[1], ("batch member", q, ns))
    for b in out:
        b.close()


@pytest.mark.parametrize("ns,planar", [(1, 0), (2, 0), (4, 0), (2, 1), (4, 1)])
def test_fused_kernel_matches_the_oracle(ns, planar):
    prob = inputs.random_mesh(3, 6, seed=45)
    g, o = pair(prob, gpu_kw=dict(nsubgrid=ns, planar=planar, tile=128, schedule=1))
    for _ in range(2):
        dtg = g.advance(1, sync=True)
        dto = o.advance(1)
        assert abs(dtg - dto) <= 1e-12 * dto
    compare_all(g, o, 1e-11)


@pytest.mark.parametrize("precision", [8, 4])
def test_autotuner_choice_is_reported_and_exact(precision):
    prob = inputs.sedov(4, 6, radii={5: 0.15, 6: 0.08})
    auto = _mesh(prob, precision=precision)
    ref = _mesh(prob, nsubgrid=0, tile=128, schedule=0, precision=precision)
    auto.advance(2, sync=True)
    ref.advance(2, sync=True)
    assert auto.info()["nsubgrid"] in (0, 1, 2, 4) and auto.info()["planar"] in (0, 1)
    _same(ref, auto, "autotuned")


def test_bad_nsubgrid_is_refused():
    from paper_2607_20704_gb300 import amr
    prob = inputs.sod(3, 4)
    for bad, prec, planar in ((3, 8, -1), (-2, 8, -1), (8, 4, -1), (2, 8, 2)):
        with pytest.raises(amr.AmrError) as e:
            _mesh(prob, nsubgrid=bad, precision=prec, planar=planar)
        assert e.value.status == amr.AMR_EINVAL
    for prec in (8, 4):  # a fixed nsubgrid stages the cube unless planar is asked for
        m = _mesh(prob, nsubgrid=4, precision=prec)
        assert m.info()["planar"] == 0
        m.close()


@pytest.mark.parametrize("precision", [8, 4])
def test_levels_narrower_than_the_block(precision):
    """Levels of 1, 2 and 4 octs per side with nsubgrid up to 4: the block
    meets its own octs again across the periodic wrap; results equal the
    per-cell passes bit for bit."""
    rng = np.random.default_rng(7)
    for lev in (1, 2, 3):
        def fn(x, y, z):
            return (1.0 + 0.5 * rng.random(x.shape), rng.standard_normal(x.shape),
                    rng.standard_normal(x.shape), rng.standard_normal(x.shape),
                    0.5 + rng.random(x.shape))
        prob = inputs.uniform_grid(lev, fn)
        for ns in (1, 2, 4):
            ref = _mesh(prob, precision=precision, nsubgrid=0, tile=128, schedule=0)
            rk = _mesh(prob, precision=precision, nsubgrid=ns, planar=0, tile=128, schedule=0)
            ref.advance(2, sync=True)
            rk.advance(2, sync=True)
            _same(ref, rk, ("narrow level", lev, ns, precision))
            ref.close()
            rk.close()
