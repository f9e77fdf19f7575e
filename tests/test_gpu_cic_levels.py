"""CIC deposition onto the AMR levels on the GPU (Sec. 4) against the oracle:
the size of every level's particle list exactly, and every cell's density.

Bound (FP64): both sides form each contribution as m ((wx wy) wz) 2^(3l)
with the same operations, so the terms agree bit for bit and the sums differ
only in order; a sum of K non-negative terms has a rounding error of at most
(K - 1) u of its value in any order (u = 2^-53), so |gpu - oracle| <= 2 K u
rho with K at most the level's list size.  FP32: positions are given as
FP32 values (exact in both), the GPU's weights and products round at 2^-24;
the relative L1 error of each level is held below 1e-5."""
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


def _particles(seed, n, lo=0.0, hi=1.0, f32=False):
    rng = np.random.default_rng(seed)
    x, y, z = (lo + (hi - lo) * rng.random(n) for _ in range(3))
    m = np.exp(rng.standard_normal(n))
    if f32:
        x, y, z, m = (a.astype(np.float32).astype(np.float64) for a in (x, y, z, m))
        x, y, z = (np.minimum(a, np.nextafter(np.float32(1), np.float32(0))) for a in (x, y, z))
    return x, y, z, m


def _meshes():
    return [inputs.sedov(3, 5, radii={4: 0.3, 5: 0.15}), inputs.random_mesh(3, 6, seed=81),
            inputs.sod(3, 5)]


@pytest.mark.parametrize("precision", [8, 4])
def test_levels_match_the_oracle(precision):
    import oracle
    from paper_2607_20704_gb300 import amr
    for t, prob in enumerate(_meshes()):
        x, y, z, m = _particles(10 + t, 3000, 0.05, 0.95, f32=precision == 4)
        o = oracle.Mesh(*prob.mesh_args(), **prob.params())
        want, cnt_o = o.cic_deposit_levels(x, y, z, m)
        g = amr.Mesh(*prob.mesh_args(), **prob.params(), precision=precision)
        cnt = g.cic_deposit_levels(x, y, z, m)
        assert np.array_equal(cnt, cnt_o), (prob.name, cnt, cnt_o)
        for l in o.levels():
            got = g.particle_rho(l)
            ref = want[l]
            if precision == 8:
                assert np.all(np.abs(got - ref) <= 2 * cnt_o[l] * U * np.abs(ref) + 1e-300), (prob.name, l)
            else:
                l1 = np.abs(got - ref).sum() / max(np.abs(ref).sum(), 1e-300)
                assert l1 < 1e-5, (prob.name, l, l1)
        g.close()


def test_device_arrays_and_repeat_calls():
    """The device-array entry point gives the host one's result (within the
    order bound), twice in a row on the same buffers; an empty set gives
    zeros."""
    import torch
    from paper_2607_20704_gb300 import amr
    prob = _meshes()[0]
    x, y, z, m = _particles(21, 5000)
    g = amr.Mesh(*prob.mesh_args(), **prob.params())
    cnt = g.cic_deposit_levels(x, y, z, m)
    ref = {l: g.particle_rho(l) for l in g.levels()}
    dev = [torch.from_numpy(a).cuda() for a in (x, y, z, m)]
    for _ in range(2):
        c2 = g.cic_deposit_levels_device(*dev)
        assert np.array_equal(c2, cnt)
        for l in g.levels():
            got = g.particle_rho(l)
            assert np.all(np.abs(got - ref[l]) <= 2 * cnt[l] * U * np.abs(ref[l]) + 1e-300), l
    e = np.zeros(0)
    c0 = g.cic_deposit_levels(e, e, e, e)
    assert c0.sum() == 0
    for l in g.levels():
        assert not g.particle_rho(l).any()
    g.close()


def test_batch_member_equals_the_mesh_alone():
    from paper_2607_20704_gb300 import amr
    probs = [inputs.sod(3, 4), inputs.sedov(3, 5, radii={4: 0.3, 5: 0.15})]
    x, y, z, m = _particles(31, 2000, 0.1, 0.9)
    a = amr.Mesh(*probs[1].mesh_args(), **probs[1].params())
    ca = a.cic_deposit_levels(x, y, z, m)
    b = amr.Mesh.batch(probs)
    b.select(1)
    cb = b.cic_deposit_levels(x, y, z, m)
    assert np.array_equal(ca, cb)
    for l in a.levels():
        ra, rb = a.particle_rho(l), b.particle_rho(l)
        assert np.all(np.abs(ra - rb) <= 2 * ca[l] * U * np.abs(ra) + 1e-300), l
    a.close()
    b.close()


def test_bad_particles_are_refused_on_the_host():
    from paper_2607_20704_gb300 import amr
    prob = inputs.sod(3, 4)
    g = amr.Mesh(*prob.mesh_args(), **prob.params())
    ok = np.array([0.25, 0.5])
    for bad in (np.array([0.25, 1.0]), np.array([-0.1, 0.5]), np.array([0.25, np.nan])):
        with pytest.raises(amr.AmrError) as e:
            g.cic_deposit_levels(bad, ok, ok, np.ones(2))
        assert e.value.status == amr.AMR_EINVAL
    with pytest.raises(amr.AmrError):
        g.particle_rho(3) if False else g.cic_deposit_levels(ok, ok, ok, np.array([1.0, np.inf]))
    g.close()
