"""Poisson on the refined levels on the GPU (Sec. 5: the potential built level
by level, each level's boundary values from the level below) against the
oracle.

Given the same coarse potential, initial guess and density, the GPU's level
solve performs the oracle's floating-point operations in the oracle's order,
each rounded once (no contraction into fused multiply-adds on either side):
the red-black sweeps update cells of one colour from cells of the other, so
the order in which the threads run does not change any value.  The
potential must then be identical bit for bit.  The residual norms are sums
of n squares taken in another order: |sum - sum'| <= 2 (n - 1) u sum with
u = 2^-53, halved by the square root; the tests allow 2 n u.

For the chained solve (every level from the base up) each level is compared
on its own, given the GPU's potential of the level below: the only
difference to the oracle is then the mean density rho_bar, a sum of the
base cells in another order (relative difference <= 2 m u); it enters the
source as fourpiG rho_bar and moves the solution by at most the solution's
response to a constant source of that size, well below 1e-12 of max|phi|
on these meshes (the tests allow 1e-11)."""
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


def _same_state(o, g):
    """The GPU mesh's state (its FP32 values, restriction included, on an
    FP32 mesh) written into the oracle's, so that both see one density."""
    for l in o.levels():
        _, Ug = g.read(l)
        o.write(l, Ug)


def _meshes():
    return [inputs.sedov(3, 5, radii={4: 0.3, 5: 0.15}), inputs.random_mesh(3, 6, seed=91),
            inputs.sedov(4, 6, radii={5: 0.35, 6: 0.2})]


def _smooth(rng, n):
    return np.sin(np.linspace(0.0, 6.0, n) + rng.random()) + 0.1 * rng.standard_normal(n)


def _refined(o):
    return [l for l in o.levels() if l > o.levelmin and o.num_octs(l) > 0]


@pytest.mark.parametrize("precision", [8, 4])
def test_level_solve_is_bitwise_the_oracle(precision):
    import oracle
    from paper_2607_20704_gb300 import amr
    for t, prob in enumerate(_meshes()):
        o = oracle.Mesh(*prob.mesh_args(), **prob.params())
        g = amr.Mesh(*prob.mesh_args(), **prob.params(), precision=precision)
        if precision == 4:
            _same_state(o, g)
        rng = np.random.default_rng(40 + t)
        for L in _refined(o):
            phic = _smooth(rng, 8 * o.num_octs(L - 1))
            phi0 = 0.01 * rng.standard_normal(8 * o.num_octs(L))
            want, res_o = o.mg_level(L, phic, fourpiG=2.5, rho_bar=0.9, ncycles=3, phi0=phi0)
            g.write_phi(L - 1, phic)
            g.write_phi(L, phi0)
            res = g.poisson_level(L, fourpiG=2.5, rho_bar=0.9, n_vcycles=3)
            got = g.read_phi_level(L)
            assert np.array_equal(got, want), (prob.name, L, np.abs(got - want).max())
            n = want.size
            assert np.all(np.abs(res - res_o) <= 2 * n * U * res_o + 1e-300), (prob.name, L, res, res_o)
            # the coarse data are left as they were
            assert np.array_equal(g.read_phi_level(L - 1), phic)
        g.close()


def test_repeated_calls_continue_from_the_result():
    """A second call starts from the first one's result: two calls of 2
    cycles equal one of 4, also with a solve of another level (and so a
    rebuild of the tables) in between."""
    import oracle
    from paper_2607_20704_gb300 import amr
    prob = _meshes()[1]
    o = oracle.Mesh(*prob.mesh_args(), **prob.params())
    g = amr.Mesh(*prob.mesh_args(), **prob.params())
    levels = _refined(o)
    L = levels[-1]
    rng = np.random.default_rng(5)
    phic = _smooth(rng, 8 * o.num_octs(L - 1))
    want, _ = o.mg_level(L, phic, fourpiG=1.0, rho_bar=1.0, ncycles=4)
    for other in (None, *[l for l in levels if l not in (L, L - 1)][:1]):
        g.write_phi(L - 1, phic)
        g.write_phi(L, np.zeros(8 * o.num_octs(L)))
        g.poisson_level(L, 1.0, 1.0, 2)
        if other is not None:
            g.poisson_level(other, 1.0, 1.0, 1)
        g.poisson_level(L, 1.0, 1.0, 2)
        assert np.array_equal(g.read_phi_level(L), want), other
    g.close()


def test_residual_contracts_like_the_oracle():
    """Six V-cycles from a zero guess: the residual history is the oracle's
    (within the order bound of the norm) and falls by at least half per cycle
    on every level (the asymptotic factor on these nested balls is near 0.4,
    from 0.04 in the first cycle)."""
    import oracle
    from paper_2607_20704_gb300 import amr
    prob = _meshes()[2]
    o = oracle.Mesh(*prob.mesh_args(), **prob.params())
    g = amr.Mesh(*prob.mesh_args(), **prob.params())
    rng = np.random.default_rng(8)
    for L in _refined(o):
        phic = _smooth(rng, 8 * o.num_octs(L - 1))
        _, res_o = o.mg_level(L, phic, fourpiG=1.0, rho_bar=1.0, ncycles=6)
        g.write_phi(L - 1, phic)
        g.write_phi(L, np.zeros(8 * o.num_octs(L)))
        res = g.poisson_level(L, 1.0, 1.0, 6)
        n = 8 * o.num_octs(L)
        assert np.all(np.abs(res - res_o) <= 2 * n * U * res_o + 1e-300), (L, res, res_o)
        assert np.all(res[1:] < 0.5 * res[:-1]), (L, res)
    g.close()


def _father_guess(o, L, phic):
    """Every cell of level L takes its father cell's potential."""
    keys, _ = o.read(L)
    ckeys, _ = o.read(L - 1)
    ck = ckeys.astype(np.int64)
    where = {(int(a), int(b), int(c)): q for q, (a, b, c) in
             enumerate(zip((ck >> 40) & 0xFFFFF, (ck >> 20) & 0xFFFFF, ck & 0xFFFFF))}
    k = keys.astype(np.int64)
    out = np.zeros(8 * keys.size)
    for q, (i, j, l) in enumerate(zip((k >> 40) & 0xFFFFF, (k >> 20) & 0xFFFFF, k & 0xFFFFF)):
        f = where[(int(i) >> 1, int(j) >> 1, int(l) >> 1)]
        c = (int(i) & 1) + 2 * (int(j) & 1) + 4 * (int(l) & 1)
        out[8 * q:8 * q + 8] = phic[8 * f + c]
    return out


@pytest.mark.parametrize("t", [0, 1])
def test_all_levels_from_the_base_up(t):
    import oracle
    from paper_2607_20704_gb300 import amr
    prob = _meshes()[t]
    o = oracle.Mesh(*prob.mesh_args(), **prob.params())
    g = amr.Mesh(*prob.mesh_args(), **prob.params())
    res = g.poisson_levels(fourpiG=1.0, n_vcycles=4)
    base = g.read_phi_level(o.levelmin)
    assert np.array_equal(base, g.read_phi())
    _, Ub = o.read(o.levelmin)
    rho_bar = Ub[0].sum() / Ub[0].size
    phic = base
    for L in _refined(o):
        got = g.read_phi_level(L)
        want, res_o = o.mg_level(L, phic, fourpiG=1.0, rho_bar=rho_bar, ncycles=4,
                                 phi0=_father_guess(o, L, phic))
        scale = max(np.abs(want).max(), 1e-300)
        assert np.abs(got - want).max() <= 1e-11 * scale, (L, np.abs(got - want).max() / scale)
        assert np.allclose(res[L], res_o, rtol=1e-9, atol=1e-12 * res_o[0]), (L, res[L], res_o)
        phic = got
    g.close()


def test_batch_member_equals_the_mesh_alone():
    from paper_2607_20704_gb300 import amr
    probs = [inputs.sod(3, 4), _meshes()[0]]
    a = amr.Mesh(*probs[1].mesh_args(), **probs[1].params())
    a.poisson_levels(1.0, 3)
    b = amr.Mesh.batch(probs)
    b.select(1)
    b.poisson_levels(1.0, 3)
    for l in a.levels():
        assert np.array_equal(a.read_phi_level(l), b.read_phi_level(l)), l
    a.close()
    b.close()


def test_errors_and_regrid():
    from paper_2607_20704_gb300 import amr
    prob = _meshes()[1]
    g = amr.Mesh(*prob.mesh_args(), **prob.params())
    for bad in (lambda: g.poisson_level(g.levelmin), lambda: g.poisson_level(g.levelmax + 1),
                lambda: g.poisson_level(g.levelmin + 1, n_vcycles=-1),
                lambda: g.write_phi(g.levelmin, np.zeros(3))):
        with pytest.raises(amr.AmrError) as e:
            bad()
        assert e.value.status == amr.AMR_EINVAL
    with pytest.raises(amr.AmrError):
        g.read_phi_level(g.levelmin)  # no potential yet
    g.poisson_levels(1.0, 2)
    assert np.abs(g.read_phi_level(g.levelmax)).max() > 0
    before = g.read_phi_level(g.levelmin)
    created, removed = g.regrid()
    if created + removed:
        with pytest.raises(amr.AmrError):
            g.read_phi_level(g.levelmin)  # a new mesh discards the potential
    else:
        assert np.array_equal(g.read_phi_level(g.levelmin), before)
    g.close()
