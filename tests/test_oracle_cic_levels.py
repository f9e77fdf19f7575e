"""Pins of the oracle's Cloud-in-Cell deposition onto the AMR levels (Sec. 4:
at level l the particles of level l and of every finer level deposit, then
the list is split for level l+1).  Against what the definitions fix on their
own: on a single level it is the uniform-grid deposition; on each level of a
refined mesh the density of every existing cell equals the overlap of the
cubic clouds (side dx_l) of the level's particles with that cell, computed by
brute force; the level lists are the particles whose host cell at every
coarser level is split, found by brute force from the mesh's keys."""
import numpy as np

import oracle
from paper_2607_20704_gb300 import inputs


def _hat_at(cells, n, x, y, z, m):
    """CIC density at the given cells (i, j, k) of an n^3 periodic grid: the
    overlap of each particle's cloud (a cube of side 1/n) with the cell."""
    c = (np.asarray(cells, dtype=np.float64) + 0.5) / n  # [ncell, 3]

    def hat(p, cc):
        d = np.abs(p[:, None] - cc[None, :])
        d = np.minimum(d, 1.0 - d)
        return np.maximum(0.0, 1.0 - d * n)
    w = hat(x, c[:, 0]) * hat(y, c[:, 1]) * hat(z, c[:, 2])  # [np, ncell]
    return (m[:, None] * w).sum(axis=0) * n ** 3


def _cells_of(keys):
    k = keys.astype(np.int64)
    oi, oj, ok = (k >> 40) & 0xFFFFF, (k >> 20) & 0xFFFFF, k & 0xFFFFF
    c = np.arange(8)
    return np.stack([(2 * oi[:, None] + (c & 1)).ravel(), (2 * oj[:, None] + ((c >> 1) & 1)).ravel(),
                     (2 * ok[:, None] + ((c >> 2) & 1)).ravel()], axis=1)


def _particles(rng, n, lo=0.0, hi=1.0):
    x, y, z = (lo + (hi - lo) * rng.random(n) for _ in range(3))
    return x, y, z, np.exp(rng.standard_normal(n))


def test_single_level_equals_the_uniform_deposition():
    rng = np.random.default_rng(1)
    prob = inputs.uniform_grid(3, lambda x, y, z: (1 + 0 * x, 0 * x, 0 * x, 0 * x, 1 + 0 * x))
    o = oracle.Mesh(*prob.mesh_args(), **prob.params())
    x, y, z, m = _particles(rng, 500)
    rho, cnt = o.cic_deposit_levels(x, y, z, m)
    assert cnt[3] == 500 and cnt[4:].sum() == 0
    uni = oracle.cic_deposit(8, x, y, z, m)  # [i, j, k]
    keys, _ = o.read(3)
    cells = _cells_of(keys)
    assert np.array_equal(rho[3], uni[cells[:, 0], cells[:, 1], cells[:, 2]])


def test_each_level_is_the_cloud_overlap_of_its_particles():
    rng = np.random.default_rng(2)
    prob = inputs.sedov(3, 5, radii={4: 0.3, 5: 0.15})
    o = oracle.Mesh(*prob.mesh_args(), **prob.params())
    x, y, z, m = _particles(rng, 400, 0.2, 0.8)
    rho, cnt = o.cic_deposit_levels(x, y, z, m)
    # level lists by brute force: the host cell at every coarser level is split
    split = {}
    for l in o.levels():
        keys, _ = o.read(l)
        cells = _cells_of(keys)
        sp = o.read_split(l).ravel()
        split[l] = {tuple(c) for c, s in zip(cells, sp) if s}
    inlist = np.ones(x.size, bool)
    for l in o.levels():
        assert cnt[l] == inlist.sum(), (l, cnt[l], inlist.sum())
        n = 1 << l
        keys, _ = o.read(l)
        cells = _cells_of(keys)
        want = _hat_at(cells, n, x[inlist], y[inlist], z[inlist], m[inlist])
        got = rho[l]
        assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * want.max()), l
        host = np.stack([np.floor(a * n).astype(np.int64) for a in (x, y, z)], axis=1)
        inlist &= np.array([tuple(h) in split[l] for h in host])
    assert cnt[o.levels()[-1]] > 0  # particles reach the finest level


def test_a_particle_deep_inside_deposits_its_whole_mass_on_every_level():
    prob = inputs.sedov(3, 5, radii={4: 0.3, 5: 0.15})
    o = oracle.Mesh(*prob.mesh_args(), **prob.params())
    x, y, z, m = (np.array([0.51]), np.array([0.49]), np.array([0.503]), np.array([2.5]))
    rho, cnt = o.cic_deposit_levels(x, y, z, m)
    for l in o.levels():
        assert cnt[l] == 1
        total = rho[l].sum() * 2.0 ** (-3 * l)
        assert abs(total - 2.5) <= 1e-14 * 2.5, (l, total)
