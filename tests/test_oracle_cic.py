"""Pins of the oracle's Cloud-in-Cell deposition (Sec. 4, mass deposition)
against what the definition of CIC fixes independently of its
floor-and-shift formulation: the overlap of a particle's cube-shaped cloud of
side dx with each cell (a hat function of the centre distance), closed forms
for particles at cell centres and faces, conservation of mass and of the
centre of mass, and the uniform density of a shifted lattice."""
import numpy as np
import pytest

import oracle
from paper_2607_20704_gb300 import inputs


def _hat_density(n, x, y, z, m):
    """CIC as the overlap of the particle's cloud (a cube of side dx centred
    on it) with every cell, on the periodic grid: per axis the overlap
    fraction is max(0, 1 - |distance between particle and cell centre| / dx),
    the distance taken to the nearest periodic image.  Dense brute force."""
    c = (np.arange(n) + 0.5) / n

    def hat(p):
        d = np.abs(p[:, None] - c[None, :])
        d = np.minimum(d, 1.0 - d)
        return np.maximum(0.0, 1.0 - d * n)
    hx, hy, hz = hat(x), hat(y), hat(z)
    rho = np.einsum("p,pi,pj,pk->ijk", m, hx, hy, hz)
    return rho * n ** 3


@pytest.mark.parametrize("n,np_,seed", [(2, 5, 1), (4, 37, 2), (8, 300, 3), (16, 1000, 4)])
def test_cic_equals_the_cloud_overlap(n, np_, seed):
    rng = np.random.default_rng(seed)
    x, y, z = rng.random(np_), rng.random(np_), rng.random(np_)
    m = np.exp(rng.standard_normal(np_))
    got = oracle.cic_deposit(n, x, y, z, m)
    ref = _hat_density(n, x, y, z, m)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * ref.max())


def test_particle_at_a_cell_centre_fills_that_cell_only():
    n = 8
    for (i, j, k) in [(0, 0, 0), (3, 5, 7), (7, 7, 7)]:
        x, y, z = (np.array([(a + 0.5) / n]) for a in (i, j, k))
        rho = oracle.cic_deposit(n, x, y, z, np.array([2.0]))
        want = np.zeros((n, n, n))
        want[i, j, k] = 2.0 * n ** 3
        assert np.array_equal(rho, want)


def test_particle_on_a_corner_splits_equally_over_eight_cells():
    n = 8
    rho = oracle.cic_deposit(n, np.array([3 / n]), np.array([0.0]), np.array([5 / n]),
                             np.array([1.0]))
    nz = np.argwhere(rho != 0)
    cells = {tuple(c) for c in nz}
    assert cells == {(a, b, c) for a in (2, 3) for b in (7, 0) for c in (4, 5)}
    assert np.all(rho[rho != 0] == n ** 3 / 8.0)


def test_mass_and_centre_of_mass_are_conserved():
    n = 32
    ps = inputs.particles(n, "uniform", seed=5, n_particles=5000, masses="random")
    rho = oracle.cic_deposit(*ps.args())
    dv = 1.0 / n ** 3
    assert abs(rho.sum() * dv - ps.m.sum()) <= 1e-13 * ps.m.sum()
    # centre of mass along x, for particles away from the periodic seam
    keep = (ps.x > 2 / n) & (ps.x < 1 - 2 / n)
    rho_k = oracle.cic_deposit(n, ps.x[keep], ps.y[keep], ps.z[keep], ps.m[keep])
    xc = (np.arange(n) + 0.5) / n
    com = np.einsum("ijk,i->", rho_k, xc) * dv
    assert abs(com - np.dot(ps.m[keep], ps.x[keep])) <= 1e-12 * ps.m[keep].sum()


def test_shifted_lattice_deposits_a_uniform_density():
    n = 16
    a = (np.arange(n) + 0.37) / n
    X, Y, Z = np.meshgrid(a, a, a, indexing="ij")
    x, y, z = X.ravel(), Y.ravel(), Z.ravel()
    rho = oracle.cic_deposit(n, x, y, z, np.full(x.shape, 1.0 / n ** 3))
    assert np.allclose(rho, 1.0, rtol=1e-14, atol=0)


def test_deposit_is_linear_and_order_free():
    n = 8
    ps = inputs.particles(n, "uniform", seed=6, n_particles=700, masses="random")
    rho = oracle.cic_deposit(*ps.args())
    perm = np.random.default_rng(0).permutation(ps.np)
    rho_p = oracle.cic_deposit(n, ps.x[perm], ps.y[perm], ps.z[perm], ps.m[perm])
    assert np.allclose(rho_p, rho, rtol=1e-13, atol=0)
    half = oracle.cic_deposit(n, ps.x, ps.y, ps.z, 0.5 * ps.m)
    assert np.array_equal(2.0 * half, rho)


def test_empty_set_and_bad_grid():
    e = np.zeros(0)
    assert np.array_equal(oracle.cic_deposit(4, e, e, e, e), np.zeros((4, 4, 4)))
    with pytest.raises(oracle.OracleError):
        oracle.cic_deposit(6, e, e, e, e)


def test_particle_generator_shapes():
    ps = inputs.particles(16, "cosmo", seed=1)
    assert ps.np == 16 ** 3
    for a in (ps.x, ps.y, ps.z):
        assert a.min() >= 0.0 and a.max() < 1.0
    assert abs(ps.m.sum() - 1.0) < 1e-12
    idx = (ps.x * 16).astype(int) + 16 * ((ps.y * 16).astype(int) + 16 * (ps.z * 16).astype(int))
    counts = np.bincount(idx, minlength=16 ** 3)
    assert counts.max() >= 30 and (counts == 0).mean() > 0.2  # halos and voids
