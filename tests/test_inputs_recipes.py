"""The seeded workloads have the sizes and structure their recipes state
(oct, leaf-cell and cell-update counts of the benchmark meshes; level range
and mix of the batched ensemble; displacement and halo fraction of the
cosmological particle set).  Counts come from the generators' oct lists
alone: leaf cells of level l = 8 octs(l) - octs(l+1)."""
import numpy as np
import pytest

from paper_2607_20704_gb300 import inputs


def _counts(prob):
    c = np.bincount(prob.level, minlength=17)
    leaf = {l: int(8 * c[l] - c[l + 1]) for l in range(16) if c[l]}
    updates = sum(v * 2 ** (l - prob.levelmin) for l, v in leaf.items())
    return int(prob.level.shape[0]), sum(leaf.values()), updates


def test_sod_configuration():
    p = inputs.sod(6, 7)
    assert _counts(p) == (57344, 434176, 630784)
    assert int(np.count_nonzero(p.level == 6)) == 32 ** 3


def test_sedov_benchmark_mesh():
    p = inputs.sedov(7, 10)
    assert (p.levelmin, p.levelmax) == (7, 10)
    assert _counts(p) == (307720, 2416184, 3692312)
    assert int(np.count_nonzero(p.level == 7)) == 64 ** 3  # 128^3 base cells


def test_cosmology_shaped_mesh():
    p = inputs.lognormal(8, 4)
    n, leaf, _ = _counts(p)
    assert (n, leaf) == (2473160, 19409272)
    assert int(np.count_nonzero(p.level == 8)) == 128 ** 3  # 256^3 base cells
    assert p.level.max() == 11


def test_batched_ensemble():
    members = inputs.batched(512, seed=11)
    assert len(members) == 512
    tot = np.array([_counts(m) for m in members]).sum(axis=0)
    assert tuple(int(x) for x in tot) == (11288552, 85568344, 165944440)
    names = [m.name for m in members]
    assert sum(n == "sod" for n in names) + sum(n == "sedov" for n in names) == 512
    assert 200 <= sum(n == "sod" for n in names) <= 312  # 50/50 draws
    assert {m.levelmin for m in members} == {4, 5, 6}
    assert max(m.levelmax - m.levelmin for m in members) == 3


@pytest.mark.parametrize("n,rms", [(64, 1.0), (128, 0.73)])
def test_cosmological_particles(n, rms):
    """Displacements are scaled to an rms of one cell at the 64^3 points of the
    potential; on a finer lattice the linear interpolation between those
    points leaves a smaller rms (0.73 cells at 128^3, 0.75 at 512^3)."""
    ps = inputs.particles(n, "cosmo", seed=3)
    assert ps.np == n ** 3 and abs(ps.m.sum() - 1.0) < 1e-12
    # lattice point of particle t = (i n + j) n + k, i along x
    t = np.arange(ps.np)
    q = [((t // (n * n)) + 0.5) / n, (((t // n) % n) + 0.5) / n, ((t % n) + 0.5) / n]
    d = [(a - b + 0.5) % 1.0 - 0.5 for a, b in zip((ps.x, ps.y, ps.z), q)]
    r = np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2) * n  # displacement in cells
    halo = r > 5.0  # moved into a halo (the lattice displacements stay within a few cells)
    assert abs(halo.mean() - 0.25) < 0.01
    assert abs(np.sqrt(np.mean(r[~halo] ** 2)) - rms) < 0.03
