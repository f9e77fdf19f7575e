"""Cloud-in-Cell deposition on the GPU (Sec. 4) against the oracle: the
atomic (warp-combining) and the deterministic segment algorithm in FP64 and
FP32, the source-cell Hilbert sort, reproducibility, edge cases, and the
full-size cosmological configuration on sampled cells.

Tolerances.  Both sides form the same weights (exactly), but the oracle
multiplies a contribution as m ((wx wy) wz) and the GPU as ((m wx) wy) wz:
each is three roundings from the exact product, so within (1 + u)^3 - 1 of
it (u = 2^-53), and the two differ by at most 6.001 u of the term.  Over the
K non-negative terms that reach a cell these differences sum to at most
6.001 u rho.  Then the sums differ in order: a sum of K non-negative terms
has a rounding error of at most (K - 1) u times its value in any order, so
the two sums are at most 2 (K - 1) u rho apart beyond the terms' own
difference.  Hence |gpu - oracle| <= (2 K + 8) u rho per cell (the 8 covers
6.001 u and the second-order terms), K the number of particles whose
stencil touches the cell; the final scaling by 1/dx^3 is exact.  FP32 adds
the rounding of the positions (x n - 1/2 moves by at most n 2^-24, each
weight by at most (n + 1) 2^-24), of the masses and of the products, and
sums in FP32: |gpu - oracle| <= (6 n + 12 + K) 2^-24 M per cell, M the sum
of m n^3 over the particles whose stencil may reach the cell after rounding
(and K their number)."""
import numpy as np
import pytest

from paper_2607_20704_gb300 import inputs

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
U32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_20704_gb300 import amr, build
    build.build()
    amr.load()


def _touch_counts(n, x, y, z):
    """K per cell: particles whose 2^3 stencil covers it (test-side count)."""
    i0 = [np.floor(a * n - 0.5).astype(np.int64) for a in (x, y, z)]
    K = np.zeros(n ** 3, np.int64)
    for c in range(8):
        ii = (i0[0] + (c & 1)) % n
        jj = (i0[1] + ((c >> 1) & 1)) % n
        kk = (i0[2] + (c >> 2)) % n
        np.add.at(K, ii + n * (jj + n * kk), 1)
    return K.reshape((n, n, n), order="F")


def _fp32_reach(n, x, y, z, m):
    """K and the mass sum M = sum of m n^3 per cell over the particles whose
    stencil may cover it once the positions are rounded to FP32 (the stencil
    start floor(x n - 1/2) moves by at most one cell when x n - 1/2 lies
    within n 2^-23 of an integer)."""
    d = n * 2.0 ** -23
    lo = [np.floor(a * n - 0.5 - d).astype(np.int64) for a in (x, y, z)]
    hi = [np.floor(a * n - 0.5 + d).astype(np.int64) + 1 for a in (x, y, z)]
    K = np.zeros(n ** 3, np.int64)
    M = np.zeros(n ** 3)
    for ox in range(3):
        for oy in range(3):
            for oz in range(3):
                ok = (lo[0] + ox <= hi[0]) & (lo[1] + oy <= hi[1]) & (lo[2] + oz <= hi[2])
                idx = ((lo[0] + ox) % n) + n * (((lo[1] + oy) % n) + n * ((lo[2] + oz) % n))
                np.add.at(K, idx[ok], 1)
                np.add.at(M, idx[ok], m[ok] * float(n) ** 3)
    return K.reshape((n, n, n), order="F"), M.reshape((n, n, n), order="F")


def _bound(n, x, y, z, m, ref, precision):
    if precision == 8:
        return (2 * _touch_counts(n, x, y, z) + 8) * U64 * ref
    K, M = _fp32_reach(n, x, y, z, m)
    return (6 * n + 12 + K) * U32 * M


def _assert_close(got, ref, bound, what):
    bad = np.abs(got - ref) > bound + 1e-300
    assert not bad.any(), (what, int(bad.sum()), float(np.abs(got - ref)[bad].max()),
                           np.argwhere(bad)[:3].tolist())


def _sets():
    return [inputs.particles(8, "uniform", seed=1, n_particles=1000, masses="random"),
            inputs.particles(16, "cosmo", seed=2),
            inputs.particles(32, "cosmo", seed=3, masses="random"),
            inputs.particles(32, "uniform", seed=4, n_particles=12345),
            inputs.particles(64, "clump", seed=5, n_particles=20000),
            inputs.particles(2, "uniform", seed=6, n_particles=77, masses="random")]


@pytest.mark.parametrize("precision", [8, 4])
@pytest.mark.parametrize("algo", ["atomic", "segment"])
def test_deposit_matches_the_oracle(algo, precision):
    import oracle
    from paper_2607_20704_gb300 import amr
    for ps in _sets():
        ref = oracle.cic_deposit(*ps.args())
        bound = _bound(*ps.args(), ref, precision)
        p = amr.Particles(*ps.args(), precision=precision)
        p.sort()
        p.deposit(algo)
        _assert_close(p.rho(), ref, bound, (ps.name, ps.n, algo))
        p.close()


@pytest.mark.parametrize("precision", [8, 4])
def test_atomic_deposit_needs_no_sort(precision):
    import oracle
    from paper_2607_20704_gb300 import amr
    ps = inputs.particles(32, "cosmo", seed=7)
    p = amr.Particles(*ps.args(), precision=precision)
    p.deposit("atomic")
    ref = oracle.cic_deposit(*ps.args())
    _assert_close(p.rho(), ref, _bound(*ps.args(), ref, precision), "unsorted")
    p.close()


def test_sort_orders_by_source_cell_hilbert_key_stably():
    import oracle
    from paper_2607_20704_gb300 import amr
    for ps in (inputs.particles(32, "cosmo", seed=8), inputs.particles(4, "uniform", seed=9, n_particles=3000)):
        n, bits = ps.n, ps.n.bit_length() - 1
        p = amr.Particles(*ps.args())
        p.sort()
        x, y, z, m, ids = p.read()
        assert np.array_equal(np.sort(ids), np.arange(ps.np))
        assert np.array_equal(x, ps.x[ids]) and np.array_equal(m, ps.m[ids])
        src = [np.floor(a * n - 0.5).astype(np.int64) % n for a in (x, y, z)]
        keys = np.array([oracle.hilbert3(int(a), int(b), int(c), bits)
                         for a, b, c in zip(*src)], dtype=np.uint64)
        assert np.all(keys[1:] >= keys[:-1])
        same = keys[1:] == keys[:-1]
        assert np.all(ids[1:][same] > ids[:-1][same])  # stable: input order kept within a cell
        # a second sort of a sorted set keeps it
        p.sort()
        assert np.array_equal(p.read()[4], ids)
        p.close()


@pytest.mark.parametrize("precision", [8, 4])
def test_segment_deposit_is_bit_reproducible(precision):
    from paper_2607_20704_gb300 import amr
    ps = inputs.particles(64, "cosmo", seed=10)
    out = []
    for _ in range(2):
        p = amr.Particles(*ps.args(), precision=precision)
        p.sort()
        p.deposit("segment")
        r1 = p.rho()
        p.deposit("atomic")
        p.deposit("segment")
        out += [r1, p.rho()]
        p.close()
    for r in out[1:]:
        assert np.array_equal(r, out[0])


def test_segment_deposit_needs_a_sort_after_each_write():
    from paper_2607_20704_gb300 import amr
    ps = inputs.particles(8, "uniform", seed=11, n_particles=100)
    p = amr.Particles(*ps.args())
    with pytest.raises(amr.AmrError) as e:
        p.deposit("segment")
    assert e.value.status == amr.AMR_EINVAL
    p.sort()
    p.deposit("segment")
    p.write(ps.x[::-1].copy(), ps.y, ps.z, ps.m)
    with pytest.raises(amr.AmrError):
        p.deposit("segment")
    with pytest.raises(amr.AmrError):
        p.deposit(7)
    p.close()


def test_edge_cases():
    import oracle
    from paper_2607_20704_gb300 import amr
    n = 8
    # no particles
    e = np.zeros(0)
    for algo in ("atomic", "segment"):
        p = amr.Particles(n, e, e, e, e)
        p.sort()
        p.deposit(algo)
        assert np.array_equal(p.rho(), np.zeros((n, n, n)))
        p.close()
    # particles on cell centres, faces, the origin and just below 1
    c = np.array([0.5 / n, 3.5 / n, 1.0 / n, 0.0, 1.0 - 2.0 ** -53, 0.5, 7.5 / n])
    x, y, z = c, np.roll(c, 1), np.roll(c, 2)
    m = np.arange(1.0, 8.0)
    ref = oracle.cic_deposit(n, x, y, z, m)
    for prec in (8, 4):
        for algo in ("atomic", "segment"):
            p = amr.Particles(n, x, y, z, m, precision=prec)
            p.sort()
            p.deposit(algo)
            _assert_close(p.rho(), ref, _bound(n, x, y, z, m, ref, prec), ("edges", algo))
            p.close()
    # all particles in one source cell: full-warp and multi-warp segments
    for cnt in (31, 32, 33, 1000, 4099):
        x = np.full(cnt, 0.3)
        y = 0.3 + np.linspace(0, 0.01, cnt)
        z = np.full(cnt, 0.71)
        m = np.linspace(1.0, 2.0, cnt)
        ref = oracle.cic_deposit(16, x, y, z, m)
        bound = _bound(16, x, y, z, m, ref, 8)
        for algo in ("atomic", "segment"):
            p = amr.Particles(16, x, y, z, m)
            p.sort()
            p.deposit(algo)
            _assert_close(p.rho(), ref, bound, ("one cell", cnt, algo))
            p.close()


def test_info_and_timing():
    from paper_2607_20704_gb300 import amr
    ps = inputs.particles(16, "cosmo", seed=12)
    p = amr.Particles(*ps.args())
    p.set_timing(True)
    p.sort()
    p.deposit("atomic")
    p.deposit("segment")
    t = p.read_timing()
    for k in ("part_keys", "psort_hist", "psort_scatter", "part_gather", "cic_atomic", "seg_partial",
              "seg_gather"):
        assert k in t and t[k][1] >= 1, k
    inf = p.info()
    assert inf["np"] == ps.np and inf["sorted"] == 1
    src = [np.floor(a * 16 - 0.5).astype(np.int64) % 16 for a in (ps.x, ps.y, ps.z)]
    assert inf["n_segments"] == np.unique(src[0] + 16 * (src[1] + 16 * src[2])).shape[0]
    p.close()


@pytest.mark.parametrize("precision", [8, 4])
def test_device_view_of_the_grid(precision):
    from paper_2607_20704_gb300 import amr
    ps = inputs.particles(16, "cosmo", seed=13)
    p = amr.Particles(*ps.args(), precision=precision)
    p.deposit("atomic")
    view = p.rho_device()
    assert view.shape == (16 ** 3,) and view.is_cuda
    assert str(view.dtype) == ("torch.float64" if precision == 8 else "torch.float32")
    host = p.rho().reshape(-1, order="F")
    assert np.array_equal(view.double().cpu().numpy(), host)
    p.close()


def _sampled_parity(ps, precision, algo, n_samples=48, seed=0):
    """Full-size check: total mass, and the oracle's density at sampled cells
    computed from just the particles whose stencils reach them."""
    import oracle
    from paper_2607_20704_gb300 import amr
    n = ps.n
    p = amr.Particles(*ps.args(), precision=precision)
    p.sort()
    p.deposit(algo)
    rho = p.rho()
    p.close()
    tol_mass = 1e-12 if precision == 8 else 1e-5
    assert abs(rho.sum() / n ** 3 - ps.m.sum()) <= tol_mass * ps.m.sum()
    rng = np.random.default_rng(seed)
    # sample cells: random ones and the densest ones
    flat = rho.reshape(-1, order="F")
    cells = np.concatenate([rng.integers(0, n ** 3, n_samples // 2),
                            np.argpartition(flat, -n_samples // 2)[-n_samples // 2:]])
    src = [np.floor(a * n - 0.5).astype(np.int64) % n for a in (ps.x, ps.y, ps.z)]
    lin = src[0] + n * (src[1] + n * src[2])
    ci, cj, ck = cells % n, (cells // n) % n, cells // (n * n)
    # every particle whose (FP32-widened) stencil may reach a sampled cell:
    # source cells at offsets -2..1 behind it per axis
    want = set()
    for ox in range(-2, 2):
        for oy in range(-2, 2):
            for oz in range(-2, 2):
                want.update((((ci + ox) % n) + n * (((cj + oy) % n) + n * ((ck + oz) % n))).tolist())
    sel = np.isin(lin, np.fromiter(want, np.int64))
    sub = [a[sel] for a in (ps.x, ps.y, ps.z, ps.m)]
    ref_grid = oracle.cic_deposit(n, *sub)
    bound = _bound(n, *sub, ref_grid, precision).reshape(-1, order="F")[cells]
    ref = ref_grid.reshape(-1, order="F")[cells]
    got = flat[cells]
    assert np.all(np.abs(got - ref) <= bound + 1e-300), (np.abs(got - ref) - bound).max()


@pytest.mark.parametrize("precision,algo", [(8, "atomic"), (8, "segment"), (4, "atomic")])
def test_full_size_cosmological_configuration(precision, algo):
    """512^3 particles on the 512^3 grid (the benchmarked configuration)."""
    ps = _full_set()
    _sampled_parity(ps, precision, algo)


_FULL = {}


def _full_set():
    if "ps" not in _FULL:
        _FULL["ps"] = inputs.particles(512, "cosmo", seed=2607)
    return _FULL["ps"]


def bound_at(n, x, y, z, m, ref, cells, precision):
    """_bound() at the given cells only (flat indices i + n (j + n k), no
    repeats), without n^3 arrays: K and M summed over the particles whose
    (FP32-widened) stencil covers each cell."""
    order = np.argsort(cells)
    sc = cells[order]
    K = np.zeros(cells.shape[0], np.int64)
    M = np.zeros(cells.shape[0])
    if precision == 8:
        lo = [np.floor(a * n - 0.5).astype(np.int64) for a in (x, y, z)]
        hi = [v + 1 for v in lo]
    else:
        d = n * 2.0 ** -23
        lo = [np.floor(a * n - 0.5 - d).astype(np.int64) for a in (x, y, z)]
        hi = [np.floor(a * n - 0.5 + d).astype(np.int64) + 1 for a in (x, y, z)]
    reach = 2 if precision == 8 else 3
    for ox in range(reach):
        for oy in range(reach):
            for oz in range(reach):
                ok = (lo[0] + ox <= hi[0]) & (lo[1] + oy <= hi[1]) & (lo[2] + oz <= hi[2])
                idx = ((lo[0] + ox) % n) + n * (((lo[1] + oy) % n) + n * ((lo[2] + oz) % n))
                pos = np.minimum(np.searchsorted(sc, idx), sc.shape[0] - 1)
                hit = ok & (sc[pos] == idx)
                np.add.at(K, order[pos[hit]], 1)
                np.add.at(M, order[pos[hit]], m[hit] * float(n) ** 3)
    if precision == 8:
        return (2 * K + 8) * U64 * ref
    return (6 * n + 12 + K) * U32 * M


@pytest.mark.parametrize("precision,algo", [(8, "atomic"), (8, "segment"), (4, "atomic"), (4, "segment")])
def test_largest_grid(precision, algo):
    """The largest grid a handle accepts (1024^3 cells: 30-bit source-cell
    keys, sorted in four radix passes of 8, 8, 8 and 6 bits), with a
    clustered set of 64^3 lattice particles and their halos: total mass and
    sampled cells (read on the device; the oracle deposits only the
    particles that reach them)."""
    import torch
    import oracle
    from paper_2607_20704_gb300 import amr
    ps = _largest_set()
    n = ps.n
    p = amr.Particles(*ps.args(), precision=precision)
    p.sort()
    p.deposit(algo)
    rho = p.rho_device()
    total = float(rho.double().sum()) / n ** 3
    tol_mass = 1e-12 if precision == 8 else 1e-5
    assert abs(total - ps.m.sum()) <= tol_mass * ps.m.sum()
    rng = np.random.default_rng(1)
    dense = torch.topk(rho, 32).indices.cpu().numpy().astype(np.int64)
    cells = np.unique(np.concatenate([rng.integers(0, n ** 3, 32), dense]))
    got = rho[torch.as_tensor(cells, device="cuda")].double().cpu().numpy()
    del rho
    p.close()
    src = [np.floor(a * n - 0.5).astype(np.int64) % n for a in (ps.x, ps.y, ps.z)]
    lin = src[0] + n * (src[1] + n * src[2])
    ci, cj, ck = cells % n, (cells // n) % n, cells // (n * n)
    want = set()
    for ox in range(-2, 2):
        for oy in range(-2, 2):
            for oz in range(-2, 2):
                want.update((((ci + ox) % n) + n * (((cj + oy) % n) + n * ((ck + oz) % n))).tolist())
    sel = np.isin(lin, np.fromiter(want, np.int64))
    sub = [a[sel] for a in (ps.x, ps.y, ps.z, ps.m)]
    ref = oracle.cic_deposit(n, *sub).reshape(-1, order="F")[cells]
    bound = bound_at(n, *sub, ref, cells, precision)
    assert np.all(np.abs(got - ref) <= bound + 1e-300), (np.abs(got - ref) - bound).max()


def _largest_set():
    if "big" not in _FULL:
        _FULL["big"] = inputs.particles(1024, "cosmo", seed=31, lattice=64, disp=4.0, halo_particles=512)
    return _FULL["big"]
