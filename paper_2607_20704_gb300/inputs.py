"""Seeded synthetic inputs: graded oct lists and initial states.

This module is shared by the CUDA path's tests and benchmark and by the
oracle's tests.  It holds none of the method's arithmetic (no hashing, no
ordering, no neighbour search, no hydro): it only lays out which octs exist
and what the initial primitive fields are at cell centres.

Conventions: an oct of level ``l`` has integer coordinates in
``[0, 2^(l-1))^3``; its 8 cells are ``c = cx + 2cy + 4cz``; a cell of level
``l`` has size ``2^-l`` in the periodic unit box.  The oct with coordinates
``(i, j, k)`` at level ``l+1`` is the child block of cell ``(i, j, k)`` of
level ``l``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

NV = 5
COORD_BITS = 20


# ---------------------------------------------------------------------------
# cell sets as packed int64 codes
# ---------------------------------------------------------------------------
def _code(x, y, z):
    return (np.asarray(x, np.int64) << 40) | (np.asarray(y, np.int64) << 20) | np.asarray(z, np.int64)


def _decode(c):
    c = np.asarray(c, np.int64)
    return (c >> 40) & 0xFFFFF, (c >> 20) & 0xFFFFF, c & 0xFFFFF


def _neighbourhood_fathers(cells, level):
    """Codes of the level-(l-1) cells that must be split so that the 27
    level-l cells around each of ``cells`` (level l) exist."""
    x, y, z = _decode(cells)
    side = 1 << level
    out = []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                nx = (x + dx) % side
                ny = (y + dy) % side
                nz = (z + dz) % side
                out.append(_code(nx >> 1, ny >> 1, nz >> 1))
    return np.unique(np.concatenate(out)) if out else np.zeros(0, np.int64)


def graded_octs(levelmin: int, split: dict[int, np.ndarray]):
    """Oct list of a graded octree.

    ``split[l]`` holds codes of level-l cells to split (l >= levelmin).  Cells
    are added to coarser split sets until every oct of level l+1 has the 27
    level-l cells around its father present (the 2:1 grading rule).
    Returns (level, i, j, k) arrays, octs of each level in (i, j, k) order.
    """
    split = {l: np.unique(np.asarray(v, np.int64)) for l, v in split.items() if len(v)}
    levels = sorted(split)
    if levels:
        for l in range(max(levels), levelmin, -1):
            cur = split.get(l)
            if cur is None or len(cur) == 0:
                continue
            need = _neighbourhood_fathers(cur, l)
            prev = split.get(l - 1, np.zeros(0, np.int64))
            split[l - 1] = np.union1d(prev, need)
    side = 1 << (levelmin - 1)
    g = np.arange(side, dtype=np.int64)
    I, J, K = np.meshgrid(g, g, g, indexing="ij")
    lv = [np.full(side ** 3, levelmin, np.uint8)]
    ii, jj, kk = [I.ravel()], [J.ravel()], [K.ravel()]
    for l in sorted(split):
        x, y, z = _decode(split[l])
        lv.append(np.full(len(x), l + 1, np.uint8))
        ii.append(x)
        jj.append(y)
        kk.append(z)
    return (np.concatenate(lv), np.concatenate(ii).astype(np.uint32),
            np.concatenate(jj).astype(np.uint32), np.concatenate(kk).astype(np.uint32))


def cell_centres(level, i, j, k):
    """Cell-centre coordinates, arrays of shape (n, 8) in cell order."""
    level = np.asarray(level, np.int64)
    dx = np.ldexp(1.0, -level)[:, None]
    c = np.arange(8)
    cx, cy, cz = c & 1, (c >> 1) & 1, (c >> 2) & 1
    x = (2 * np.asarray(i, np.int64)[:, None] + cx[None, :] + 0.5) * dx
    y = (2 * np.asarray(j, np.int64)[:, None] + cy[None, :] + 0.5) * dx
    z = (2 * np.asarray(k, np.int64)[:, None] + cz[None, :] + 0.5) * dx
    return x, y, z


def cells_of_level(level: int):
    """Codes and centres of every cell of a level over the whole box."""
    side = 1 << level
    g = np.arange(side, dtype=np.int64)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    dx = 2.0 ** -level
    return _code(X.ravel(), Y.ravel(), Z.ravel()), (X.ravel() + 0.5) * dx, (Y.ravel() + 0.5) * dx, (Z.ravel() + 0.5) * dx


def cells_in_ball(level: int, centre, radius: float):
    """Codes of level-l cells whose centre lies within ``radius`` of
    ``centre`` (periodic distance), without enumerating the whole box."""
    dx = 2.0 ** -level
    side = 1 << level
    lo = np.floor((np.asarray(centre) - radius) / dx).astype(np.int64) - 1
    hi = np.ceil((np.asarray(centre) + radius) / dx).astype(np.int64) + 1
    gx = np.arange(lo[0], hi[0] + 1)
    gy = np.arange(lo[1], hi[1] + 1)
    gz = np.arange(lo[2], hi[2] + 1)
    X, Y, Z = np.meshgrid(gx, gy, gz, indexing="ij")
    cx, cy, cz = (X + 0.5) * dx, (Y + 0.5) * dx, (Z + 0.5) * dx
    r2 = (cx - centre[0]) ** 2 + (cy - centre[1]) ** 2 + (cz - centre[2]) ** 2
    m = r2 < radius * radius
    return np.unique(_code(X[m] % side, Y[m] % side, Z[m] % side))


def prim_to_cons(gamma, rho, u, v, w, p):
    """Initial conservative state [5][8n] from primitive fields of shape (n, 8)."""
    n = rho.shape[0]
    U = np.empty((NV, 8 * n), np.float64)
    U[0] = rho.ravel()
    U[1] = (rho * u).ravel()
    U[2] = (rho * v).ravel()
    U[3] = (rho * w).ravel()
    U[4] = (p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)).ravel()
    return U


# ---------------------------------------------------------------------------
# problems
# ---------------------------------------------------------------------------
@dataclass
class Problem:
    name: str
    levelmin: int
    levelmax: int
    gamma: float
    cfl: float
    level: np.ndarray
    i: np.ndarray
    j: np.ndarray
    k: np.ndarray
    U: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n_oct(self) -> int:
        return int(self.level.shape[0])

    def mesh_args(self):
        return self.level, self.i, self.j, self.k, self.U

    def params(self):
        return dict(levelmin=self.levelmin, levelmax=self.levelmax, gamma=self.gamma, cfl=self.cfl)

    def shuffled(self, seed: int) -> "Problem":
        """Same problem with the oct list in a seeded random order."""
        rng = np.random.default_rng(seed)
        p = rng.permutation(self.n_oct)
        cells = (8 * p[:, None] + np.arange(8)[None, :]).ravel()
        return Problem(self.name, self.levelmin, self.levelmax, self.gamma, self.cfl,
                       self.level[p], self.i[p], self.j[p], self.k[p],
                       np.ascontiguousarray(self.U[:, cells]), dict(self.meta))

    def leaf_cells(self) -> int:
        """Number of leaf cells: each oct above levelmin splits one cell."""
        return int(8 * self.n_oct - np.count_nonzero(self.level > self.levelmin))


def _state(gamma, level, i, j, k, fn):
    x, y, z = cell_centres(level, i, j, k)
    rho, u, v, w, p = fn(x, y, z)
    return prim_to_cons(gamma, rho, u, v, w, p)


def sod(levelmin: int = 6, levelmax: int = 7, slab=(0.45, 0.55), gamma: float = 1.4,
        cfl: float = 0.8, axis: int = 0) -> Problem:
    """3-D Sod tube along ``axis``: left (rho=1, p=1) for coordinate < 0.5,
    right (rho=0.125, p=0.1) otherwise, at rest; the level-``levelmin`` cells
    whose centre lies in ``slab`` are refined once when levelmax > levelmin.
    The periodic box holds a second, reversed interface at 0 (not refined)."""
    split = {}
    if levelmax > levelmin:
        codes, cx, cy, cz = cells_of_level(levelmin)
        c = (cx, cy, cz)[axis]
        split[levelmin] = codes[(c > slab[0]) & (c < slab[1])]
    lv, i, j, k = graded_octs(levelmin, split)

    def fn(x, y, z):
        c = (x, y, z)[axis]
        left = c < 0.5
        rho = np.where(left, 1.0, 0.125)
        p = np.where(left, 1.0, 0.1)
        zero = np.zeros_like(rho)
        return rho, zero, zero.copy(), zero.copy(), p

    return Problem("sod", levelmin, levelmax, gamma, cfl, lv, i, j, k, _state(gamma, lv, i, j, k, fn),
                   {"slab": slab, "axis": axis})


def sedov(levelmin: int = 7, levelmax: int = 10, radii=None, gamma: float = 5.0 / 3.0,
          cfl: float = 0.8, energy: float = 1.0, rho0: float = 1.0, p0: float = 1e-5,
          centre=(0.5, 0.5, 0.5)) -> Problem:
    """Sedov blast: ambient rho0, p0 at rest; ``energy`` added uniformly to
    the finest-level cells whose centre lies within two finest-cell widths
    of ``centre``.  Levels levelmin+1..levelmax are static nested balls of
    radius ``radii[l]`` (default 0.12 / 0.06 / 0.03 for the three finest
    levels, doubling further out), graded."""
    if radii is None:
        radii = {}
        r = 0.03
        for l in range(levelmax, levelmin, -1):
            radii[l] = r
            r *= 2.0
    split = {}
    for l in range(levelmin + 1, levelmax + 1):
        split[l - 1] = cells_in_ball(l - 1, centre, radii[l])
    lv, i, j, k = graded_octs(levelmin, split)
    x, y, z = cell_centres(lv, i, j, k)
    rho = np.full(x.shape, rho0)
    zero = np.zeros_like(rho)
    p = np.full(x.shape, p0)
    U = prim_to_cons(gamma, rho, zero, zero, zero, p)
    # energy deposit on the finest level present
    lfine = int(lv.max())
    dxf = 2.0 ** -lfine
    r2 = (x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2
    hot = (r2 < (2.0 * dxf) ** 2) & (lv[:, None] == lfine)
    nhot = int(hot.sum())
    if nhot:
        U[4] = U[4] + np.where(hot.ravel(), energy / (nhot * dxf ** 3), 0.0)
    return Problem("sedov", levelmin, levelmax, gamma, cfl, lv, i, j, k, U,
                   {"radii": radii, "n_hot": nhot, "energy": energy, "rho0": rho0, "p0": p0,
                    "centre": centre})


def gaussian_field(n: int, index: float, sigma: float, rng,
                   smooth: float = 0.0) -> tuple[np.ndarray, np.ndarray]:
    """Gaussian random field on an n^3 periodic grid with power spectrum
    P(k) ~ k^index (k = 0 removed), smoothed by a Gaussian of ``smooth`` grid
    cells, rescaled to standard deviation sigma.  Returns the real field and
    its Fourier transform (rfftn layout)."""
    kx = np.fft.fftfreq(n) * n
    kz = np.fft.rfftfreq(n) * n
    KX, KY, KZ = np.meshgrid(kx, kx, kz, indexing="ij")
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    amp = np.zeros_like(k2)
    nz = k2 > 0
    amp[nz] = k2[nz] ** (index / 4.0)  # sqrt(P) = k^(index/2)
    if smooth > 0:
        amp *= np.exp(-0.5 * k2 * (2.0 * np.pi * smooth / n) ** 2)
    noise = np.fft.rfftn(rng.standard_normal((n, n, n)))
    gk = noise * amp
    g = np.fft.irfftn(gk, s=(n, n, n), axes=(0, 1, 2))
    s = g.std()
    return g * (sigma / s), gk * (sigma / s)


def lognormal(levelmin: int = 8, extra: int = 4, sigma: float = 1.5, index: float = -2.0,
              seed: int = 7, vsigma: float = 0.1, gamma: float = 5.0 / 3.0,
              cfl: float = 0.8, threshold: float = 8.0, smooth: float = 0.0,
              isothermal: float | None = None) -> Problem:
    """Cosmology-shaped clustered mesh: lognormal density rho = exp(g - s^2/2)
    of a Gaussian field g (spectrum k^index, optionally smoothed over
    ``smooth`` base cells, std ``sigma``) on the base level; velocities
    v_a ~ i k_a / k^2 g_k, each component rescaled to std ``vsigma``;
    p = 1e-4 rho^(5/3), or p = ``isothermal`` * rho when given.  The default
    (unsmoothed, adiabat) state has flows up to Mach ~150 between nearly
    uncorrelated neighbouring cells: fine for single level steps, but over
    whole coarse steps the minmod prolongation of such ghosts drives coarse
    cells negative; ``smooth=1, isothermal=0.01`` (peak Mach ~3) is the
    well-posed variant for multi-step runs.  A cell of level l is refined where its
    mass exceeds ``threshold`` times the mean base-cell mass, i.e.
    rho > threshold^(1 + l - levelmin); up to ``extra`` levels, graded.
    Refined cells pass their values unchanged to their children."""
    rng = np.random.default_rng(seed)
    n = 1 << levelmin
    g, gk = gaussian_field(n, index, sigma, rng, smooth)
    rho_b = np.exp(g - 0.5 * sigma * sigma)
    kx = np.fft.fftfreq(n) * n
    kz = np.fft.rfftfreq(n) * n
    KX, KY, KZ = np.meshgrid(kx, kx, kz, indexing="ij")
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    k2[0, 0, 0] = 1.0
    vel = []
    for K in (KX, KY, KZ):
        vk = 1j * K / k2 * gk
        vk[0, 0, 0] = 0.0
        v = np.fft.irfftn(vk, s=(n, n, n), axes=(0, 1, 2))
        vel.append(v * (vsigma / v.std()))
    del gk, KX, KY, KZ, k2
    # refinement, top down; children inherit the father's density
    split = {}
    cur = None  # codes of base cells covered by the current level's octs
    base_codes, _, _, _ = cells_of_level(levelmin)
    rho_flat = rho_b.ravel()  # index = x * n^2 + y * n + z (ij meshgrid order)
    flagged = base_codes[rho_flat > threshold]
    if extra > 0 and len(flagged):
        split[levelmin] = flagged
        cur = flagged
        for l in range(levelmin + 1, levelmin + extra):
            x, y, z = _decode(cur)
            kids = []
            for c in range(8):
                kids.append(_code(2 * x + (c & 1), 2 * y + ((c >> 1) & 1), 2 * z + ((c >> 2) & 1)))
            kids = np.concatenate(kids)
            kx_, ky_, kz_ = _decode(kids)
            sh = l - levelmin
            bi = ((kx_ >> sh) * n + (ky_ >> sh)) * n + (kz_ >> sh)
            sel = rho_flat[bi] > threshold ** (1 + l - levelmin)
            cur = np.unique(kids[sel])
            if len(cur) == 0:
                break
            split[l] = cur
    lv, i, j, k = graded_octs(levelmin, split)
    x, y, z = cell_centres(lv, i, j, k)
    # sample the base-level fields at the base cell containing each centre
    bx = np.minimum((x * n).astype(np.int64), n - 1)
    by = np.minimum((y * n).astype(np.int64), n - 1)
    bz = np.minimum((z * n).astype(np.int64), n - 1)
    rho = rho_b[bx, by, bz]
    u = vel[0][bx, by, bz]
    v = vel[1][bx, by, bz]
    w = vel[2][bx, by, bz]
    p = 1e-4 * rho ** (5.0 / 3.0) if isothermal is None else isothermal * rho
    U = prim_to_cons(gamma, rho, u, v, w, p)
    return Problem("lognormal", levelmin, int(lv.max()), gamma, cfl, lv, i, j, k, U,
                   {"sigma": sigma, "index": index, "seed": seed, "extra": extra})


def random_mesh(levelmin: int, levelmax: int, seed: int, gamma: float = 1.4,
                cfl: float = 0.8, n_seeds: int = 3, radius: float = 0.2,
                mach: float = 1.5) -> Problem:
    """Random graded mesh and a rough random state, for parity tests: refined
    balls around ``n_seeds`` random points per level; smooth density and
    pressure with seeded noise and velocities up to about ``mach`` times the
    sound speed, so that every branch of the Riemann solver is taken."""
    rng = np.random.default_rng(seed)
    split = {}
    for l in range(levelmin + 1, levelmax + 1):
        sets = []
        r = radius * 0.6 ** (l - levelmin - 1)
        for _ in range(n_seeds):
            sets.append(cells_in_ball(l - 1, rng.random(3), r))
        split[l - 1] = np.unique(np.concatenate(sets))
    lv, i, j, k = graded_octs(levelmin, split)
    x, y, z = cell_centres(lv, i, j, k)
    ph = rng.random(6) * 2 * np.pi
    rho = 1.0 + 0.5 * np.sin(2 * np.pi * x + ph[0]) * np.cos(2 * np.pi * y + ph[1]) \
        + 0.2 * rng.random(x.shape)
    p = 1.0 + 0.5 * np.cos(2 * np.pi * z + ph[2]) + 0.3 * rng.random(x.shape)
    c = np.sqrt(gamma * p / rho)
    u = mach * c * (np.sin(2 * np.pi * y + ph[3]) + 0.3 * rng.standard_normal(x.shape))
    v = mach * c * (np.sin(2 * np.pi * z + ph[4]) + 0.3 * rng.standard_normal(x.shape))
    w = mach * c * (np.sin(2 * np.pi * x + ph[5]) + 0.3 * rng.standard_normal(x.shape))
    U = prim_to_cons(gamma, rho, u, v, w, p)
    return Problem("random", levelmin, levelmax, gamma, cfl, lv, i, j, k, U, {"seed": seed})


def uniform_state(levelmin: int, levelmax: int, seed: int, gamma: float = 1.4,
                  prim=(1.3, 0.7, -0.4, 0.25, 2.0)) -> Problem:
    """A constant moving state on a random graded mesh (every flux equal)."""
    base = random_mesh(levelmin, levelmax, seed, gamma=gamma)
    rho, u, v, w, p = prim
    shape = (base.n_oct, 8)
    U = prim_to_cons(gamma, np.full(shape, rho), np.full(shape, u), np.full(shape, v),
                     np.full(shape, w), np.full(shape, p))
    return Problem("uniform", levelmin, levelmax, gamma, base.cfl, base.level, base.i, base.j,
                   base.k, U, {"prim": prim})


def uniform_grid(level: int, fn, gamma: float = 1.4, cfl: float = 0.8) -> Problem:
    """Single-level mesh with primitive fields fn(x, y, z) at cell centres."""
    lv, i, j, k = graded_octs(level, {})
    return Problem("uniform_grid", level, level, gamma, cfl, lv, i, j, k,
                   _state(gamma, lv, i, j, k, fn))


def to_array(prob: Problem) -> np.ndarray:
    """State of a single-level problem as an n^3 array U[v][x + n(y + n z)]."""
    assert prob.levelmin == prob.levelmax
    n = 1 << prob.levelmin
    out = np.empty((NV, n ** 3))
    c = np.arange(8)
    gx = (2 * prob.i.astype(np.int64)[:, None] + (c & 1)[None, :]).ravel()
    gy = (2 * prob.j.astype(np.int64)[:, None] + ((c >> 1) & 1)[None, :]).ravel()
    gz = (2 * prob.k.astype(np.int64)[:, None] + ((c >> 2) & 1)[None, :]).ravel()
    out[:, gx + n * (gy + n * gz)] = prob.U
    return out


def batched(n_members: int = 512, seed: int = 11, max_extra: int = 3):
    """Ensemble of independent meshes for batched advancing: Sod or Sedov
    (50/50), base 16^3, 32^3 or 64^3 cells (uniform in log), 0..max_extra
    extra levels (Sod: nested slabs around the interface; Sedov: nested
    balls), all drawn from one seeded generator."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_members):
        kind = "sod" if rng.random() < 0.5 else "sedov"
        lmin = int(rng.integers(4, 7))
        extra = int(rng.integers(0, max_extra + 1))
        lmax = lmin + extra
        if kind == "sod":
            prob = _nested_sod(lmin, lmax, axis=int(rng.integers(0, 3)))
        else:
            radii = {l: 0.24 * 0.5 ** (l - lmin - 1) for l in range(lmin + 1, lmax + 1)}
            prob = sedov(lmin, lmax, radii=radii)
        out.append(prob)
    return out


def _nested_sod(levelmin: int, levelmax: int, axis: int = 0, gamma: float = 1.4, cfl: float = 0.8):
    """Sod tube with nested refined slabs around the interface at 1/2:
    level l+1 covers the level-l cells within 0.05 * 2^-(l-levelmin) of it
    and, below the first extra level, within 0.3 * 2^-(l-levelmin) of the
    tube's axis (a patch of the interface)."""
    split = {}
    for l in range(levelmin, levelmax):
        half = 0.05 * 0.5 ** (l - levelmin)
        side = 1 << l
        g = np.arange(side, dtype=np.int64)
        c = (g + 0.5) / side
        sel = g[np.abs(c - 0.5) < half]
        A, B, Cc = np.meshgrid(sel, g, g, indexing="ij")
        A, B, Cc = A.ravel(), B.ravel(), Cc.ravel()
        if l > levelmin:
            r = 0.3 * 0.5 ** (l - levelmin)
            tb, tc = (B + 0.5) / side - 0.5, (Cc + 0.5) / side - 0.5
            keep = tb * tb + tc * tc < r * r
            A, B, Cc = A[keep], B[keep], Cc[keep]
        coords = [None, None, None]
        coords[axis] = A
        others = [d for d in range(3) if d != axis]
        coords[others[0]] = B
        coords[others[1]] = Cc
        split[l] = _code(*coords)
    lv, i, j, k = graded_octs(levelmin, split)

    def fn(x, y, z):
        c = (x, y, z)[axis]
        left = c < 0.5
        rho = np.where(left, 1.0, 0.125)
        p = np.where(left, 1.0, 0.1)
        zero = np.zeros_like(rho)
        return rho, zero, zero.copy(), zero.copy(), p

    return Problem("sod", levelmin, levelmax, gamma, cfl, lv, i, j, k, _state(gamma, lv, i, j, k, fn),
                   {"axis": axis})


def serving_requests(n_requests: int, seed: int = 13, pool: int = 24, max_level_base: int = 7,
                     max_steps: int = 200):
    """Seeded request stream for the serving loop: each request draws a mesh
    from a pool of Sod / Sedov / lognormal-clustered problems (base 16^3 to
    128^3 cells uniform in log, 0-3 extra levels), a number of coarse steps
    (10..max_steps, uniform in log) and a precision (FP32 or FP64, 50/50).
    Returns (problems, [(pool index, steps, precision)])."""
    rng = np.random.default_rng(seed)
    probs = []
    for t in range(pool):
        kind = ("sod", "sedov", "lognormal")[int(rng.integers(0, 3))]
        lmin = int(rng.integers(4, max_level_base + 1))
        extra = int(rng.integers(0, 4))
        if kind == "sod":
            probs.append(_nested_sod(lmin, lmin + extra, axis=int(rng.integers(0, 3))))
        elif kind == "sedov":
            radii = {l: 0.24 * 0.5 ** (l - lmin - 1) for l in range(lmin + 1, lmin + extra + 1)}
            probs.append(sedov(lmin, lmin + extra, radii=radii))
        else:
            probs.append(lognormal(lmin, extra, seed=int(rng.integers(0, 1 << 30)),
                                   threshold=4.0, smooth=1.0, isothermal=0.01))
    reqs = []
    for _ in range(n_requests):
        steps = int(round(np.exp(rng.uniform(np.log(10), np.log(max_steps)))))
        reqs.append((int(rng.integers(0, pool)), steps, 4 if rng.random() < 0.5 else 8))
    return probs, reqs


# ---------------------------------------------------------------------------
# particles in the periodic unit box (mass deposition workloads)
# ---------------------------------------------------------------------------
@dataclass
class ParticleSet:
    name: str
    n: int  # grid cells per axis of the deposition
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    m: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def np(self) -> int:
        return int(self.x.shape[0])

    def args(self):
        return self.n, self.x, self.y, self.z, self.m


def _into_box(a: np.ndarray) -> np.ndarray:
    a = np.mod(a, 1.0)
    a[a >= 1.0] = 0.0  # a tiny negative value rounds up to 1.0 under mod
    return a


def _upsample_axis(f: np.ndarray, axis: int, L: int) -> np.ndarray:
    """Periodic linear interpolation of f along `axis` from its m points
    (cell centres of an m-grid) to the centres of an L-grid."""
    m = f.shape[axis]
    u = (np.arange(L) + 0.5) * (m / L) - 0.5
    i0 = np.floor(u).astype(np.int64)
    w1 = u - i0
    shape = [1] * f.ndim
    shape[axis] = L
    a = np.take(f, i0 % m, axis=axis)
    b = np.take(f, (i0 + 1) % m, axis=axis)
    return a * (1.0 - w1).reshape(shape) + b * w1.reshape(shape)


def particles(n: int, kind: str = "cosmo", seed: int = 0, lattice: int | None = None,
              n_particles: int | None = None, disp: float = 1.0, halo_fraction: float = 0.25,
              halo_particles: int = 4096, index: float = -3.0, masses: str = "equal",
              chunk: int = 32) -> ParticleSet:
    """Seeded particle sets for deposition on an n^3 grid.

    kind "cosmo": a cosmological-simulation-shaped distribution -- a lattice
    of `lattice`^3 particles (default n^3, one per cell) displaced by a
    Zel'dovich-like field (the gradient of a Gaussian potential with power
    spectrum k^index on a coarse 64^3 grid, scaled to an rms displacement
    of `disp` cells at those points, then linearly interpolated to the
    lattice, which lowers the rms on lattices finer than 64^3: 0.73 `disp`
    at 128^3, 0.75 `disp` at 512^3), with a fraction `halo_fraction`
    of the particles moved into compact halos of about `halo_particles`
    particles each (Gaussian profiles with radii log-uniform in 0.3..3
    cells), so that voids hold ~1 particle per cell and halo cores hundreds.
    kind "uniform": `n_particles` positions uniform in the box.
    kind "clump": `n_particles` in one Gaussian clump of radius one cell.
    masses "equal": every particle 1/N (mean density 1); "random": lognormal
    masses of unit median."""
    rng = np.random.default_rng(seed)
    if kind == "cosmo":
        L = int(lattice or n)
        N = L ** 3
        mc = min(L, 64)
        phi, _ = gaussian_field(mc, index, 1.0, rng)
        psi = [0.5 * (np.roll(phi, -1, axis=a) - np.roll(phi, 1, axis=a)) for a in range(3)]
        rms = np.sqrt(np.mean(psi[0] ** 2 + psi[1] ** 2 + psi[2] ** 2))
        psi = [p * (disp / n / max(rms, 1e-300)) for p in psi]
        x, y, z = (np.empty(N) for _ in range(3))
        q = (np.arange(L) + 0.5) / L
        # psi at the lattice points, `chunk` planes of the first axis at a time
        up1 = [_upsample_axis(_upsample_axis(p, 1, L), 2, L) for p in psi]  # (mc, L, L)
        for a0 in range(0, L, chunk):
            a1 = min(L, a0 + chunk)
            u = (np.arange(a0, a1) + 0.5) * (mc / L) - 0.5
            i0 = np.floor(u).astype(np.int64)
            w1 = (u - i0)[:, None, None]
            sl = slice(a0 * L * L, a1 * L * L)
            for out, comp, axis_q in ((x, 0, 0), (y, 1, 1), (z, 2, 2)):
                f = up1[comp]
                d = f[i0 % mc] * (1.0 - w1) + f[(i0 + 1) % mc] * w1  # (a1-a0, L, L)
                qq = np.broadcast_to(
                    (q[a0:a1][:, None, None], q[None, :, None], q[None, None, :])[axis_q],
                    d.shape)
                out[sl] = (qq + d).reshape(-1)
        nh = int(round(halo_fraction * N))
        if nh > 0:
            pick = np.flatnonzero(rng.random(N) < halo_fraction)
            nh = pick.shape[0]
            n_halo = max(1, nh // max(1, halo_particles))
            centre = rng.random((n_halo, 3))
            radius = np.exp(rng.uniform(np.log(0.3), np.log(3.0), n_halo)) / n
            hid = rng.integers(0, n_halo, nh)
            for out, a in ((x, 0), (y, 1), (z, 2)):
                out[pick] = centre[hid, a] + radius[hid] * rng.standard_normal(nh)
        meta = {"lattice": L, "disp_cells": disp, "halo_fraction": halo_fraction,
                "halo_particles": halo_particles, "index": index}
    elif kind in ("uniform", "clump"):
        N = int(n_particles if n_particles is not None else n ** 3)
        if kind == "uniform":
            x, y, z = rng.random(N), rng.random(N), rng.random(N)
        else:
            c = rng.random(3)
            x, y, z = (c[a] + rng.standard_normal(N) / n for a in range(3))
        meta = {}
    else:
        raise ValueError(f"unknown particle set kind {kind!r}")
    x, y, z = _into_box(x), _into_box(y), _into_box(z)
    if masses == "equal":
        m = np.full(N, 1.0 / max(N, 1))
    elif masses == "random":
        m = np.exp(0.5 * rng.standard_normal(N))
    else:
        raise ValueError(f"unknown masses {masses!r}")
    return ParticleSet(kind, int(n), x, y, z, m, meta)
