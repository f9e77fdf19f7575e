"""Near-threshold refinement decisions, computed on the test side.

The regrid criterion (a reading of Sec. 2.2) flags a cell when the relative
jump J = 2|a-b|/(|a|+|b|) of rho or p to one of its six face neighbours (the
same-level cell, else the coarser cell covering it) exceeds a threshold.
The oracle evaluates that quotient with p from the primitive conversion; a
GPU may decide the same inequality in another rounding (the division-free
form, another association of the kinetic energy).  Both are within a few
rounding errors of the exact decision, so the two can differ only for cells
whose J lies within a band around the threshold:

    band_rho = 16 u thr
    band_p   = 16 u thr + (2 + thr) eps_p,   eps_p = 8 u (E + e_k) / |E - e_k|

u = 2^-53; eps_p bounds the relative difference of two evaluations of
p = (gamma-1)(E - e_k) whose kinetic energies e_k differ by a few rounding
errors (the cancellation E - e_k amplifies them by (E + e_k)/|E - e_k|), and
a relative change eps of both arguments moves J by at most (2 + J) eps.

A raw flag that changes moves the final flags of a neighbourhood: expansion
flags the 26 same-level cells around it, grading the coarser cells covering
the 27 neighbours of every flagged cell.  ``influence`` returns, per level,
the cells within that reach of an ambiguous cell (a box of +-2 cells of the
ambiguous cell's level, widened by 2 cells of every coarser level it
reaches), where final flags may legitimately differ.

Everything here is written from those definitions in numpy; it calls
nothing of the oracle's or the GPU's arithmetic."""
import numpy as np

U_ROUND = 2.0 ** -53
SMALLR = 1e-10
SMALLC = 1e-10


def pack(level, i, j, k):
    return ((np.uint64(level) << np.uint64(60)) | (i.astype(np.uint64) << np.uint64(40)) |
            (j.astype(np.uint64) << np.uint64(20)) | k.astype(np.uint64))


def unpack(keys):
    keys = keys.astype(np.uint64)
    m = np.uint64((1 << 20) - 1)
    return ((keys >> np.uint64(40)) & m).astype(np.int64), ((keys >> np.uint64(20)) & m).astype(
        np.int64), (keys & m).astype(np.int64)


class Levels:
    """Keys and states of every level of a mesh (as ``read`` returns them)."""

    def __init__(self, mesh, gamma):
        self.gamma = gamma
        self.lv = {}
        for l in mesh.levels():
            keys, U = mesh.read(l)
            order = np.argsort(keys)
            self.lv[l] = (keys, U, keys[order], order)
        self.lmin = min(self.lv)

    def cell_values(self, L, x, y, z):
        """States [5][n] of level-L cells (x, y, z) (periodic), else of the
        coarser cell covering them; NaN where none exists."""
        n = x.shape[0]
        out = np.full((5, n), np.nan)
        todo = np.arange(n)
        x, y, z = x.copy(), y.copy(), z.copy()
        while todo.size and L >= self.lmin:
            side = 1 << L
            X, Y, Z = x[todo] % side, y[todo] % side, z[todo] % side
            if L in self.lv:
                keys, U, skeys, order = self.lv[L]
                want = pack(L, X >> 1, Y >> 1, Z >> 1)
                pos = np.searchsorted(skeys, want)
                pos = np.minimum(pos, skeys.size - 1)
                hit = skeys[pos] == want
                o = order[pos[hit]]
                c = (X[hit] & 1) + 2 * (Y[hit] & 1) + 4 * (Z[hit] & 1)
                out[:, todo[hit]] = U[:, 8 * o + c]
                miss = ~hit
            else:
                miss = np.ones(todo.size, bool)
            todo = todo[miss]
            x[todo] = X[miss] >> 1
            y[todo] = Y[miss] >> 1
            z[todo] = Z[miss] >> 1
            L -= 1
        return out


def _prim(U, gamma):
    r = np.maximum(U[0], SMALLR)
    v = U[1:4] / r
    ek = 0.5 * r * (v * v).sum(axis=0)
    p = np.maximum((gamma - 1.0) * (U[4] - ek), r * SMALLC * SMALLC / gamma)
    eps = 8.0 * U_ROUND * (np.abs(U[4]) + ek) / np.maximum(np.abs(U[4] - ek), 1e-300)
    return r, p, eps


def _jump(a, b):
    s = np.abs(a) + np.abs(b)
    return np.where(s > 0, 2.0 * np.abs(a - b) / np.where(s > 0, s, 1.0), 0.0)


def ambiguous(mesh, gamma, levelmax, grad_rho, grad_p, mass=0.0, **_):
    """Per level, a boolean [8 n] mask of the cells whose raw flag lies
    within the band of a threshold (the mass test is exact on both sides:
    a power-of-two scaling, no band)."""
    L = Levels(mesh, gamma)
    out = {}
    for l, (keys, U, _, _) in L.lv.items():
        n = keys.size
        amb = np.zeros(8 * n, bool)
        if l >= levelmax or n == 0 or not (grad_rho > 0 or grad_p > 0):
            out[l] = amb
            continue
        i, j, k = unpack(keys)
        c = np.arange(8)
        x = (2 * i[:, None] + (c & 1)).ravel()
        y = (2 * j[:, None] + ((c >> 1) & 1)).ravel()
        z = (2 * k[:, None] + ((c >> 2) & 1)).ravel()
        rc, pc, ec = _prim(U, gamma)
        for d in range(3):
            for s in (-1, 1):
                sh = [x, y, z]
                sh = [a + (s if q == d else 0) for q, a in enumerate(sh)]
                un = L.cell_values(l, *sh)
                have = ~np.isnan(un[0])
                un = np.where(have, un, U)
                rn, pn, en = _prim(un, gamma)
                if grad_rho > 0:
                    J = _jump(rn, rc)
                    amb |= have & (np.abs(J - grad_rho) <= 16 * U_ROUND * grad_rho)
                if grad_p > 0:
                    J = _jump(pn, pc)
                    band = 16 * U_ROUND * grad_p + (2.0 + grad_p) * np.maximum(en, ec)
                    amb |= have & (np.abs(J - grad_p) <= band)
        out[l] = amb
    return out


def influence(mesh, amb):
    """Per level, a boolean [8 n] mask of the cells whose final flag an
    ambiguous raw flag can reach through expansion and grading."""
    boxes = []  # (level, lo[3], hi[3]) in level coordinates, inclusive
    lv = {}
    for l in mesh.levels():
        keys, _ = mesh.read(l)
        i, j, k = unpack(keys)
        c = np.arange(8)
        x = (2 * i[:, None] + (c & 1)).ravel()
        y = (2 * j[:, None] + ((c >> 1) & 1)).ravel()
        z = (2 * k[:, None] + ((c >> 2) & 1)).ravel()
        lv[l] = (x, y, z)
        if l in amb and amb[l].any():
            q = np.flatnonzero(amb[l])
            for t in q:
                boxes.append((l, np.array([x[t], y[t], z[t]]) - 2, np.array([x[t], y[t], z[t]]) + 2))
    out = {l: np.zeros(v[0].size, bool) for l, v in lv.items()}
    for (la, lo, hi) in boxes:
        for l, (x, y, z) in lv.items():
            if l > la:
                continue
            # the box seen at level l (coarsened), widened by 2 cells per level crossed
            w = 2 * (la - l)
            sh = la - l
            blo = (lo >> sh) - w
            bhi = (hi >> sh) + w
            side = 1 << l
            inside = np.ones(x.size, bool)
            for a, b0, b1 in ((x, blo[0], bhi[0]), (y, blo[1], bhi[1]), (z, blo[2], bhi[2])):
                d0 = (a - b0) % side
                inside &= d0 <= (b1 - b0)
            out[l] |= inside
    return out
