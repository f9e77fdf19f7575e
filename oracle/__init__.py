"""Python handle on the plain FP64 C oracle (``amr_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path (the
CUDA library and its binding) never imports this package.

The oracle follows the paper's own structure for one level step (Sec. 3):
gather a 6x6x6 stencil of ``uold`` per oct, convert to primitives, limited
slopes, Hancock predictor, HLLC on every face of the oct's cells, update.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "amr_oracle.c")
HDR = os.path.join(HERE, "amr_oracle.h")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")

NV = 5
ERRORS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "EGRADING", 4: "EDUP"}

_lock = threading.Lock()
_lib = None


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what}: {ERRORS.get(code, code)}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-ffp-contract=off: source-order IEEE)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    newest = max(os.path.getmtime(SRC), os.path.getmtime(HDR))
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < newest:
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


class _Params(C.Structure):
    _fields_ = [("levelmin", C.c_int), ("levelmax", C.c_int),
                ("gamma", C.c_double), ("cfl", C.c_double),
                ("smallr", C.c_double), ("smallc", C.c_double),
                ("reflux", C.c_int)]


class _RegridParams(C.Structure):
    _fields_ = [("grad_rho", C.c_double), ("grad_p", C.c_double), ("mass", C.c_double),
                ("expand", C.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P, I64, U64, D, I = C.c_void_p, C.c_int64, C.c_uint64, C.c_double, C.c_int
            sig = {
                "orc_pack_key": (U64, [I, C.c_uint32, C.c_uint32, C.c_uint32]),
                "orc_fnv1a64_bytes": (U64, [P, C.c_size_t]),
                "orc_fnv1a64_key": (U64, [U64]),
                "orc_hilbert3": (U64, [C.c_uint32, C.c_uint32, C.c_uint32, I]),
                "orc_create": (I, [C.POINTER(_Params), I64, P, P, P, P, P, C.POINTER(P)]),
                "orc_destroy": (None, [P]),
                "orc_num_octs": (I64, [P, I]),
                "orc_level_offset": (I64, [P, I]),
                "orc_num_cache": (I64, [P, I]),
                "orc_lookup": (I64, [P, U64]),
                "orc_read": (I, [P, I, P, P]),
                "orc_read_R": (I, [P, I, P]),
                "orc_read_split": (I, [P, I, P]),
                "orc_read_nbr": (I, [P, I, P]),
                "orc_read_cache": (I, [P, I, P]),
                "orc_ghost": (I, [P, I, P]),
                "orc_write": (I, [P, I, P]),
                "orc_totals": (None, [P, P]),
                "orc_level_totals": (None, [P, I, P]),
                "orc_cic_deposit_levels": (I, [P, I64, P, P, P, P, P, P]),
                "orc_mg_level": (I, [P, I, D, D, P, I, P, P]),
                "orc_cfl_dt": (D, [P]),
                "orc_step_level": (I, [P, I, D]),
                "orc_step_sample": (I, [P, I, D, I64, P, P]),
                "orc_advance": (I, [P, I, C.POINTER(D)]),
                "orc_uniform_step": (I, [I, P, D, D, D, D]),
                "orc_uniform_cfl_dt": (D, [I, P, D, D, D, D]),
                "orc_1d_step": (I, [I, P, D, D, D, D]),
                "orc_flags": (I, [P, C.POINTER(_RegridParams), P]),
                "orc_mg_solve": (I, [I, D, P, D, I, I, I, P, P]),
                "orc_cic_deposit": (I, [I, I64, P, P, P, P, P]),
                "orc_mg_residual": (D, [I, D, P, D, P]),
                "orc_regrid": (I, [C.POINTER(P), C.POINTER(_RegridParams), C.POINTER(I64),
                                   C.POINTER(I64)]),
                "orc_regrid_flags": (I, [C.POINTER(P), P, C.POINTER(I64), C.POINTER(I64)]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def pack_key(level, i, j, k) -> int:
    return int(lib().orc_pack_key(int(level), int(i), int(j), int(k)))


def fnv1a64_bytes(b: bytes) -> int:
    buf = np.frombuffer(b, dtype=np.uint8).copy() if b else np.zeros(1, np.uint8)
    return int(lib().orc_fnv1a64_bytes(_ptr(buf), len(b)))


def fnv1a64_key(key: int) -> int:
    return int(lib().orc_fnv1a64_key(int(key)))


def hilbert3(x, y, z, bits) -> int:
    return int(lib().orc_hilbert3(int(x), int(y), int(z), int(bits)))


class Mesh:
    """An oracle mesh built from an oct list (same inputs as ``amr_create``)."""

    def __init__(self, level, i, j, k, U, *, levelmin, levelmax, gamma, cfl=0.8,
                 smallr=1e-10, smallc=1e-10, reflux=True):
        self.params = _Params(levelmin, levelmax, gamma, cfl, smallr, smallc, int(reflux))
        level = np.ascontiguousarray(level, dtype=np.uint8)
        i = np.ascontiguousarray(i, dtype=np.uint32)
        j = np.ascontiguousarray(j, dtype=np.uint32)
        k = np.ascontiguousarray(k, dtype=np.uint32)
        U = np.ascontiguousarray(U, dtype=np.float64)
        n = level.shape[0]
        assert U.shape == (NV, 8 * n), U.shape
        h = C.c_void_p()
        rc = lib().orc_create(C.byref(self.params), n, _ptr(level), _ptr(i), _ptr(j),
                              _ptr(k), _ptr(U), C.byref(h))
        if rc:
            raise OracleError(rc, "create")
        self._h = h
        self.levelmin, self.levelmax = levelmin, levelmax
        self.gamma = gamma

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    # -- introspection -----------------------------------------------------
    def num_octs(self, level: int) -> int:
        return int(lib().orc_num_octs(self._h, level))

    def level_offset(self, level: int) -> int:
        return int(lib().orc_level_offset(self._h, level))

    def num_cache(self, level: int) -> int:
        return int(lib().orc_num_cache(self._h, level))

    def lookup(self, key: int) -> int:
        return int(lib().orc_lookup(self._h, int(key)))

    def read(self, level: int):
        n = self.num_octs(level)
        keys = np.zeros(max(n, 1), np.uint64)
        U = np.zeros((NV, 8 * max(n, 1)), np.float64)
        lib().orc_read(self._h, level, _ptr(keys), _ptr(U))
        return keys[:n], U[:, :8 * n]

    def read_R(self, level: int):
        n = self.num_octs(level)
        R = np.zeros((NV, 8 * max(n, 1)), np.float64)
        lib().orc_read_R(self._h, level, _ptr(R))
        return R[:, :8 * n]

    def read_split(self, level: int):
        n = self.num_octs(level)
        s = np.zeros(8 * max(n, 1), np.uint8)
        lib().orc_read_split(self._h, level, _ptr(s))
        return s[:8 * n]

    def read_nbr(self, level: int):
        n = self.num_octs(level)
        nb = np.zeros((max(n, 1), 27), np.int64)
        lib().orc_read_nbr(self._h, level, _ptr(nb))
        return nb[:n]

    def read_cache(self, level: int):
        n = self.num_cache(level)
        keys = np.zeros(max(n, 1), np.uint64)
        lib().orc_read_cache(self._h, level, _ptr(keys))
        return keys[:n]

    def ghost(self, level: int):
        n = self.num_cache(level)
        Ug = np.zeros((NV, 8 * max(n, 1)), np.float64)
        rc = lib().orc_ghost(self._h, level, _ptr(Ug))
        if rc:
            raise OracleError(rc, "ghost")
        return Ug[:, :8 * n]

    def write(self, level: int, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        assert U.shape == (NV, 8 * self.num_octs(level))
        lib().orc_write(self._h, level, _ptr(U))

    def totals(self):
        t = np.zeros(NV, np.float64)
        lib().orc_totals(self._h, _ptr(t))
        return t

    def cic_deposit_levels(self, x, y, z, m):
        """CIC deposition onto every level (Sec. 4): per level the density of
        its cells [8 n_level] (read order) and the size of its particle list."""
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z, m)]
        n = int(sum(self.num_octs(l) for l in range(16)))
        rho = np.zeros(8 * max(n, 1), np.float64)
        cnt = np.zeros(16, np.int64)
        rc = lib().orc_cic_deposit_levels(self._h, int(arrs[0].size), *[_ptr(a) for a in arrs],
                                          _ptr(rho), _ptr(cnt))
        if rc:
            raise OracleError(rc, "cic_deposit_levels")
        out = {}
        for l in self.levels():
            a = self.level_offset(l)
            out[l] = rho[8 * a: 8 * (a + self.num_octs(l))]
        return out, cnt

    def mg_level(self, level, phic, fourpiG=1.0, rho_bar=1.0, ncycles=4, phi0=None):
        """Poisson on refined level `level` with the Dirichlet data of the
        coarser level's potential phic (8 n_{level-1}, read order); returns
        (phi [8 n_level], residual norms)."""
        n = self.num_octs(level)
        phic = np.ascontiguousarray(phic, dtype=np.float64)
        assert phic.size == 8 * self.num_octs(level - 1)
        phi = np.zeros(8 * n) if phi0 is None else np.array(phi0, dtype=np.float64)
        res = np.zeros(max(ncycles, 1))
        rc = lib().orc_mg_level(self._h, int(level), float(fourpiG), float(rho_bar), _ptr(phic),
                                int(ncycles), _ptr(phi), _ptr(res))
        if rc:
            raise OracleError(rc, "mg_level")
        return phi, res[:ncycles]

    def level_totals(self, level: int):
        """Sum of U dx^3 over the leaf cells of one level."""
        t = np.zeros(NV, np.float64)
        lib().orc_level_totals(self._h, int(level), _ptr(t))
        return t

    # -- stepping ------------------------------------------------------------
    def cfl_dt(self) -> float:
        return float(lib().orc_cfl_dt(self._h))

    def step_level(self, level: int, dt: float):
        rc = lib().orc_step_level(self._h, level, float(dt))
        if rc:
            raise OracleError(rc, "step_level")

    def step_sample(self, level: int, dt: float, octs):
        octs = np.ascontiguousarray(octs, dtype=np.int64)
        ns = octs.shape[0]
        out = np.zeros((NV, 8 * max(ns, 1)), np.float64)
        rc = lib().orc_step_sample(self._h, level, float(dt), ns, _ptr(octs), _ptr(out))
        if rc:
            raise OracleError(rc, "step_sample")
        return out[:, :8 * ns]

    def advance(self, nsteps: int = 1) -> float:
        dt = C.c_double(0.0)
        rc = lib().orc_advance(self._h, int(nsteps), C.byref(dt))
        if rc:
            raise OracleError(rc, "advance")
        return dt.value

    # -- regrid (Sec. 2.2) ------------------------------------------------------
    def flags(self, grad_rho=0.1, grad_p=0.1, mass=0.0, expand=1):
        """Final refinement flags [8n] in mesh order (all levels)."""
        rp = _RegridParams(grad_rho, grad_p, mass, int(expand))
        n = int(sum(self.num_octs(l) for l in range(16)))
        out = np.zeros(8 * max(n, 1), np.uint8)
        rc = lib().orc_flags(self._h, C.byref(rp), _ptr(out))
        if rc:
            raise OracleError(rc, "flags")
        return out[:8 * n]

    def level_flags(self, level, **kw):
        """Final flags of the cells of one level, [8 n_level]."""
        f = self.flags(**kw)
        a = self.level_offset(level)
        return f[8 * a: 8 * (a + self.num_octs(level))]

    def regrid(self, grad_rho=0.1, grad_p=0.1, mass=0.0, expand=1):
        """Regrid in place; returns (octs created, octs removed)."""
        rp = _RegridParams(grad_rho, grad_p, mass, int(expand))
        h = C.c_void_p(self._h.value if isinstance(self._h, C.c_void_p) else self._h)
        cr, rm = C.c_int64(), C.c_int64()
        rc = lib().orc_regrid(C.byref(h), C.byref(rp), C.byref(cr), C.byref(rm))
        if rc:
            raise OracleError(rc, "regrid")
        self._h = h
        return cr.value, rm.value

    def regrid_flags(self, flags):
        """Regrid in place with the given final flags ([8n] in mesh order, as
        ``flags`` returns them); returns (octs created, octs removed)."""
        n = int(sum(self.num_octs(l) for l in range(16)))
        f = np.ascontiguousarray(flags, dtype=np.uint8)
        assert f.shape == (8 * n,), (f.shape, n)
        h = C.c_void_p(self._h.value if isinstance(self._h, C.c_void_p) else self._h)
        cr, rm = C.c_int64(), C.c_int64()
        rc = lib().orc_regrid_flags(C.byref(h), _ptr(f), C.byref(cr), C.byref(rm))
        if rc:
            raise OracleError(rc, "regrid_flags")
        self._h = h
        return cr.value, rm.value

    def levels(self):
        return [l for l in range(self.levelmin, self.levelmax + 1) if self.num_octs(l) > 0]


def uniform_step(U, gamma, dt, smallr=1e-10, smallc=1e-10):
    """One step of the independent uniform periodic 3-D solver; U is [5][n^3]."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    n = round(U.shape[1] ** (1.0 / 3.0))
    assert n ** 3 == U.shape[1]
    rc = lib().orc_uniform_step(n, _ptr(U), gamma, dt, smallr, smallc)
    if rc:
        raise OracleError(rc, "uniform_step")
    return U


def uniform_cfl_dt(U, gamma, cfl, smallr=1e-10, smallc=1e-10):
    U = np.ascontiguousarray(U, dtype=np.float64)
    n = round(U.shape[1] ** (1.0 / 3.0))
    return float(lib().orc_uniform_cfl_dt(n, _ptr(U), gamma, cfl, smallr, smallc))


def step_1d(U, gamma, dt, smallr=1e-10, smallc=1e-10):
    """One step of the 1-D restriction of the scheme; U is [5][n], periodic."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    rc = lib().orc_1d_step(U.shape[1], _ptr(U), gamma, dt, smallr, smallc)
    if rc:
        raise OracleError(rc, "1d_step")
    return U


def mg_solve(rho, dx, fourpiG=1.0, ncycles=4, nu1=2, nu2=2, phi0=None):
    """Multigrid V-cycles (Sec. 5) for (Laplacian phi) = fourpiG (rho - mean)
    on a periodic n^3 grid.  rho is an (n, n, n) array indexed [x, y, z].
    Returns (phi [x, y, z] with zero mean, residual L2 norm after each cycle)."""
    rho = np.asarray(rho, dtype=np.float64)
    n = rho.shape[0]
    assert rho.shape == (n, n, n)
    r = np.ascontiguousarray(rho.ravel(order="F"))
    phi = np.zeros(n ** 3) if phi0 is None else np.ascontiguousarray(
        np.asarray(phi0, dtype=np.float64).ravel(order="F"))
    res = np.zeros(max(ncycles, 1))
    rc = lib().orc_mg_solve(n, float(dx), _ptr(r), float(fourpiG), int(ncycles), int(nu1),
                            int(nu2), _ptr(phi), _ptr(res))
    if rc:
        raise OracleError(rc, "mg_solve")
    return phi.reshape((n, n, n), order="F"), res[:ncycles]


def mg_residual(rho, dx, phi, fourpiG=1.0):
    rho = np.asarray(rho, dtype=np.float64)
    n = rho.shape[0]
    r = np.ascontiguousarray(rho.ravel(order="F"))
    p = np.ascontiguousarray(np.asarray(phi, dtype=np.float64).ravel(order="F"))
    return float(lib().orc_mg_residual(n, float(dx), _ptr(r), float(fourpiG), _ptr(p)))


def cic_deposit(n, x, y, z, m):
    """Cloud-in-cell density (Sec. 4) of particles on an n^3 periodic grid,
    returned as an (n, n, n) array indexed [i, j, k]."""
    x, y, z, m = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z, m))
    rho = np.zeros(n ** 3)
    rc = lib().orc_cic_deposit(int(n), int(x.shape[0]), _ptr(x), _ptr(y), _ptr(z), _ptr(m),
                               _ptr(rho))
    if rc:
        raise OracleError(rc, "cic_deposit")
    return rho.reshape((n, n, n), order="F")
