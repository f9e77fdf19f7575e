"""Python binding of the C ABI in ``include/amr.h`` (argument marshalling only).

Every step of the mesh build, index and level step runs in the CUDA kernels
of ``_build/libamr.so``.  There is no CPU fallback: if the library has not
been built (``python -m paper_2607_20704_gb300.build`` or
``__graft_entry__.build()``) or no GPU is visible, loading raises.

PyTorch provides the stream the library runs on and, by default, its device
memory (through the caching allocator, handed to the library as a callback).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from .build import LIB

NV = 5

AMR_OK, AMR_EINVAL, AMR_ENOMEM, AMR_EGRADING, AMR_EDUP, AMR_ECUDA, AMR_ETIMEOUT, AMR_ENAN = range(8)
STATUS = {0: "AMR_OK", 1: "AMR_EINVAL", 2: "AMR_ENOMEM", 3: "AMR_EGRADING", 4: "AMR_EDUP",
          5: "AMR_ECUDA", 6: "AMR_ETIMEOUT", 7: "AMR_ENAN"}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class amr_params(C.Structure):
    _fields_ = [("levelmin", C.c_int), ("levelmax", C.c_int),
                ("gamma", C.c_double), ("cfl", C.c_double),
                ("smallr", C.c_double), ("smallc", C.c_double),
                ("refine_grad_rho", C.c_double), ("refine_grad_p", C.c_double),
                ("refine_mass", C.c_double),
                ("precision", C.c_int), ("reflux", C.c_int),
                ("reindex_every_step", C.c_int), ("use_graphs", C.c_int),
                ("hbm_budget_bytes", C.c_size_t), ("stream", C.c_void_p),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p),
                ("tile", C.c_int), ("schedule", C.c_int),
                ("regrid_expand", C.c_int), ("regrid_every_step", C.c_int),
                ("nsubgrid", C.c_int), ("planar", C.c_int)]


class amr_info(C.Structure):
    _fields_ = [("n_oct", C.c_int64), ("n_cache", C.c_int64), ("n_leaf_cells", C.c_int64),
                ("level_octs", C.c_int64 * 16), ("level_cache", C.c_int64 * 16),
                ("level_leaf_cells", C.c_int64 * 16),
                ("device_bytes", C.c_int64), ("kernel_launches", C.c_int64),
                ("graph_launches", C.c_int64), ("hash_capacity", C.c_int64),
                ("work_per_step", C.c_int64),
                ("precision", C.c_int), ("n_members", C.c_int), ("member", C.c_int),
                ("phases", C.c_int), ("tile", C.c_int), ("schedule", C.c_int),
                ("nsubgrid", C.c_int), ("planar", C.c_int), ("cached_bytes", C.c_int64)]


class amr_member(C.Structure):
    _fields_ = [("levelmin", C.c_int), ("levelmax", C.c_int),
                ("gamma", C.c_double), ("cfl", C.c_double),
                ("smallr", C.c_double), ("smallc", C.c_double),
                ("n_oct", C.c_int64),
                ("level", C.c_void_p), ("i", C.c_void_p), ("j", C.c_void_p), ("k", C.c_void_p),
                ("hilbert_key", C.c_void_p), ("U", C.c_void_p)]


class amr_server_params(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("max_waves", C.c_int),
                ("max_wave_members", C.c_int), ("device", C.c_int), ("tile", C.c_int),
                ("schedule", C.c_int)]


class amr_request(C.Structure):
    _fields_ = [("mesh", amr_member), ("n_coarse_steps", C.c_int), ("precision", C.c_int)]


class amr_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64),
                ("failed", C.c_int64), ("queued", C.c_int64), ("running_waves", C.c_int64),
                ("latency_p50_ms", C.c_double), ("latency_p99_ms", C.c_double),
                ("latency_mean_ms", C.c_double), ("queue_p50_ms", C.c_double),
                ("cell_updates", C.c_double), ("span_s", C.c_double),
                ("device_bytes", C.c_int64)]


class AmrError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None
_lock = threading.Lock()

# exported symbols of the C ABI (checked by the CPU tests against amr.h)
SYMBOLS = ["amr_params_default", "amr_create", "amr_destroy", "amr_cfl_dt", "amr_step_level",
           "amr_advance", "amr_reindex", "amr_read", "amr_read_reflux", "amr_write",
           "amr_lookup", "amr_read_index", "amr_read_cache", "amr_fill_ghosts", "amr_get_info",
           "amr_set_timing", "amr_read_timing", "amr_kernel_name", "amr_sync", "amr_last_error",
           "amr_status_string", "amr_cfl_dt_static", "amr_create_batch", "amr_select_member",
           "amr_member_dt", "amr_set_member_steps", "amr_member_errors", "amr_regrid", "amr_flag",
           "amr_regrid_flags", "amr_totals", "amr_hash", "amr_read_hash", "amr_batch_repack",
           "amr_cic_deposit_levels", "amr_cic_deposit_levels_device", "amr_read_particle_rho",
           "amr_poisson", "amr_read_phi", "amr_poisson_level", "amr_poisson_levels", "amr_write_phi",
           "amr_read_phi_level", "amr_fma_rate", "amr_load_state_async", "amr_store_state_async",
           "amr_server_create", "amr_server_submit",
           "amr_server_wait", "amr_server_read", "amr_server_release", "amr_server_get_stats",
           "amr_server_destroy"]

# exported symbols of the particle C ABI (include/amr_particles.h)
PART_SYMBOLS = ["amr_part_create", "amr_part_write", "amr_part_sort", "amr_cic_deposit",
                "amr_part_read_rho", "amr_part_read", "amr_part_device", "amr_part_get_info",
                "amr_part_set_timing", "amr_part_read_timing", "amr_part_kernel_name",
                "amr_part_destroy"]

AMR_CIC_ATOMIC, AMR_CIC_SEGMENT = 2, 3
CIC_ALGOS = {"atomic": AMR_CIC_ATOMIC, "segment": AMR_CIC_SEGMENT}


class amr_part_params(C.Structure):
    _fields_ = [("n", C.c_int), ("precision", C.c_int), ("stream", C.c_void_p)]


class amr_part_info(C.Structure):
    _fields_ = [("np", C.c_int64), ("n", C.c_int), ("precision", C.c_int), ("sorted", C.c_int),
                ("n_segments", C.c_int64), ("device_bytes", C.c_int64),
                ("kernel_launches", C.c_int64)]


# fixed scratch limit of amr_cfl_dt_static (AMR_CFL_STATIC_MAX_CELLS in amr.h)
CFL_STATIC_MAX_CELLS = 65536 * 256


def load(path: str | None = None):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing "
                               "(run paper_2607_20704_gb300.build.build())")
        L = C.CDLL(path)
        P, I, I64, D = C.c_void_p, C.c_int, C.c_int64, C.c_double
        sig = {
            "amr_params_default": (None, [C.POINTER(amr_params)]),
            "amr_create": (I, [C.POINTER(amr_params), I64, P, P, P, P, P, P, C.POINTER(P)]),
            "amr_destroy": (I, [P]),
            "amr_cfl_dt": (I, [P, C.POINTER(D)]),
            "amr_step_level": (I, [P, I, D]),
            "amr_advance": (I, [P, I, P]),
            "amr_reindex": (I, [P]),
            "amr_read": (I, [P, I, C.POINTER(I64), P, P, I64]),
            "amr_read_reflux": (I, [P, I, P, I64]),
            "amr_write": (I, [P, I, P, I64]),
            "amr_lookup": (I, [P, I64, P, P]),
            "amr_read_index": (I, [P, I, P, P, I64]),
            "amr_read_cache": (I, [P, I, C.POINTER(I64), C.POINTER(I64), P, P, I64]),
            "amr_fill_ghosts": (I, [P, I]),
            "amr_get_info": (I, [P, C.POINTER(amr_info)]),
            "amr_set_timing": (I, [P, I]),
            "amr_read_timing": (I, [P, I, P, P]),
            "amr_kernel_name": (C.c_char_p, [I]),
            "amr_sync": (I, [P]),
            "amr_last_error": (C.c_char_p, []),
            "amr_status_string": (C.c_char_p, [I]),
            "amr_cfl_dt_static": (I, [P, I64, I64, I, D, D, D, D, P, P]),
            "amr_create_batch": (I, [C.POINTER(amr_params), I, C.POINTER(amr_member), C.POINTER(P)]),
            "amr_select_member": (I, [P, I]),
            "amr_member_dt": (I, [P, P, I]),
            "amr_set_member_steps": (I, [P, P, I]),
            "amr_member_errors": (I, [P, P, I]),
            "amr_regrid": (I, [P, P, P]),
            "amr_regrid_flags": (I, [P, P, I64, P, P]),
            "amr_totals": (I, [P, I, P]),
            "amr_batch_repack": (I, [P, I, P, I, P, P]),
            "amr_cic_deposit_levels": (I, [P, I64, P, P, P, P, P]),
            "amr_cic_deposit_levels_device": (I, [P, I64, P, P, P, P, P]),
            "amr_read_particle_rho": (I, [P, I, P, I64]),
            "amr_hash": (I, [P, I64, P, P]),
            "amr_read_hash": (I, [P, P, P, P, I64]),
            "amr_flag": (I, [P, I, P, I64]),
            "amr_poisson": (I, [P, D, I, P]),
            "amr_read_phi": (I, [P, P, I64]),
            "amr_poisson_level": (I, [P, I, D, D, I, P]),
            "amr_poisson_levels": (I, [P, D, I, P]),
            "amr_write_phi": (I, [P, I, P, I64]),
            "amr_read_phi_level": (I, [P, I, P, I64]),
            "amr_fma_rate": (I, [I, I, C.POINTER(D)]),
            "amr_server_create": (I, [C.POINTER(amr_server_params), C.POINTER(P)]),
            "amr_server_submit": (I, [P, C.POINTER(amr_request), C.POINTER(I64)]),
            "amr_server_wait": (I, [P, I64, D, C.POINTER(I)]),
            "amr_server_read": (I, [P, I64, I, C.POINTER(I64), P, P, I64]),
            "amr_server_release": (I, [P, I64]),
            "amr_server_get_stats": (I, [P, C.POINTER(amr_server_stats)]),
            "amr_server_destroy": (I, [P]),
            "amr_load_state_async": (I, [P, P, I64]),
            "amr_store_state_async": (I, [P, P, I64]),
            "amr_part_create": (I, [C.POINTER(amr_part_params), I64, P, P, P, P, C.POINTER(P)]),
            "amr_part_write": (I, [P, P, P, P, P]),
            "amr_part_sort": (I, [P]),
            "amr_cic_deposit": (I, [P, I]),
            "amr_part_read_rho": (I, [P, P, I64]),
            "amr_part_read": (I, [P, P, P, P, P, P, I64]),
            "amr_part_device": (I, [P, C.POINTER(P), C.POINTER(P), C.POINTER(P), C.POINTER(P),
                                    C.POINTER(P)]),
            "amr_part_get_info": (I, [P, C.POINTER(amr_part_info)]),
            "amr_part_set_timing": (I, [P, I]),
            "amr_part_read_timing": (I, [P, I, P, P]),
            "amr_part_kernel_name": (C.c_char_p, [I]),
            "amr_part_destroy": (I, [P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def _check(rc: int, where: str):
    if rc != AMR_OK:
        raise AmrError(rc, where, load().amr_last_error().decode())


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# -- PyTorch plumbing: streams and the caching allocator ----------------------
def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device visible: the AMR library has no CPU path")
    return torch


@ALLOC_FN
def _torch_alloc(nbytes, stream, user):
    try:
        import torch
        return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
    except Exception:
        return None


@FREE_FN
def _torch_free(ptr, nbytes, stream, user):
    try:
        import torch
        torch.cuda.caching_allocator_delete(int(ptr))
    except Exception:
        pass


def kernel_names():
    L = load()
    out = []
    t = 0
    while True:
        n = L.amr_kernel_name(t)
        if n is None:
            return out
        out.append(n.decode())
        t += 1


def _member_array(members):
    """ctypes array of amr_member for a list of member dicts, and the numpy
    arrays it points into (the caller keeps them alive during the call)."""
    keep = []
    arr = (amr_member * len(members))()
    for t, mb in enumerate(members):
        lv = np.ascontiguousarray(mb["level"], dtype=np.uint8)
        ii = np.ascontiguousarray(mb["i"], dtype=np.uint32)
        jj = np.ascontiguousarray(mb["j"], dtype=np.uint32)
        kk = np.ascontiguousarray(mb["k"], dtype=np.uint32)
        uu = np.ascontiguousarray(mb["U"], dtype=np.float64)
        n = lv.shape[0]
        if uu.shape != (NV, 8 * n):
            raise ValueError(f"U must have shape (5, {8 * n}), got {uu.shape}")
        hk = mb.get("hilbert_key")
        hk = None if hk is None else np.ascontiguousarray(hk, dtype=np.uint64)
        keep += [lv, ii, jj, kk, uu, hk]
        m = arr[t]
        m.levelmin, m.levelmax = int(mb["levelmin"]), int(mb["levelmax"])
        m.gamma, m.cfl = float(mb["gamma"]), float(mb.get("cfl", 0.8))
        m.smallr, m.smallc = float(mb.get("smallr", 1e-10)), float(mb.get("smallc", 1e-10))
        m.n_oct = n
        m.level, m.i, m.j, m.k, m.U = (_ptr(lv), _ptr(ii), _ptr(jj), _ptr(kk), _ptr(uu))
        m.hilbert_key = _ptr(hk) if hk is not None else None
    return arr, keep


def fma_rate(device: int = 0, precision: int = 8) -> float:
    """FMA throughput of the GPU in FLOP/s (2 per FMA), FP64 or FP32."""
    out = C.c_double()
    _check(load().amr_fma_rate(int(device), int(precision), C.byref(out)), "amr_fma_rate")
    return out.value


class Mesh:
    """One resident handle (wraps an ``amr_handle``): a single mesh, or with
    ``Mesh.batch`` many independent member meshes advanced together."""

    def __init__(self, level=None, i=None, j=None, k=None, U=None, *, levelmin=1, levelmax=1,
                 gamma=1.4, cfl=0.8, smallr=1e-10, smallc=1e-10, precision=8, reflux=True,
                 reindex_every_step=False, use_graphs=True, hbm_budget_bytes=0,
                 hilbert_key=None, allocator="torch", stream=None, members=None, tile=0,
                 schedule=-1, refine_grad_rho=0.0, refine_grad_p=0.0, refine_mass=0.0,
                 regrid_expand=True, regrid_every_step=False, nsubgrid=-1, planar=-1):
        torch = _torch()
        L = load()
        p = amr_params()
        L.amr_params_default(C.byref(p))
        p.levelmin, p.levelmax = int(levelmin), int(levelmax)
        p.gamma, p.cfl, p.smallr, p.smallc = float(gamma), float(cfl), float(smallr), float(smallc)
        p.precision = int(precision)
        p.reflux = int(bool(reflux))
        p.reindex_every_step = int(bool(reindex_every_step))
        p.use_graphs = int(bool(use_graphs))
        p.hbm_budget_bytes = int(hbm_budget_bytes)
        p.tile, p.schedule = int(tile), int(schedule)
        p.refine_grad_rho, p.refine_grad_p = float(refine_grad_rho), float(refine_grad_p)
        p.refine_mass = float(refine_mass)
        p.regrid_expand = int(bool(regrid_expand))
        p.regrid_every_step = int(bool(regrid_every_step))
        p.nsubgrid = int(nsubgrid)
        p.planar = int(planar)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        p.stream = C.c_void_p(self.stream.cuda_stream)
        if allocator == "torch":
            p.alloc, p.free = _torch_alloc, _torch_free
        self.params = p
        if members is None:
            members = [dict(level=level, i=i, j=j, k=k, U=U, levelmin=levelmin, levelmax=levelmax,
                            gamma=gamma, cfl=cfl, smallr=smallr, smallc=smallc,
                            hilbert_key=hilbert_key)]
        arr, keep = _member_array(members)
        h = C.c_void_p()
        rc = L.amr_create_batch(C.byref(p), len(members), arr, C.byref(h))
        _check(rc, "amr_create")
        self._h = h
        self.n_members = len(members)
        self.member_levels = [(int(mb["levelmin"]), int(mb["levelmax"])) for mb in members]
        self.levelmin, self.levelmax = self.member_levels[0]
        self.gamma = float(members[0]["gamma"])
        self.precision = int(precision)
        self._member = 0

    def repack(self, keep, problems=(), steps=()):
        """Continuous batching: keep the members listed in ``keep`` (increasing
        order; their states stay on the device) and append the meshes of
        ``problems`` (``inputs.Problem``), each taking ``steps[q]`` coarse
        steps (-1: unlimited)."""
        kp = np.ascontiguousarray(keep, dtype=np.int32)
        members = []
        for pr in problems:
            lv, i, j, k, U = pr.mesh_args()
            members.append(dict(level=lv, i=i, j=j, k=k, U=U, **pr.params()))
        arr, hold = _member_array(members) if members else (None, [])
        st = np.ascontiguousarray(steps, dtype=np.int32)
        assert st.size == len(members)
        _check(load().amr_batch_repack(self._h, int(kp.size), _ptr(kp) if kp.size else None,
                                       len(members), arr, _ptr(st) if st.size else None),
               "amr_batch_repack")
        del hold
        self.member_levels = [self.member_levels[int(q)] for q in kp] + \
            [(int(mb["levelmin"]), int(mb["levelmax"])) for mb in members]
        self.n_members = len(self.member_levels)
        self._member = 0
        self.levelmin, self.levelmax = self.member_levels[0]

    @classmethod
    def batch(cls, problems, **kw):
        """A handle over several ``inputs.Problem`` meshes (one member each)."""
        members = []
        for pr in problems:
            lv, i, j, k, U = pr.mesh_args()
            members.append(dict(level=lv, i=i, j=j, k=k, U=U, **pr.params()))
        return cls(members=members, **kw)

    def select(self, member: int):
        """Member that read/write/lookup/index calls refer to."""
        _check(load().amr_select_member(self._h, int(member)), "amr_select_member")
        self._member = int(member)
        self.levelmin, self.levelmax = self.member_levels[int(member)]
        return self

    def set_member_steps(self, steps):
        """Coarse steps each member still takes (-1: unlimited)."""
        st = np.ascontiguousarray(steps, dtype=np.int32)
        _check(load().amr_set_member_steps(self._h, _ptr(st), len(st)), "amr_set_member_steps")

    def regrid(self):
        """One regrid (Sec. 2.2) with the handle's criteria; returns
        (octs created, octs removed)."""
        cr, rm = C.c_int64(), C.c_int64()
        _check(load().amr_regrid(self._h, C.byref(cr), C.byref(rm)), "amr_regrid")
        return cr.value, rm.value

    def cic_deposit_levels(self, x, y, z, m):
        """CIC deposition of the particles onto every level of the selected
        member (Sec. 4); returns the size of each level's particle list."""
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z, m)]
        cnt = np.zeros(16, np.int64)
        _check(load().amr_cic_deposit_levels(self._h, int(arrs[0].size), *[_ptr(a) for a in arrs],
                                             _ptr(cnt)), "amr_cic_deposit_levels")
        return cnt

    def cic_deposit_levels_device(self, x, y, z, m, counts=True):
        """The same from device tensors of the handle's precision."""
        cnt = np.zeros(16, np.int64)
        _check(load().amr_cic_deposit_levels_device(
            self._h, int(x.numel()), C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
            C.c_void_p(z.data_ptr()), C.c_void_p(m.data_ptr()), _ptr(cnt) if counts else None),
            "amr_cic_deposit_levels_device")
        return cnt if counts else None

    def particle_rho(self, level: int):
        """Density of the last deposition at the cells of one level [8 n]."""
        n = self.num_octs(level)
        out = np.zeros(8 * max(n, 1), np.float64)
        _check(load().amr_read_particle_rho(self._h, int(level), _ptr(out), max(n, 1)),
               "amr_read_particle_rho")
        return out[:8 * n]

    def totals(self, level: int = 0):
        """FP64 totals of the leaf cells' U dx^3 (one level, or 0: all levels),
        computed on the device in a fixed order."""
        out = np.zeros(5, np.float64)
        _check(load().amr_totals(self._h, int(level), _ptr(out)), "amr_totals")
        return out

    def hash(self, keys):
        """FNV-1a 64 of each 64-bit value, evaluated by the device function
        the hash table uses."""
        k = np.ascontiguousarray(keys, dtype=np.uint64)
        out = np.zeros(max(k.size, 1), np.uint64)
        _check(load().amr_hash(self._h, int(k.size), _ptr(k), _ptr(out)), "amr_hash")
        return out[:k.size]

    def read_hash(self):
        """The hash table as stored: (internal keys [cap], values [cap])."""
        cap = C.c_int64()
        L = load()
        _check(L.amr_read_hash(self._h, C.byref(cap), None, None, 0), "amr_read_hash")
        keys = np.zeros(cap.value, np.uint64)
        vals = np.zeros(cap.value, np.int32)
        _check(L.amr_read_hash(self._h, C.byref(cap), _ptr(keys), _ptr(vals), cap.value),
               "amr_read_hash")
        return keys, vals

    def regrid_flags(self, flags):
        """Regrid with the given final flags: one byte per cell of the whole
        handle in mesh order (levels ascending, amr_read order within a
        level); returns (octs created, octs removed)."""
        f = np.ascontiguousarray(flags, dtype=np.uint8)
        cr, rm = C.c_int64(), C.c_int64()
        _check(load().amr_regrid_flags(self._h, _ptr(f), int(f.size), C.byref(cr), C.byref(rm)),
               "amr_regrid_flags")
        return cr.value, rm.value

    def flags(self, level: int):
        """Refinement flags [8 n_level] of the selected member's level."""
        n = self.num_octs(level)
        out = np.zeros(8 * max(n, 1), np.uint8)
        _check(load().amr_flag(self._h, int(level), _ptr(out), 8 * max(n, 1)), "amr_flag")
        return out[:8 * n]

    def poisson(self, fourpiG: float = 1.0, n_vcycles: int = 4, residuals: bool = True):
        """Multigrid V-cycles (Sec. 5) on the base level; returns the L2 norm
        of the residual after each cycle (None when residuals=False, which
        skips computing them)."""
        if not residuals:
            _check(load().amr_poisson(self._h, float(fourpiG), int(n_vcycles), None), "amr_poisson")
            return None
        res = np.zeros(max(int(n_vcycles), 1), np.float64)
        _check(load().amr_poisson(self._h, float(fourpiG), int(n_vcycles), _ptr(res)), "amr_poisson")
        return res[:int(n_vcycles)]

    def read_phi(self):
        """Potential of the base-level cells, [8 n] in read order."""
        n = self.num_octs(self.levelmin)
        out = np.zeros(8 * max(n, 1), np.float64)
        _check(load().amr_read_phi(self._h, _ptr(out), 8 * max(n, 1)), "amr_read_phi")
        return out[:8 * n]

    def poisson_level(self, level: int, fourpiG: float = 1.0, rho_bar: float = 1.0, n_vcycles: int = 4,
                      residuals: bool = True):
        """V-cycles (Sec. 5) on refined level `level`: the Dirichlet data are
        the per-cell potential of level-1, the initial guess that of the
        level, which receives the result; returns the residual norms."""
        res = np.zeros(max(int(n_vcycles), 1), np.float64)
        _check(load().amr_poisson_level(self._h, int(level), float(fourpiG), float(rho_bar), int(n_vcycles),
                                        _ptr(res) if residuals else None), "amr_poisson_level")
        return res[:int(n_vcycles)] if residuals else None

    def poisson_levels(self, fourpiG: float = 1.0, n_vcycles: int = 4, residuals: bool = True):
        """The potential of every level, base level first, each refined level
        from its father cells' values; returns {level: residual norms}."""
        nv = int(n_vcycles)
        res = np.zeros(max((self.levelmax + 1) * nv, 1), np.float64)
        _check(load().amr_poisson_levels(self._h, float(fourpiG), nv, _ptr(res) if residuals else None),
               "amr_poisson_levels")
        if not residuals:
            return None
        return {l: res[l * nv:(l + 1) * nv] for l in range(self.levelmin, self.levelmax + 1)
                if self.num_octs(l) > 0}

    def write_phi(self, level: int, phi):
        """Per-cell potential of one level, [8 n] in read order."""
        a = np.ascontiguousarray(phi, dtype=np.float64)
        _check(load().amr_write_phi(self._h, int(level), _ptr(a), a.size), "amr_write_phi")

    def read_phi_level(self, level: int):
        """Per-cell potential of one level, [8 n] in read order."""
        n = self.num_octs(level)
        out = np.zeros(8 * max(n, 1), np.float64)
        _check(load().amr_read_phi_level(self._h, int(level), _ptr(out), 8 * max(n, 1)), "amr_read_phi_level")
        return out[:8 * n]

    def member_errors(self):
        """Per-member flags (1: a leaf state was not finite); clears the
        handle-wide error the next synchronising call would otherwise report."""
        out = np.zeros(self.n_members, np.int32)
        _check(load().amr_member_errors(self._h, _ptr(out), self.n_members), "amr_member_errors")
        return out

    def member_dt(self):
        out = np.zeros(self.n_members, np.float64)
        _check(load().amr_member_dt(self._h, _ptr(out), self.n_members), "amr_member_dt")
        return out

    # -- lifetime ----------------------------------------------------------------
    def close(self):
        h = getattr(self, "_h", None)
        if h:
            load().amr_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    # -- stepping ------------------------------------------------------------------
    def cfl_dt(self) -> float:
        dt = C.c_double()
        _check(load().amr_cfl_dt(self._h, C.byref(dt)), "amr_cfl_dt")
        return dt.value

    def step_level(self, level: int, dt: float):
        _check(load().amr_step_level(self._h, int(level), float(dt)), "amr_step_level")

    def advance(self, n: int = 1, sync: bool = False):
        if sync:
            dt = C.c_double()
            _check(load().amr_advance(self._h, int(n), C.byref(dt)), "amr_advance")
            return dt.value
        _check(load().amr_advance(self._h, int(n), None), "amr_advance")
        return None

    def reindex(self):
        _check(load().amr_reindex(self._h), "amr_reindex")

    def fill_ghosts(self, level: int):
        _check(load().amr_fill_ghosts(self._h, int(level)), "amr_fill_ghosts")

    def sync(self):
        _check(load().amr_sync(self._h), "amr_sync")
        self._keep = []

    # -- state -----------------------------------------------------------------------
    def num_octs(self, level: int) -> int:
        n = C.c_int64()
        _check(load().amr_read(self._h, int(level), C.byref(n), None, None, 0), "amr_read")
        return n.value

    def read(self, level: int, out_U=None, keys=True):
        n = self.num_octs(level)
        kk = np.zeros(max(n, 1), np.uint64) if keys else None
        U = out_U if out_U is not None else np.zeros((NV, 8 * max(n, 1)), np.float64)
        cnt = C.c_int64()
        _check(load().amr_read(self._h, int(level), C.byref(cnt), _ptr(kk), _ptr(U), max(n, 1)),
               "amr_read")
        return (kk[:n] if keys else None), U[:, :8 * n]

    def read_reflux(self, level: int):
        n = self.num_octs(level)
        R = np.zeros((NV, 8 * max(n, 1)), np.float64)
        _check(load().amr_read_reflux(self._h, int(level), _ptr(R), max(n, 1)), "amr_read_reflux")
        return R[:, :8 * n]

    def load_state_async(self, U):
        """Queue the whole state (all levels, mesh order, [5][8 n] doubles)
        as the input of the work queued next; returns at once.  U must stay
        untouched until sync() (pinned memory overlaps the copy)."""
        U = np.asarray(U)
        if U.dtype != np.float64 or not U.flags.c_contiguous or U.ndim != 2 or U.shape[0] != NV:
            raise ValueError("U must be a C-contiguous float64 array of shape (5, 8 n)")
        self._keep = getattr(self, "_keep", [])
        self._keep.append(U)
        _check(load().amr_load_state_async(self._h, _ptr(U), U.shape[1] // 8), "amr_load_state_async")

    def store_state_async(self, out):
        """Queue a copy of the whole state after the work queued so far into
        `out` ((5, 8 n) float64); complete after sync()."""
        if out.dtype != np.float64 or not out.flags.c_contiguous or out.ndim != 2 or out.shape[0] != NV:
            raise ValueError("out must be a C-contiguous float64 array of shape (5, 8 n)")
        self._keep = getattr(self, "_keep", [])
        self._keep.append(out)
        _check(load().amr_store_state_async(self._h, _ptr(out), out.shape[1] // 8),
               "amr_store_state_async")
        return out

    def state_octs(self) -> int:
        """Octs of the selected member, all levels."""
        return int(sum(self.num_octs(l) for l in self.levels()))

    def write(self, level: int, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        n = U.shape[1] // 8
        _check(load().amr_write(self._h, int(level), _ptr(U), n), "amr_write")

    # -- index introspection ---------------------------------------------------------
    def lookup(self, keys):
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        out = np.zeros(max(len(keys), 1), np.int64)
        _check(load().amr_lookup(self._h, len(keys), _ptr(keys), _ptr(out)), "amr_lookup")
        return out[:len(keys)]

    def read_index(self, level: int):
        n = self.num_octs(level)
        nb = np.zeros((max(n, 1), 27), np.int64)
        sp = np.zeros(8 * max(n, 1), np.uint8)
        _check(load().amr_read_index(self._h, int(level), _ptr(nb), _ptr(sp), max(n, 1)),
               "amr_read_index")
        return nb[:n], sp[:8 * n]

    def read_cache(self, level: int):
        n, first = C.c_int64(), C.c_int64()
        L = load()
        _check(L.amr_read_cache(self._h, int(level), C.byref(n), C.byref(first), None, None, 0),
               "amr_read_cache")
        nc = n.value
        keys = np.zeros(max(nc, 1), np.uint64)
        Ug = np.zeros((NV, 8 * max(nc, 1)), np.float64)
        _check(L.amr_read_cache(self._h, int(level), C.byref(n), C.byref(first), _ptr(keys),
                                _ptr(Ug), max(nc, 1)), "amr_read_cache")
        return keys[:nc], Ug[:, :8 * nc], first.value

    def info(self) -> dict:
        inf = amr_info()
        _check(load().amr_get_info(self._h, C.byref(inf)), "amr_get_info")
        return {
            "n_oct": inf.n_oct, "n_cache": inf.n_cache, "n_leaf_cells": inf.n_leaf_cells,
            "level_octs": list(inf.level_octs), "level_cache": list(inf.level_cache),
            "level_leaf_cells": list(inf.level_leaf_cells), "device_bytes": inf.device_bytes,
            "kernel_launches": inf.kernel_launches, "graph_launches": inf.graph_launches,
            "hash_capacity": inf.hash_capacity, "precision": inf.precision,
            "work_per_step": inf.work_per_step, "n_members": inf.n_members,
            "member": inf.member, "phases": inf.phases, "tile": inf.tile,
            "schedule": inf.schedule, "nsubgrid": inf.nsubgrid, "planar": inf.planar,
            "cached_bytes": inf.cached_bytes,
        }

    def set_timing(self, on: bool):
        _check(load().amr_set_timing(self._h, int(bool(on))), "amr_set_timing")

    def read_timing(self) -> dict:
        names = kernel_names()
        ms = np.zeros(len(names), np.float64)
        n = np.zeros(len(names), np.int64)
        _check(load().amr_read_timing(self._h, len(names), _ptr(ms), _ptr(n)), "amr_read_timing")
        return {nm: (float(ms[t]), int(n[t])) for t, nm in enumerate(names) if n[t]}

    def levels(self):
        return [l for l in range(self.levelmin, self.levelmax + 1) if self.num_octs(l) > 0]


# -- the C names, one thin wrapper each ---------------------------------------------
def amr_create(prob_or_args, **kw) -> Mesh:
    """``amr_create`` from an ``inputs.Problem`` or a (level, i, j, k, U) tuple."""
    if hasattr(prob_or_args, "mesh_args"):
        args = prob_or_args.mesh_args()
        params = dict(prob_or_args.params())
        params.update(kw)
        return Mesh(*args, **params)
    return Mesh(*prob_or_args, **kw)


def amr_destroy(m: Mesh):
    m.close()


def amr_cfl_dt(m: Mesh) -> float:
    return m.cfl_dt()


def amr_step_level(m: Mesh, level: int, dt: float):
    m.step_level(level, dt)


def amr_advance(m: Mesh, n: int = 1, sync: bool = False):
    return m.advance(n, sync=sync)


def amr_read(m: Mesh, level: int):
    return m.read(level)


def amr_write(m: Mesh, level: int, U):
    m.write(level, U)


def amr_cfl_dt_static(U_ptr: int, n_cells: int, stride: int, level: int, gamma: float,
                      cfl: float, smallr: float, smallc: float, dt_out_ptr: int,
                      stream_ptr: int = 0):
    """Time-step reduction on caller-owned device buffers, allocating nothing
    on the device (for callers that cannot allocate: see include/amr.h).
    U_ptr and dt_out_ptr are device addresses; asynchronous on stream_ptr."""
    L = load()
    _check(L.amr_cfl_dt_static(C.c_void_p(U_ptr), int(n_cells), int(stride), int(level),
                               float(gamma), float(cfl), float(smallr), float(smallc),
                               C.c_void_p(dt_out_ptr), C.c_void_p(stream_ptr or None)),
           "amr_cfl_dt_static")


class Server:
    """Continuous-batching serving loop (wraps ``amr_server_t``)."""

    def __init__(self, hbm_budget_bytes=0, max_waves=0, max_wave_members=0, device=-1,
                 tile=0, schedule=0):
        _torch()
        L = load()
        p = amr_server_params(int(hbm_budget_bytes), int(max_waves), int(max_wave_members),
                              int(device), int(tile), int(schedule))
        h = C.c_void_p()
        _check(L.amr_server_create(C.byref(p), C.byref(h)), "amr_server_create")
        self._h = h
        self._levels = {}

    def submit(self, prob, steps: int, precision: int = 8) -> int:
        """Queue one solve of an ``inputs.Problem`` (its arrays are copied)."""
        lv = np.ascontiguousarray(prob.level, dtype=np.uint8)
        ii = np.ascontiguousarray(prob.i, dtype=np.uint32)
        jj = np.ascontiguousarray(prob.j, dtype=np.uint32)
        kk = np.ascontiguousarray(prob.k, dtype=np.uint32)
        uu = np.ascontiguousarray(prob.U, dtype=np.float64)
        r = amr_request()
        m = r.mesh
        m.levelmin, m.levelmax = int(prob.levelmin), int(prob.levelmax)
        m.gamma, m.cfl, m.smallr, m.smallc = float(prob.gamma), float(prob.cfl), 1e-10, 1e-10
        m.n_oct = lv.shape[0]
        m.level, m.i, m.j, m.k, m.U = _ptr(lv), _ptr(ii), _ptr(jj), _ptr(kk), _ptr(uu)
        m.hilbert_key = None
        r.n_coarse_steps, r.precision = int(steps), int(precision)
        rid = C.c_int64()
        _check(load().amr_server_submit(self._h, C.byref(r), C.byref(rid)), "amr_server_submit")
        self._levels[rid.value] = (int(prob.levelmin), int(prob.levelmax))
        return rid.value

    def wait(self, rid: int = -1, timeout: float = -1.0) -> bool:
        done = C.c_int()
        _check(load().amr_server_wait(self._h, int(rid), float(timeout), C.byref(done)), "amr_server_wait")
        return bool(done.value)

    def read(self, rid: int, level: int):
        L = load()
        n = C.c_int64()
        _check(L.amr_server_read(self._h, int(rid), int(level), C.byref(n), None, None, 0), "amr_server_read")
        keys = np.zeros(max(n.value, 1), np.uint64)
        U = np.zeros((NV, 8 * max(n.value, 1)), np.float64)
        _check(L.amr_server_read(self._h, int(rid), int(level), C.byref(n), _ptr(keys), _ptr(U),
                                 max(n.value, 1)), "amr_server_read")
        return keys[:n.value], U[:, :8 * n.value]

    def release(self, rid: int):
        _check(load().amr_server_release(self._h, int(rid)), "amr_server_release")

    def stats(self) -> dict:
        st = amr_server_stats()
        _check(load().amr_server_get_stats(self._h, C.byref(st)), "amr_server_get_stats")
        return {f: getattr(st, f) for f, _ in amr_server_stats._fields_}

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            load().amr_server_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def part_kernel_names():
    L = load()
    out = []
    while True:
        n = L.amr_part_kernel_name(len(out))
        if n is None:
            return out
        out.append(n.decode())


class Particles:
    """Particles resident on the device with a periodic n^3 grid (wraps an
    ``amr_part_handle``): the source-cell Hilbert sort and the Cloud-in-Cell
    mass deposition of Sec. 4."""

    def __init__(self, n, x, y, z, m, *, precision=8, stream=None):
        torch = _torch()
        L = load()
        x, y, z, m = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z, m))
        if not (x.shape == y.shape == z.shape == m.shape and x.ndim == 1):
            raise ValueError("x, y, z, m must be 1-D arrays of one length")
        p = amr_part_params()
        p.n, p.precision = int(n), int(precision)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        p.stream = C.c_void_p(self.stream.cuda_stream)
        h = C.c_void_p()
        _check(L.amr_part_create(C.byref(p), x.shape[0], _ptr(x), _ptr(y), _ptr(z), _ptr(m),
                                 C.byref(h)), "amr_part_create")
        self._h = h
        self.n, self.np, self.precision = int(n), int(x.shape[0]), int(precision)

    def write(self, x, y, z, m):
        x, y, z, m = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z, m))
        if any(a.shape != (self.np,) for a in (x, y, z, m)):
            raise ValueError(f"arrays must have shape ({self.np},)")
        _check(load().amr_part_write(self._h, _ptr(x), _ptr(y), _ptr(z), _ptr(m)), "amr_part_write")

    def sort(self):
        _check(load().amr_part_sort(self._h), "amr_part_sort")

    def deposit(self, algo="atomic"):
        _check(load().amr_cic_deposit(self._h, CIC_ALGOS.get(algo, algo)), "amr_cic_deposit")

    def rho(self) -> np.ndarray:
        """The grid as an (n, n, n) array indexed [i, j, k]."""
        out = np.empty(self.n ** 3)
        _check(load().amr_part_read_rho(self._h, _ptr(out), out.shape[0]), "amr_part_read_rho")
        return out.reshape((self.n,) * 3, order="F")

    def rho_device(self):
        """The grid as a flat torch tensor on the device (cell i + n (j + n k);
        the handle's precision), viewing the handle's memory without a copy.
        The caller's current stream is ordered after the handle's work; the
        view is valid until the next deposit or close()."""
        torch = _torch()

        class _View:
            pass

        v = _View()
        v.__cuda_array_interface__ = {"shape": (self.n ** 3,), "typestr": "<f8" if self.precision == 8 else "<f4",
                                      "data": (self.device()["rho"], False), "version": 2}
        torch.cuda.current_stream().wait_stream(self.stream)
        return torch.as_tensor(v, device="cuda")

    def read(self):
        """Positions, masses and identifiers in the handle's current order."""
        x, y, z, m = (np.empty(self.np) for _ in range(4))
        ids = np.empty(self.np, np.int64)
        _check(load().amr_part_read(self._h, _ptr(x), _ptr(y), _ptr(z), _ptr(m), _ptr(ids),
                                    self.np), "amr_part_read")
        return x, y, z, m, ids

    def device(self) -> dict:
        ptrs = [C.c_void_p() for _ in range(5)]
        _check(load().amr_part_device(self._h, *[C.byref(q) for q in ptrs]), "amr_part_device")
        return dict(zip(("rho", "x", "y", "z", "m"), (q.value for q in ptrs)))

    def info(self) -> dict:
        inf = amr_part_info()
        _check(load().amr_part_get_info(self._h, C.byref(inf)), "amr_part_get_info")
        return {f: getattr(inf, f) for f, _ in amr_part_info._fields_}

    def set_timing(self, on=True):
        _check(load().amr_part_set_timing(self._h, int(bool(on))), "amr_part_set_timing")

    def read_timing(self) -> dict:
        names = part_kernel_names()
        ms = np.zeros(len(names))
        n = np.zeros(len(names), np.int64)
        _check(load().amr_part_read_timing(self._h, len(names), _ptr(ms), _ptr(n)),
               "amr_part_read_timing")
        return {nm: (float(ms[t]), int(n[t])) for t, nm in enumerate(names) if n[t]}

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            load().amr_part_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
