"""CPU checks of the boundary: the C-ABI library loads without a GPU and
exports every function that include/amr.h declares; host-side argument
validation answers without touching a device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2607_20704_gb300 import amr, build
    build.build()
    return amr.load()


def _declared(header="amr.h"):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(amr_[a-z_]+)\s*\(", text))
    return sorted(n for n in names if not n.endswith("_fn"))


def test_every_declared_symbol_is_exported(lib):
    from paper_2607_20704_gb300 import amr
    declared = _declared()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(amr.SYMBOLS) == declared
    part = [n for n in _declared("amr_particles.h") if n not in declared]
    for name in part:
        assert hasattr(lib, name), name
    assert sorted(amr.PART_SYMBOLS) == part


def test_status_strings_and_kernel_names(lib):
    from paper_2607_20704_gb300 import amr
    for code, name in amr.STATUS.items():
        assert lib.amr_status_string(code).decode() == name
    names = amr.kernel_names()
    for k in ("prolong", "predict", "flux", "update", "reflux_restrict", "cfl", "neighbours"):
        assert k in names


def test_params_default(lib):
    from paper_2607_20704_gb300 import amr
    p = amr.amr_params()
    lib.amr_params_default(C.byref(p))
    assert (p.precision, p.reflux, p.reindex_every_step, p.use_graphs) == (8, 1, 0, 1)
    assert p.gamma == 1.4 and p.cfl == 0.8 and p.smallr == 1e-10
    assert p.stream is None and p.hbm_budget_bytes == 0


@pytest.mark.parametrize("field,value", [("levelmin", 0), ("levelmax", 16), ("gamma", 1.0),
                                         ("precision", 2), ("cfl", 0.0)])
def test_create_rejects_bad_parameters_on_the_host(lib, field, value):
    from paper_2607_20704_gb300 import amr
    import numpy as np
    p = amr.amr_params()
    lib.amr_params_default(C.byref(p))
    setattr(p, field, value)
    one = np.zeros(1, np.uint8) + 1
    z = np.zeros(1, np.uint32)
    U = np.ones((5, 8))
    h = C.c_void_p()
    rc = lib.amr_create(C.byref(p), 1, one.ctypes.data, z.ctypes.data, z.ctypes.data,
                        z.ctypes.data, None, U.ctypes.data, C.byref(h))
    assert rc == amr.AMR_EINVAL
    assert lib.amr_last_error().decode()
    assert not h.value


def test_null_handle_calls_fail_cleanly(lib):
    from paper_2607_20704_gb300 import amr
    dt = C.c_double()
    assert lib.amr_cfl_dt(None, C.byref(dt)) == amr.AMR_EINVAL
    assert lib.amr_step_level(None, 3, 0.1) == amr.AMR_EINVAL
    assert lib.amr_advance(None, 1, None) == amr.AMR_EINVAL
    assert lib.amr_destroy(None) == amr.AMR_OK


HANDLES = ("amr_handle", "amr_server_t", "amr_part_handle")


def _handle_entry_points():
    """(name, parameter types) of every call in the headers that takes a
    handle (mesh, server or particle set) first, read from the header text."""
    out = []
    for header in ("amr.h", "amr_particles.h"):
        text = open(os.path.join(ROOT, "include", header)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for name, args in re.findall(r"\bamr_status\s+(amr_\w+)\s*\(([^;{]*?)\)\s*;", text, re.S):
            params = [" ".join(p.split()) for p in args.split(",")]
            if not params[0].split()[0] in HANDLES:
                continue
            out.append((name, [p if p.endswith("*") or "*" in p.split()[-1] else re.sub(r"\s*\b\w+$", "", p)
                               for p in params[1:]]))
    return out


def test_every_handle_call_refuses_a_null_handle(lib):
    """Every call that takes a handle returns AMR_EINVAL for NULL (the destroy
    calls: AMR_OK) before it touches any other argument or the device."""
    from paper_2607_20704_gb300 import amr
    scalar = {"int": C.c_int, "int64_t": C.c_int64, "double": C.c_double}
    calls = _handle_entry_points()
    assert len(calls) >= 50
    own = C.CDLL(amr.LIB)  # prototypes set here stay off the binding's functions
    own.amr_last_error.restype = C.c_char_p
    for name, params in calls:
        fn = getattr(own, name)
        types = [C.c_void_p] + [C.c_void_p if "*" in t else scalar[t] for t in params]
        fn.argtypes = types
        fn.restype = C.c_int
        args = [None] + [None if t is C.c_void_p else t(0) for t in types[1:]]
        want = amr.AMR_OK if name.endswith("_destroy") else amr.AMR_EINVAL
        assert fn(*args) == want, name
        if want == amr.AMR_EINVAL:
            assert own.amr_last_error().decode(), name


def test_particle_calls_check_their_arguments_on_the_host(lib):
    from paper_2607_20704_gb300 import amr
    import numpy as np
    h = C.c_void_p()
    x = np.array([0.25, 0.5])
    m = np.ones(2)
    for n, prec in ((3, 8), (0, 8), (2048, 8), (16, 2)):
        p = amr.amr_part_params(n, prec, None)
        assert lib.amr_part_create(C.byref(p), 2, x.ctypes.data, x.ctypes.data, x.ctypes.data,
                                   m.ctypes.data, C.byref(h)) == amr.AMR_EINVAL
        assert not h.value
    p = amr.amr_part_params(16, 8, None)
    for bad in (np.array([0.25, 1.0]), np.array([-0.1, 0.5]), np.array([0.25, np.nan])):
        assert lib.amr_part_create(C.byref(p), 2, bad.ctypes.data, x.ctypes.data, x.ctypes.data,
                                   m.ctypes.data, C.byref(h)) == amr.AMR_EINVAL
        assert "outside" in lib.amr_last_error().decode()
    inf = np.array([1.0, np.inf])
    assert lib.amr_part_create(C.byref(p), 2, x.ctypes.data, x.ctypes.data, x.ctypes.data,
                               inf.ctypes.data, C.byref(h)) == amr.AMR_EINVAL
    assert lib.amr_part_sort(None) == amr.AMR_EINVAL
    assert lib.amr_cic_deposit(None, 2) == amr.AMR_EINVAL
    assert lib.amr_part_destroy(None) == amr.AMR_OK
    names = amr.part_kernel_names()
    for k in ("part_keys", "psort_scatter", "cic_atomic", "seg_partial", "seg_gather"):
        assert k in names


def test_create_refuses_oversize_meshes_on_the_host(lib):
    """More than 2^26 octs (one mesh, or the members of a batch together) is
    refused before any device work: the arrays are never read, no stream or
    allocation is made (this runs without a GPU).  Below that limit the
    kernels form every product with a scratch stride in 64 bits (20 x the
    local cells of a level exceeds 2^31 from about 107 M cells on)."""
    from paper_2607_20704_gb300 import amr
    import numpy as np
    p = amr.amr_params()
    lib.amr_params_default(C.byref(p))
    one = np.ones(1, np.uint8)
    z = np.zeros(1, np.uint32)
    U = np.ones((5, 8))
    h = C.c_void_p()
    rc = lib.amr_create(C.byref(p), (1 << 26) + 1, one.ctypes.data, z.ctypes.data, z.ctypes.data,
                        z.ctypes.data, None, U.ctypes.data, C.byref(h))
    assert rc == amr.AMR_EINVAL and not h.value
    assert "2^26" in lib.amr_last_error().decode()
    members = (amr.amr_member * 2)()
    for q in range(2):
        m = members[q]
        m.levelmin, m.levelmax, m.gamma, m.cfl = 3, 4, 1.4, 0.8
        m.smallr = m.smallc = 1e-10
        m.n_oct = (1 << 25) + 1
        m.level, m.i, m.j, m.k = one.ctypes.data, z.ctypes.data, z.ctypes.data, z.ctypes.data
        m.U = U.ctypes.data
    rc = lib.amr_create_batch(C.byref(p), 2, members, C.byref(h))
    assert rc == amr.AMR_EINVAL and not h.value
    assert "2^26" in lib.amr_last_error().decode()


def test_static_cfl_refuses_bad_arguments_on_the_host(lib):
    """amr_cfl_dt_static checks its pointers, sizes and parameters before any
    CUDA call (the device pointers given here are never dereferenced: every
    case is refused first)."""
    from paper_2607_20704_gb300 import amr
    own = C.CDLL(amr.LIB)
    fn = own.amr_cfl_dt_static
    fn.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_int, C.c_double, C.c_double, C.c_double,
                   C.c_double, C.c_void_p, C.c_void_p]
    fn.restype = C.c_int
    own.amr_last_error.restype = C.c_char_p
    fake = 0x1000  # stands for a device address; none of the cases below reaches it
    good = dict(U=fake, n=1024, stride=1024, level=5, gamma=1.4, cfl=0.8, smallr=1e-10, smallc=1e-10,
                dt=fake)
    cases = [dict(U=None), dict(dt=None), dict(n=0), dict(n=(65536 * 256) + 1), dict(stride=1023),
             dict(level=-1), dict(level=31), dict(gamma=1.0), dict(cfl=0.0), dict(smallr=0.0),
             dict(smallc=-1.0), dict(gamma=float("nan"))]
    for bad in cases:
        a = {**good, **bad}
        rc = fn(a["U"], a["n"], a["stride"], a["level"], a["gamma"], a["cfl"], a["smallr"], a["smallc"],
                a["dt"], None)
        assert rc == amr.AMR_EINVAL, bad
        assert own.amr_last_error().decode().startswith("amr_cfl_dt_static"), bad


def test_batch_members_are_checked_on_the_host(lib):
    """A member with a NULL array, bad levels or parameters, or no octs, and
    launch parameters outside their sets, are refused before any device work
    (this runs without a GPU; the arrays are never read)."""
    from paper_2607_20704_gb300 import amr
    import numpy as np
    one = np.ones(1, np.uint8)
    z = np.zeros(1, np.uint32)
    U = np.ones((5, 8))

    def member(**kw):
        m = amr.amr_member()
        m.levelmin, m.levelmax, m.gamma, m.cfl, m.smallr, m.smallc, m.n_oct = 3, 4, 1.4, 0.8, 1e-10, 1e-10, 1
        m.level, m.i, m.j, m.k, m.U = one.ctypes.data, z.ctypes.data, z.ctypes.data, z.ctypes.data, U.ctypes.data
        for key, v in kw.items():
            setattr(m, key, v)
        return m

    bad_members = [dict(level=None), dict(i=None), dict(U=None), dict(levelmin=0), dict(levelmax=16),
                   dict(levelmin=5, levelmax=4), dict(gamma=1.0), dict(cfl=0.0), dict(smallr=0.0),
                   dict(smallc=0.0), dict(n_oct=0)]
    p = amr.amr_params()
    lib.amr_params_default(C.byref(p))
    h = C.c_void_p()
    for bad in bad_members:
        members = (amr.amr_member * 2)(member(), member(**bad))
        assert lib.amr_create_batch(C.byref(p), 2, members, C.byref(h)) == amr.AMR_EINVAL, bad
        assert not h.value and lib.amr_last_error().decode(), bad
    members = (amr.amr_member * 1)(member())
    assert lib.amr_create_batch(C.byref(p), 0, members, C.byref(h)) == amr.AMR_EINVAL
    assert lib.amr_create_batch(C.byref(p), 1, None, C.byref(h)) == amr.AMR_EINVAL
    for field, value in (("tile", 100), ("nsubgrid", 3), ("planar", 2), ("precision", 16)):
        q = amr.amr_params()
        lib.amr_params_default(C.byref(q))
        setattr(q, field, value)
        assert lib.amr_create_batch(C.byref(q), 1, members, C.byref(h)) == amr.AMR_EINVAL, field
        assert not h.value
