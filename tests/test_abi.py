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


def _declared():
    text = open(os.path.join(ROOT, "include", "amr.h")).read()
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
    assert (p.precision, p.reflux, p.reindex_every_step, p.use_graphs) == (8, 1, 1, 1)
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
