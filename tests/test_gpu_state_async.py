"""Whole-state copies that overlap the level steps (amr_load_state_async /
amr_store_state_async): the same states, bit for bit, as the synchronous
per-level write/read path, in FP64 and FP32, pipelined over several steps,
across a regrid, with the argument checks."""
import numpy as np
import pytest

from paper_2607_20704_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_20704_gb300 import amr, build
    build.build()
    amr.load()


def _pinned(shape):
    import torch
    return torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()


def _levels_state(m):
    return np.concatenate([m.read(l)[1] for l in m.levels()], axis=1)


@pytest.mark.parametrize("precision", [8, 4])
def test_pipelined_steps_equal_the_synchronous_path(precision):
    from paper_2607_20704_gb300 import amr
    prob = inputs.sedov(4, 6, radii={5: 0.15, 6: 0.08})
    kw = dict(precision=precision, tile=128, schedule=0)
    a = amr.Mesh(*prob.mesh_args(), **prob.params(), **kw)
    b = amr.Mesh(*prob.mesh_args(), **prob.params(), **kw)
    n = a.state_octs()
    x0 = _levels_state(a)
    # two different inputs, alternating, each stepped once
    a.advance(1, sync=True)
    x1 = _levels_state(a)
    ins = [_pinned((5, 8 * n)), _pinned((5, 8 * n))]
    ins[0][:] = x0
    ins[1][:] = x1
    outs = [_pinned((5, 8 * n)) for _ in range(4)]
    for k in range(4):
        b.load_state_async(ins[k % 2])
        b.advance(1)
        b.store_state_async(outs[k])
    b.sync()
    # the synchronous path: write each level, step, read back
    for k in range(4):
        src = ins[k % 2]
        off = 0
        for l in a.levels():
            nl = a.num_octs(l)
            a.write(l, np.ascontiguousarray(src[:, 8 * off:8 * (off + nl)]))
            off += nl
        a.advance(1, sync=True)
        assert np.array_equal(_levels_state(a), outs[k]), (precision, k)
    a.close()
    b.close()


def test_load_then_read_and_store_after_regrid():
    from paper_2607_20704_gb300 import amr
    prob = inputs.sod(4, 6)
    m = amr.Mesh(*prob.mesh_args(), **prob.params(), refine_grad_rho=0.1, refine_grad_p=0.1)
    n = m.state_octs()
    u = _levels_state(m) * 1.0
    u[4] *= 1.5  # a different energy everywhere
    buf = _pinned((5, 8 * n))
    buf[:] = u
    m.load_state_async(buf)
    m.sync()
    assert np.array_equal(_levels_state(m), u)
    m.regrid()
    n2 = m.state_octs()
    out = _pinned((5, 8 * n2))
    m.store_state_async(out)
    m.sync()
    assert np.array_equal(out, _levels_state(m))
    m.close()


def test_bad_state_arguments():
    from paper_2607_20704_gb300 import amr
    prob = inputs.sod(3, 4)
    m = amr.Mesh(*prob.mesh_args(), **prob.params())
    n = m.state_octs()
    with pytest.raises(amr.AmrError) as e:
        m.load_state_async(np.zeros((5, 8 * (n + 1))))
    assert e.value.status == amr.AMR_EINVAL
    with pytest.raises(amr.AmrError):
        m.store_state_async(np.zeros((5, 8 * (n - 1))))
    m.close()
