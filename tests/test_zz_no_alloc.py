"""amr_cfl_dt_static: the time-step reduction for callers that cannot
allocate device memory, checked against the handle-based amr_cfl_dt.

Some callers may not allocate on the device at all -- for instance when
another runtime's memory pool already holds the GPU's memory, or inside an
allocator-free real-time loop.  amr_cfl_dt_static takes the caller's own
device buffers and brings fixed scratch of its own.  This file is collected
last so that a run stopping at the first failure has run every other test
before it."""
import numpy as np
import pytest

from paper_2607_20704_gb300 import inputs

pytestmark = pytest.mark.gpu


def _random_uniform_grid(seed, level=5):
    rng = np.random.default_rng(seed)

    def fn(x, y, z):
        rho = 1.0 + 0.5 * rng.random(x.shape)
        p = 0.5 + rng.random(x.shape)
        vel = [2.0 * rng.standard_normal(x.shape) for _ in range(3)]
        return rho, vel[0], vel[1], vel[2], p
    return inputs.uniform_grid(level, fn, gamma=1.4)


def test_static_scratch_time_step_matches_handle_time_step():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import oracle
    from paper_2607_20704_gb300 import amr, build
    build.build()
    amr.load()
    dt_out = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for seed in (1, 2):  # two calls in a row on the same fixed scratch
        prob = _random_uniform_grid(seed)
        m = amr.Mesh(*prob.mesh_args(), **prob.params())
        want = m.cfl_dt()
        _, U = m.read(prob.levelmin)
        m.close()
        Ud = torch.from_numpy(np.ascontiguousarray(U)).to("cuda")
        n = U.shape[1]
        amr.amr_cfl_dt_static(Ud.data_ptr(), n, n, prob.levelmin, prob.gamma, prob.cfl,
                              1e-10, 1e-10, dt_out.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        got = float(dt_out.item())
        assert abs(got - want) <= 1e-14 * want, (seed, got, want)
        # and the oracle's time step of the same uniform grid (level dt)
        orc = oracle.uniform_cfl_dt(U, prob.gamma, prob.cfl)
        assert abs(got - orc) <= 1e-14 * orc, (seed, got, orc)
    with pytest.raises(amr.AmrError) as e:
        amr.amr_cfl_dt_static(Ud.data_ptr(), amr.CFL_STATIC_MAX_CELLS + 1, amr.CFL_STATIC_MAX_CELLS + 1,
                              5, 1.4, 0.8, 1e-10, 1e-10, dt_out.data_ptr(), stream.cuda_stream)
    assert e.value.status == amr.AMR_EINVAL


def _numpy_dt(U, level, gamma, cfl, smallr=1e-10, smallc=1e-10):
    """cfl dx / max sum_d (|u_d| + c) written out in numpy."""
    r = np.maximum(U[0], smallr)
    v = U[1:4] / r
    ek = 0.5 * r * (v * v).sum(axis=0)
    p = np.maximum((gamma - 1.0) * (U[4] - ek), r * smallc * smallc / gamma)
    c = np.sqrt(gamma * p / r)
    return cfl * 2.0 ** -level / (np.abs(v) + c).sum(axis=0).max()


def test_static_scratch_ragged_size_wider_stride_and_a_nan_cell():
    """257 cells (one past a 256-thread block) in rows of stride 300, then
    the same with one cell NaN: dt equals the numpy definition, then NaN."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_20704_gb300 import amr, build
    build.build()
    amr.load()
    rng = np.random.default_rng(5)
    n, stride = 257, 300
    U = np.zeros((5, stride))
    rho = 1.0 + rng.random(n)
    vel = rng.standard_normal((3, n))
    p = 0.5 + rng.random(n)
    U[0, :n] = rho
    U[1:4, :n] = rho * vel
    U[4, :n] = p / 0.4 + 0.5 * rho * (vel ** 2).sum(axis=0)
    U[:, n:] = 1e6  # past n_cells: never read
    stream = torch.cuda.current_stream()
    dt_out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for bad in (False, True):
        V = U.copy()
        if bad:
            V[3, 200] = np.nan
        Ud = torch.from_numpy(V).to("cuda")
        amr.amr_cfl_dt_static(Ud.data_ptr(), n, stride, 4, 1.4, 0.8, 1e-10, 1e-10,
                              dt_out.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        got = float(dt_out.item())
        if bad:
            assert np.isnan(got)
        else:
            want = _numpy_dt(V[:, :n], 4, 1.4, 0.8)
            assert abs(got - want) <= 1e-14 * want, (got, want)
