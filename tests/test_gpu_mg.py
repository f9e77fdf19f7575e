"""Multigrid Poisson V-cycles on the GPU (Sec. 5) against the oracle: the
potential of the base-level cells and the residual after every V-cycle,
and convergence to the discrete solution.

Tolerance of the potential.  The oracle's Gauss-Seidel update divides by 6;
the GPU multiplies by fl(1/6).  Each update then differs by at most 3 units
of round-off u = 2^-53 of the updated value (fl(1/6) off by u, one product
against one quotient); the residual's 1/dx^2 is exact (dx a power of two),
so the residuals and the transfers between levels are evaluated alike.  A
V-cycle on L levels applies (nu1 + nu2) sweeps per level, 4 here, so it
adds at most 4 L x 3u max|phi| of difference per cycle; the difference is
carried by the cycle's error operator, whose contraction (residual x0.1 per
cycle, asserted below as < 0.2) sums the cycles' contributions to at most
1/(1 - 0.2) of one; allowing a factor 10 for the coarse-grid correction's
max-norm amplification gives 4 x 6 levels x 3 x 10 x 1.25 u = 900 u = 1e-13
of max|phi|.  The tests allow 1e-12 (measured differences are far below)."""
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


def _dense(keys, values, level):
    """Cell values in read order -> array [x, y, z] of the level."""
    n = 1 << level
    k = keys.astype(np.int64)
    oi, oj, ok = (k >> 40) & 0xFFFFF, (k >> 20) & 0xFFFFF, k & 0xFFFFF
    c = np.arange(8)
    x = (2 * oi[:, None] + (c & 1)).ravel()
    y = (2 * oj[:, None] + ((c >> 1) & 1)).ravel()
    z = (2 * ok[:, None] + ((c >> 2) & 1)).ravel()
    out = np.zeros((n, n, n))
    out[x, y, z] = values
    return out


def _lognormal_grid(level, seed):
    rng = np.random.default_rng(seed)
    def fn(x, y, z):
        g = 0.5 * np.sin(2 * np.pi * x + rng.random()) * np.cos(2 * np.pi * y) + \
            0.2 * rng.standard_normal(x.shape)
        zero = 0.0 * x
        return np.exp(g), zero, zero, zero, 1.0 + zero
    return inputs.uniform_grid(level, fn)


@pytest.mark.parametrize("level,precision", [(4, 8), (5, 8), (5, 4)])
def test_potential_and_residuals_match_the_oracle(level, precision):
    import oracle
    from paper_2607_20704_gb300 import amr
    prob = _lognormal_grid(level, seed=level)
    g = amr.Mesh(*prob.mesh_args(), **prob.params(), precision=precision)
    keys, U = g.read(level)
    rho = _dense(keys, U[0], level)  # the state as the GPU holds it
    dx = 2.0 ** -level
    res_g = g.poisson(fourpiG=3.0, n_vcycles=3)
    phi_o, res_o = oracle.mg_solve(rho, dx, fourpiG=3.0, ncycles=3)
    phi_g = _dense(keys, g.read_phi(), level)
    assert np.max(np.abs(phi_g - phi_o)) <= 1e-12 * np.max(np.abs(phi_o))
    assert np.allclose(res_g, res_o, rtol=1e-9, atol=0)
    assert np.all(res_g[1:] < 0.2 * res_g[:-1])
    g.close()


def test_calls_continue_from_the_previous_solution():
    from paper_2607_20704_gb300 import amr
    prob = _lognormal_grid(4, seed=9)
    a = amr.Mesh(*prob.mesh_args(), **prob.params())
    b = amr.Mesh(*prob.mesh_args(), **prob.params())
    a.poisson(2.0, 4)
    b.poisson(2.0, 2)
    b.poisson(2.0, 2)
    assert np.array_equal(a.read_phi(), b.read_phi())
    a.close()
    b.close()


def test_base_level_of_an_adaptive_mesh():
    """The base level of a refined mesh (split cells hold their children's
    mean) solved to convergence: equals the oracle's solution and the
    discrete solution from the FFT."""
    import oracle
    from paper_2607_20704_gb300 import amr
    prob = inputs.sedov(4, 6, radii={5: 0.2, 6: 0.1})
    g = amr.Mesh(*prob.mesh_args(), **prob.params())
    keys, U = g.read(4)
    rho = _dense(keys, U[0], 4)
    g.poisson(1.0, 12)
    phi_g = _dense(keys, g.read_phi(), 4)
    phi_o, _ = oracle.mg_solve(rho, 1.0 / 16, ncycles=12)
    assert np.max(np.abs(phi_g - phi_o)) <= 1e-11 * np.max(np.abs(phi_o))
    n = 16
    k = np.fft.fftfreq(n) * n
    KX, KY, KZ = np.meshgrid(k, k, k, indexing="ij")
    lam = (2 * np.cos(2 * np.pi * KX / n) + 2 * np.cos(2 * np.pi * KY / n)
           + 2 * np.cos(2 * np.pi * KZ / n) - 6) * n * n
    lam[0, 0, 0] = 1.0
    ph = np.fft.fftn(rho - rho.mean()) / lam
    ph[0, 0, 0] = 0.0
    want = np.real(np.fft.ifftn(ph))
    assert np.max(np.abs(phi_g - want)) <= 1e-9 * np.max(np.abs(want))
    g.close()
