"""Pins of the oracle's multigrid Poisson solver (Sec. 5) on a periodic
level: the discrete solution computed independently with numpy's FFT (the
7-point Laplacian is diagonal in Fourier space), the convergence rate the
paper states (about one order of magnitude of residual per V-cycle), and a
single Fourier mode."""
import numpy as np
import pytest

import oracle


def _fft_solution(rho, dx, fourpiG):
    """Exact solution of the 7-point periodic discrete Poisson problem."""
    n = rho.shape[0]
    f = fourpiG * (rho - rho.mean())
    k = np.fft.fftfreq(n) * n
    KX, KY, KZ = np.meshgrid(k, k, k, indexing="ij")
    lam = (2 * np.cos(2 * np.pi * KX / n) + 2 * np.cos(2 * np.pi * KY / n)
           + 2 * np.cos(2 * np.pi * KZ / n) - 6) / dx ** 2
    fh = np.fft.fftn(f)
    lam[0, 0, 0] = 1.0
    ph = fh / lam
    ph[0, 0, 0] = 0.0
    return np.real(np.fft.ifftn(ph))


@pytest.mark.parametrize("n", [8, 16, 32])
def test_converges_to_the_fft_solution(n):
    rng = np.random.default_rng(n)
    rho = 1.0 + 0.3 * rng.standard_normal((n, n, n))
    dx = 1.0 / n
    phi, res = oracle.mg_solve(rho, dx, fourpiG=2.5, ncycles=14)
    want = _fft_solution(rho, dx, 2.5)
    assert np.max(np.abs(phi - want)) <= 1e-9 * np.max(np.abs(want))


def test_residual_drops_about_an_order_per_vcycle():
    n = 32
    rng = np.random.default_rng(3)
    rho = np.exp(rng.standard_normal((n, n, n)))
    phi, res = oracle.mg_solve(rho, 1.0 / n, ncycles=6)
    r0 = oracle.mg_residual(rho, 1.0 / n, np.zeros_like(rho))
    rates = np.concatenate([[res[0] / r0], res[1:] / res[:-1]])
    assert np.all(rates < 0.2), rates


def test_single_fourier_mode():
    """rho - mean = sin(2 pi x) cos(4 pi y): phi = -f / |lambda(k)|, with the
    discrete eigenvalue of the 7-point operator."""
    n = 16
    dx = 1.0 / n
    c = (np.arange(n) + 0.5) * dx
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    rho = 2.0 + np.sin(2 * np.pi * X) * np.cos(4 * np.pi * Y)
    phi, _ = oracle.mg_solve(rho, dx, ncycles=14)
    lam = (2 * np.cos(2 * np.pi / n) + 2 * np.cos(4 * np.pi / n) + 2 - 6) / dx ** 2
    want = (rho - 2.0) / lam
    assert np.max(np.abs(phi - want)) <= 1e-9 * np.max(np.abs(want))


def test_linearity_and_invariance_under_a_constant():
    n = 8
    rng = np.random.default_rng(7)
    a, b = rng.random((n, n, n)), rng.random((n, n, n))
    pa, _ = oracle.mg_solve(a, 1 / n, ncycles=12)
    pb, _ = oracle.mg_solve(b, 1 / n, ncycles=12)
    pab, _ = oracle.mg_solve(a + 3.0 * b + 5.0, 1 / n, ncycles=12)
    assert np.max(np.abs(pab - (pa + 3.0 * pb))) <= 1e-9 * np.max(np.abs(pab))
