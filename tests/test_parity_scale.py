"""The per-variable level scale of the FP64 parity tolerance: max |U_v| over
the level, and for the momenta at least max sqrt(2 rho E), which bounds every
physical momentum of the level (E >= |m|^2 / (2 rho) when p >= 0)."""
import numpy as np

from parity import close, level_scale


def _state(rng, n, rest=False):
    rho = rng.uniform(0.5, 2.0, n)
    u = np.zeros((3, n)) if rest else rng.normal(0.0, 1.0, (3, n))
    p = rng.uniform(0.1, 1.0, n)
    E = p / (5.0 / 3.0 - 1.0) + 0.5 * rho * (u ** 2).sum(axis=0)
    return np.vstack([rho, rho * u, E])


def test_scale_bounds_every_momentum():
    rng = np.random.default_rng(0)
    U = _state(rng, 64)
    s = level_scale(U)
    assert np.all(s[:, 0] >= np.abs(U).max(axis=1))
    assert np.all(s[1:4, 0] == np.sqrt(2.0 * U[0] * U[4]).max())
    assert s[0, 0] == np.abs(U[0]).max() and s[4, 0] == np.abs(U[4]).max()


def test_round_off_momenta_of_a_level_at_rest():
    rng = np.random.default_rng(1)
    U = _state(rng, 64, rest=True)
    a = U.copy()
    b = U.copy()
    a[1:4] = rng.normal(0.0, 1e-19, (3, 64))
    b[1:4] = rng.normal(0.0, 1e-19, (3, 64))
    close(a, b, 1e-12)  # noise against the energy's scale: passes
    c = b.copy()
    c[2, 7] += 1e-9 * np.sqrt(2.0 * U[0] * U[4]).max()  # a real momentum error
    try:
        close(a, c, 1e-12)
    except AssertionError:
        return
    raise AssertionError("a momentum error of 1e-9 of the scale passed")


def test_empty_and_non_state_arrays():
    assert level_scale(np.zeros((5, 0))).shape == (5, 1)
    R = np.arange(12.0).reshape(3, 4)
    assert np.array_equal(level_scale(R)[:, 0], np.abs(R).max(axis=1))
