"""The per-variable level scale of the FP64 parity tolerance: max |U_v| over
the level; for the momenta of a level at rest (max |m| below AT_REST of the
level's max sqrt(2 rho E), which bounds every physical momentum since
E >= |m|^2 / (2 rho) when p >= 0) at least that max sqrt(2 rho E)."""
import numpy as np

from parity import AT_REST, close, level_scale


def _state(rng, n, rest=False):
    rho = rng.uniform(0.5, 2.0, n)
    u = np.zeros((3, n)) if rest else rng.normal(0.0, 1.0, (3, n))
    p = rng.uniform(0.1, 1.0, n)
    E = p / (5.0 / 3.0 - 1.0) + 0.5 * rho * (u ** 2).sum(axis=0)
    return np.vstack([rho, rho * u, E])


def test_moving_level_keeps_its_own_momentum_scale():
    rng = np.random.default_rng(0)
    U = _state(rng, 64)
    s = level_scale(U)
    assert np.array_equal(s[:, 0], np.abs(U).max(axis=1))


def test_level_at_rest_takes_the_energy_scale():
    rng = np.random.default_rng(2)
    U = _state(rng, 64, rest=True)
    U[1:4] = rng.normal(0.0, 1e-19, (3, 64))
    s = level_scale(U)
    e = np.sqrt(2.0 * U[0] * U[4]).max()
    assert np.all(s[1:4, 0] == e)
    assert s[0, 0] == np.abs(U[0]).max() and s[4, 0] == np.abs(U[4]).max()
    # just above the at-rest threshold the level counts as moving
    U[1, 3] = 2.0 * AT_REST * e
    assert np.array_equal(level_scale(U)[:, 0], np.abs(U).max(axis=1))


def test_momentum_error_on_a_hot_slow_sedov_level_fails():
    """A Sedov level after one coarse step of the oracle: the blast's energy
    (max sqrt(2 rho E) several times the largest momentum) above momenta
    that are real flow, not round-off.  A momentum error between 1e-12 of
    the level's largest momentum and 1e-12 of its max sqrt(2 rho E) (their
    geometric mean) must fail the 1e-12 tolerance; under the energy's scale
    it would pass."""
    import oracle
    from paper_2607_20704_gb300 import inputs
    prob = inputs.sedov(4, 6)
    o = oracle.Mesh(*prob.mesh_args(), **prob.params())
    o.advance(1)
    best = None
    for l in o.levels():
        _, U = o.read(l)
        mmax = np.abs(U[1:4]).max()
        e = np.sqrt(2.0 * np.maximum(U[0], 0) * np.maximum(U[4], 0)).max()
        if best is None or e / mmax > best[1] / best[0]:
            best = (mmax, e, U)
    mmax, e, U = best
    assert mmax > AT_REST * e and e > 3.0 * mmax, (mmax, e)
    bad = U.copy()
    c = np.unravel_index(np.abs(U[1:4]).argmax(), U[1:4].shape)
    delta = 1e-12 * np.sqrt(mmax * e)
    bad[1 + c[0], c[1]] += delta
    assert delta / e < 1e-12  # the energy's scale would pass it
    try:
        close(bad, U, 1e-12)
    except AssertionError:
        return
    raise AssertionError("a momentum error above 1e-12 of a moving level's scale passed")
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
