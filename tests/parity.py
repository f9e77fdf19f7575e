"""Helpers of the GPU-vs-oracle parity tests.

Tolerance (FP64 state, one step from identical inputs): per variable v,
|gpu - oracle| <= rtol * max(|oracle|, s_v), s_v = max |U_v| over the
level.  On a level at rest, whose momenta are pure round-off (max |m| below
1e-8 of the level's max sqrt(2 rho E), the largest momentum its energy
allows since E >= |m|^2 / 2 rho), s_v of the three momentum components is
raised to that max sqrt(2 rho E): round-off in a momentum update scales with
the fluxes, i.e. with the energy present, so such a level (1e-19 against
E ~ 1e2 on the coarse levels of a deep hierarchy) would otherwise be held to
a relative bound on noise.  Every level that moves keeps s_v = max |m|, the
tolerance of a per-cell FP64 comparison.  rtol = 1e-12 per level
step; the W-cycle tests that chain many level steps from one initial state
allow 1e-11 (round-off is re-amplified by the nonlinear limiter/Riemann
steps that follow)."""
import numpy as np

from paper_2607_20704_gb300 import inputs


# a level whose largest momentum is below this fraction of its largest
# sqrt(2 rho E) is at rest: its momenta are round-off
AT_REST = 1e-8


def level_scale(U):
    """s_v per variable of a [5][cells] state (see the module docstring)."""
    if U.shape[1] == 0:
        return np.zeros((U.shape[0], 1))
    s = np.abs(U).max(axis=1, keepdims=True).astype(np.float64)
    if U.shape[0] == 5:
        e = np.sqrt(2.0 * np.maximum(U[0], 0.0) * np.maximum(U[4], 0.0)).max()
        if s[1:4].max() < AT_REST * e:
            s[1:4] = np.maximum(s[1:4], e)
    return s


def close(gpu, orc, rtol, what=""):
    gpu = np.asarray(gpu)
    orc = np.asarray(orc)
    assert gpu.shape == orc.shape, (what, gpu.shape, orc.shape)
    if orc.size == 0:
        return 0.0
    s = level_scale(orc)
    scale = np.maximum(np.abs(orc), s)
    scale[scale == 0] = 1.0
    err = np.abs(gpu - orc) / scale
    worst = float(err.max())
    assert worst <= rtol, f"{what}: max scaled error {worst:.3e} > {rtol:.1e} at {np.unravel_index(err.argmax(), err.shape)}"
    return worst


def pair(prob, gpu_kw=None, orc_kw=None):
    import oracle
    from paper_2607_20704_gb300 import amr
    g = amr.Mesh(*prob.mesh_args(), **prob.params(), **(gpu_kw or {}))
    o = oracle.Mesh(*prob.mesh_args(), **prob.params(), **(orc_kw or {}))
    return g, o


def compare_all(g, o, rtol, levels=None, reflux=True):
    worst = 0.0
    for l in levels or o.levels():
        kg, Ug = g.read(l)
        ko, Uo = o.read(l)
        assert np.array_equal(kg, ko), f"level {l} order differs"
        worst = max(worst, close(Ug, Uo, rtol, f"U level {l}"))
        if reflux:
            Rg, Ro = g.read_reflux(l), o.read_R(l)
            s = np.maximum(level_scale(Uo), 1e-300)
            err = float((np.abs(Rg - Ro) / s).max()) if Ro.size else 0.0
            assert err <= rtol, f"R level {l}: {err:.3e}"
    return worst
