"""The sparse form of the CIC parity bound (used on the largest grid, where
n^3 host arrays are too large) equals the dense form at every cell."""
import numpy as np
import pytest

from paper_2607_20704_gb300 import inputs


@pytest.mark.parametrize("precision", [8, 4])
@pytest.mark.parametrize("n,kind", [(8, "uniform"), (16, "cosmo"), (32, "clump")])
def test_sparse_bound_equals_dense(n, kind, precision):
    import test_gpu_cic as t
    import oracle
    kw = dict(n_particles=3000) if kind != "cosmo" else {}
    ps = inputs.particles(n, kind, seed=n, masses="random", **kw)
    ref = oracle.cic_deposit(*ps.args())
    dense = t._bound(*ps.args(), ref, precision).reshape(-1, order="F")
    cells = np.unique(np.random.default_rng(n).integers(0, n ** 3, 3 * n))
    sparse = t.bound_at(*ps.args(), ref.reshape(-1, order="F")[cells], cells, precision)
    assert np.array_equal(sparse, dense[cells])
