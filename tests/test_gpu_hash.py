"""The device's hash function and table (Sec. 2.1 "fnv64"; Sec. 6 names
FNV-1a 64): the function the table uses equals the oracle's FNV-1a 64
(itself pinned by the published FNV test vectors, tests/golden/fnv1a64.txt)
on random and edge keys, and every key the device stored sits in the
linear-probing run that starts at its FNV-1a home slot, with the value of
its oct.  Lookup parity alone would hold with any hash function."""
import numpy as np
import pytest

from paper_2607_20704_gb300 import inputs

pytestmark = pytest.mark.gpu

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_20704_gb300 import amr, build
    build.build()
    amr.load()


def _internal(ext, member=0):
    """Internal key of an external key l<<60 | i<<40 | j<<20 | k."""
    e = int(ext)
    l, i, j, k = e >> 60, (e >> 40) & 0xFFFFF, (e >> 20) & 0xFFFFF, e & 0xFFFFF
    return (member << 49) | (l << 45) | (i << 30) | (j << 15) | k


def test_device_hash_is_fnv1a64():
    import oracle
    from paper_2607_20704_gb300 import amr
    prob = inputs.sod(3, 4)
    g = amr.Mesh(*prob.mesh_args(), **prob.params())
    rng = np.random.default_rng(0)
    keys = np.concatenate([rng.integers(0, 2 ** 63, 4000, dtype=np.uint64) * np.uint64(2) +
                           rng.integers(0, 2, 4000, dtype=np.uint64),
                           np.array([0, 1, 0xFF, 0x100, 2 ** 63, 2 ** 64 - 1], np.uint64)])
    got = g.hash(keys)
    want = np.array([oracle.fnv1a64_key(int(k)) for k in keys], np.uint64)
    assert np.array_equal(got, want)
    # the oracle's key hash is FNV-1a over the key's little-endian bytes
    for k in keys[:50]:
        assert oracle.fnv1a64_key(int(k)) == oracle.fnv1a64_bytes(int(k).to_bytes(8, "little"))
    g.close()


@pytest.mark.parametrize("seed", [61, 62])
def test_table_places_every_key_from_its_fnv1a_home_slot(seed):
    import oracle
    from paper_2607_20704_gb300 import amr
    prob = inputs.random_mesh(3, 6, seed=seed)
    g = amr.Mesh(*prob.mesh_args(), **prob.params())
    keys, vals = g.read_hash()
    cap = keys.size
    assert cap & (cap - 1) == 0
    occ = keys != EMPTY
    # expected contents: real octs (value 1 + mesh index), ghost octs (value
    # 1 + N + cache slot)
    want = {}
    base = 0
    for l in g.levels():
        ext, _ = g.read(l)
        for q, e in enumerate(ext):
            want[_internal(e)] = base + q + 1
        base += ext.size
    N = base
    for l in g.levels():
        ck, _, first = g.read_cache(l)
        for q, e in enumerate(ck):
            want[_internal(e)] = N + first + q + 1
    assert int(occ.sum()) == len(want)
    assert cap >= 2 * len(want)
    mask = cap - 1
    for s in np.flatnonzero(occ):
        k = int(keys[s])
        assert want.get(k) == int(vals[s]), (hex(k), int(vals[s]))
        home = oracle.fnv1a64_key(k) & mask
        # linear probing: every slot from the home slot up to s is occupied
        d = (int(s) - home) & mask
        run = (home + np.arange(d + 1)) & mask
        assert occ[run].all(), (hex(k), home, int(s))
    g.close()
