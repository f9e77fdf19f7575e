"""Pins of the oracle's integer machinery: hash function, Hilbert key, key
packing (paper Sec. 2.1 hash key (i,j,k,l); Sec. 2.2 Hilbert order; Sec. 6
FNV-1a 64)."""
import itertools
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _fnv_vectors():
    out = []
    for line in open(os.path.join(GOLD, "fnv1a64.txt")):
        if line.startswith("#") or not line.strip():
            continue
        s, h = line.split(";")
        out.append((s.strip().strip('"').encode(), int(h.strip(), 16)))
    return out


@pytest.mark.parametrize("text,expect", _fnv_vectors())
def test_fnv1a64_published_vectors(orc, text, expect):
    assert orc.fnv1a64_bytes(text) == expect


def test_fnv_key_is_hash_of_little_endian_bytes(orc):
    for key in (0, 1, 0x0123456789ABCDEF, orc.pack_key(7, 3, 5, 9)):
        b = int(key).to_bytes(8, "little")
        assert orc.fnv1a64_key(key) == orc.fnv1a64_bytes(b)


def test_pack_key_layout(orc):
    assert orc.pack_key(0, 0, 0, 1) == 1
    assert orc.pack_key(0, 0, 1, 0) == 1 << 20
    assert orc.pack_key(0, 1, 0, 0) == 1 << 40
    assert orc.pack_key(1, 0, 0, 0) == 1 << 60
    assert orc.pack_key(15, 0xFFFFF, 0xFFFFF, 0xFFFFF) == 0xFFFFFFFFFFFFFFFF


@pytest.mark.parametrize("bits", [1, 2, 3, 4])
def test_hilbert_is_a_bijection(orc, bits):
    side = 1 << bits
    seen = {}
    for x, y, z in itertools.product(range(side), repeat=3):
        h = orc.hilbert3(x, y, z, bits)
        assert 0 <= h < side ** 3
        assert h not in seen
        seen[h] = (x, y, z)
    assert len(seen) == side ** 3


@pytest.mark.parametrize("bits", [1, 2, 3, 4])
def test_hilbert_consecutive_points_are_face_neighbours(orc, bits):
    """The defining property of a Hilbert curve: successive indices are unit
    steps along exactly one axis; it starts at the origin."""
    side = 1 << bits
    inv = {}
    for x, y, z in itertools.product(range(side), repeat=3):
        inv[orc.hilbert3(x, y, z, bits)] = np.array((x, y, z))
    assert tuple(inv[0]) == (0, 0, 0)
    for h in range(side ** 3 - 1):
        d = np.abs(inv[h + 1] - inv[h])
        assert d.sum() == 1, (h, inv[h], inv[h + 1])


def test_hilbert_octants_are_contiguous(orc):
    """Self-similarity: each block of 8^(b-1) successive indices fills one
    octant of the cube."""
    bits = 3
    side = 1 << bits
    blocks = {}
    for x, y, z in itertools.product(range(side), repeat=3):
        h = orc.hilbert3(x, y, z, bits)
        blocks.setdefault(h // 64, set()).add((x >> 2, y >> 2, z >> 2))
    assert all(len(v) == 1 for v in blocks.values())
    assert len({next(iter(v)) for v in blocks.values()}) == 8


@pytest.mark.parametrize("bits", [1, 2, 5, 9, 14])
def test_hilbert_index_extends_the_parents(orc, bits):
    """The index of a cell at bits + 1 is its parent's index (coordinates
    halved, at bits) followed by one octal digit: octs whose fathers are in
    curve order are in curve order once the children of each father are
    sorted (the order a regrid builds for its new octs)."""
    rng = np.random.default_rng(bits)
    side = 1 << (bits + 1)
    for x, y, z in rng.integers(0, side, size=(2000, 3)):
        child = orc.hilbert3(x, y, z, bits + 1)
        assert child >> 3 == orc.hilbert3(x >> 1, y >> 1, z >> 1, bits), (x, y, z, bits)
