"""Hand-worked descriptors (Sec. 3.1, Eq. 1) and the table addressing of Alg. 1.

Texel indices below are worked out by hand from the definition: a virtual texture of
2^lambda texels per axis, u clamped to [0, 1], texel = floor(u * 2^lambda), u = 1
falling in the last texel.  The key packs mat<<48 | node<<32 | lambda<<26 | iu<<13 | iv.
"""
import numpy as np
import pytest

from oracle import oracle as O


def f32(x):
    return float(np.float32(x))


@pytest.mark.parametrize("u,level,expected", [
    (0.0, 10, 0),
    (1.0, 10, 1023),                      # u = 1 is the last texel, not 1024
    (0.5, 10, 512),
    (511 / 1024, 10, 511),                # exact texel edge
    (f32(np.nextafter(np.float32(0.5), np.float32(0))), 10, 511),  # just below an edge
    (-0.25, 10, 0),                       # clamped below
    (1.5, 10, 1023),                      # clamped above
    (float("nan"), 10, 0),                # NaN treated as 0
    (0.999, 0, 0),                        # one texel at level 0
    (0.75, 1, 1),
    (1.0, 13, 8191),
    (0.1, 13, 819),                       # floor(0.1f * 8192) = floor(819.2000...) = 819
])
def test_texel_hand_worked(u, level, expected):
    assert O.texel(u, level) == expected


def test_keys_hand_worked():
    # (mat, node, level, u, v) -> key, packed by hand
    assert O.key(0, 7, 10, 0.0, 0.0) == 0x0000_0007_2800_0000
    assert O.key(1, 2, 10, 1.0, 0.5) == (1 << 48) | (2 << 32) | (10 << 26) | (1023 << 13) | 512
    assert O.key(3, 0, 10, 0.25, 0.75) == 0x0003_0000_2800_0000 | (256 << 13) | 768
    assert O.key(0xFFFF, 0xFFFF, 13, 1.0, 1.0) == 0xFFFF_FFFF_37FF_FFFF
    assert O.key(5, 9, 10, 0.5, 0.5) != O.key(5, 9, 10, 0.5, f32(0.5 + 1 / 1024))
    assert O.key(5, 9, 10, 0.5, 0.5) == O.key(5, 9, 10, f32(0.5 + 0.5 / 1024), 0.5)


def test_same_texel_same_key_different_node_different_key():
    # 0.1001 * 1024 = 102.50, 0.1002 * 1024 = 102.60; 0.2101 * 1024 = 215.14, 0.2102 * 1024 = 215.24
    k1 = O.key(2, 4, 10, f32(0.1001), f32(0.2101))
    k2 = O.key(2, 4, 10, f32(0.1002), f32(0.2102))   # same texel (width 1/1024)
    k3 = O.key(2, 5, 10, f32(0.1001), f32(0.2101))
    k4 = O.key(3, 4, 10, f32(0.1001), f32(0.2101))
    assert k1 == k2 and k1 != k3 and k1 != k4


def test_cell_is_hash1_mod_cells():
    # cell = Hash(desc) % N_c (Alg. 1) for a few table sizes including the
    # 10 x 5 table of Fig. 3 and the paper's 10^7 cells.
    c = O.Cache([], 10, 5)
    assert c.n_cells == 10
    for k in (1, 12345, 0xFFFF_FFFF_37FF_FFFF):
        for nc in (10, 8192, 10**7):
            assert O.hash1(k) % nc < nc
    assert O.hash2(0x0000_0007_2800_0000) != 0
