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


def _inverse_xorshift(y, s):
    # x ^ (x >> s) inverted by repeated substitution (s >= 1, 64-bit words)
    x = y.copy()
    for _ in range(64 // s + 1):
        x = y ^ (x >> np.uint64(s))
    return x


def test_mixers_are_bijections_on_random_keys():
    """Hash and the mixer behind Hash2 are bijections of 64-bit words: no two of 2^20
    random keys collide, and the published steps undone one by one (xor-shifts and odd
    multipliers are invertible mod 2^64) give every key back."""
    rng = np.random.default_rng(17)
    keys = np.unique(rng.integers(0, 2**63, size=1 << 20, dtype=np.uint64) * np.uint64(2)
                     + rng.integers(0, 2, size=1 << 20, dtype=np.uint64))
    h1, m2 = O.mix_batch(keys)
    assert len(np.unique(h1)) == len(keys)
    assert len(np.unique(m2)) == len(keys)
    M = 1 << 64
    with np.errstate(over="ignore"):
        # SplitMix64 output function: z ^= z >> 30; z *= c1; z ^= z >> 27; z *= c2; z ^= z >> 31
        inv = lambda c: np.uint64(pow(c, -1, M))
        x = _inverse_xorshift(h1, 31) * inv(0x94D049BB133111EB)
        x = _inverse_xorshift(x, 27) * inv(0xBF58476D1CE4E5B9)
        x = _inverse_xorshift(x, 30)
        assert np.array_equal(x, keys)
        # fmix64: k ^= k >> 33; k *= c1; k ^= k >> 33; k *= c2; k ^= k >> 33
        y = _inverse_xorshift(m2, 33) * inv(0xC4CEB9FE1A85EC53)
        y = _inverse_xorshift(y, 33) * inv(0xFF51AFD7ED558CCD)
        y = _inverse_xorshift(y, 33) ^ np.uint64(0x9E3779B97F4A7C15)
        assert np.array_equal(y, keys)


def test_mixers_avalanche():
    """Flipping one key bit flips about half of the output bits, for every input bit and
    every output bit (strict avalanche, within sampling error over 4096 keys)."""
    rng = np.random.default_rng(19)
    keys = rng.integers(0, 2**63, size=4096, dtype=np.uint64)
    h1, m2 = O.mix_batch(keys)
    for base in (h1, m2):
        frac = np.zeros((64, 64))
        for b in range(64):
            f1, f2 = O.mix_batch(keys ^ np.uint64(1 << b))
            diff = base ^ (f1 if base is h1 else f2)
            bits = (diff[:, None] >> np.arange(64, dtype=np.uint64)) & np.uint64(1)
            frac[b] = bits.mean(axis=0)
        assert abs(frac.mean() - 0.5) < 0.005
        assert frac.min() > 0.42 and frac.max() < 0.58


def test_address_batch_is_the_scalar_definition():
    rng = np.random.default_rng(23)
    n = 2000
    mat = rng.integers(0, 1 << 16, n, dtype=np.uint32)
    node = rng.integers(0, 1 << 16, n, dtype=np.uint32)
    u = rng.random(n).astype(np.float32)
    v = rng.random(n).astype(np.float32)
    key, cell, h2 = O.address_batch(mat, node, u, v, 10, 10**7)
    for i in range(0, n, 97):
        k = O.key(int(mat[i]), int(node[i]), 10, float(u[i]), float(v[i]))
        assert key[i] == k and cell[i] == O.hash1(k) % 10**7 and h2[i] == O.hash2(k)
