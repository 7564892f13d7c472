"""Pins for the oracle's determinant <-> integer bijection (Eq. 12, Sec. 2.2)."""
import itertools
import math

import numpy as np
import pytest

from conftest import bits_from_string, read_golden, string_from_bits


def test_table1_gchain(orc):
    """Table 1: the successor g enumerates the (6o,3e) space in the printed order,
    and the chain distance is the index (unrank(i) is the i-th string)."""
    chain = [r[0] for r in read_golden("table1_gchain_6o3e.txt")]
    assert len(chain) == 20 == math.comb(6, 3)
    s = bits_from_string(chain[0])
    got = [string_from_bits(s, 6)]
    while True:
        s = orc.string_successor(s, 6)
        if s is None:
            break
        got.append(string_from_bits(s, 6))
    assert got == chain
    for i, st in enumerate(chain):
        assert string_from_bits(orc.string_unrank(i, 6, 3), 6) == st


def test_table2_hash_values(orc):
    """Table 2: every printed hash value, and every printed binomial term."""
    for row in read_golden("table2_hash_6o3e.txt"):
        st, n1, k1, n2, k2, n3, k3, h = row[0], *map(int, row[1:])
        bits = bits_from_string(st)
        assert orc.string_rank(bits, 6) == h
        terms = [(n1, k1), (n2, k2), (n3, k3)]
        assert sum(orc.binom(n, k) for n, k in terms) == h
        # chi_i - 1 and i of Eq. 12, read off the string
        occ = [p for p in range(6) if (bits >> p) & 1]
        assert [(chi, i + 1) for i, chi in enumerate(occ)] == terms


def test_worked_example_101010(orc):
    """Sec. 2.2: h(101010) = C(4,3) + C(2,2) + C(0,1) = 4 + 1 + 0 = 5."""
    row = read_golden("worked_example_101010.txt")[0]
    st = row[0]
    vals = list(map(int, row[1:]))
    for t in range(3):
        n, k, v = vals[3 * t: 3 * t + 3]
        assert orc.binom(n, k) == v
    assert orc.string_rank(bits_from_string(st), 6) == vals[-1] == 5


def test_binomial_convention(orc):
    """C(n,k) = 0 for n < k (Eq. 12), Pascal's rule, and exact 64-bit values."""
    for n in range(0, 65):
        for k in range(0, 65):
            assert orc.binom(n, k) == (math.comb(n, k) if k <= n else 0)
    assert orc.binom(3, 5) == 0
    assert orc.binom(64, 32) == math.comb(64, 32)


@pytest.mark.parametrize("n", [1, 2, 5, 8, 11, 12])
def test_rank_is_colex_position(orc, n):
    """The index of a string is its position among all strings with the same
    electron count, ordered by the value of the bit mask (brute force)."""
    for m in range(0, n + 1):
        masks = sorted(sum(1 << p for p in c) for c in itertools.combinations(range(n), m))
        for pos, s in enumerate(masks):
            assert orc.string_rank(s, n) == pos
            assert orc.string_unrank(pos, n, m) == s


@pytest.mark.parametrize("n,m", [(28, 7), (28, 14), (64, 32), (64, 5), (40, 20)])
def test_rank_roundtrip_sampled(orc, n, m):
    rng = np.random.default_rng(n * 100 + m)
    top = math.comb(n, m)
    rs = [0, top - 1] + [int(x) for x in rng.integers(0, top, size=300, dtype=np.uint64)]
    for r in rs:
        s = orc.string_unrank(r, n, m)
        assert bin(s).count("1") == m and s < (1 << n)
        assert orc.string_rank(s, n) == r
    # the successor moves the index by exactly one
    for r in rs[:50]:
        if r + 1 < top:
            s = orc.string_unrank(r, n, m)
            assert orc.string_rank(orc.string_successor(s, n), n) == r + 1


def test_full_rank_bijection(orc):
    """alpha-major index over the whole (8o, 4a/4b) space: a bijection onto
    [0, dim), and index 0 is the aufbau determinant."""
    n, na, nb = 8, 4, 4
    d = orc.dim(n, na, nb)
    assert d == 4900
    r = np.arange(d, dtype=np.uint64)
    a, b = orc.det_unrank(n, na, nb, r)
    assert np.all(orc.det_rank(n, nb, a, b) == r)
    assert len(set(zip(a.tolist(), b.tolist()))) == d
    assert a[0] == 0b1111 and b[0] == 0b1111
    for x, y in zip(a.tolist()[:200], b.tolist()[:200]):
        assert bin(x).count("1") == na and bin(y).count("1") == nb


def test_dim_matches_paper_sizes(orc):
    """C(n,na) C(n,nb) / |G| reproduces the printed FCI sizes (3 digits)."""
    for row in read_golden("fci_space_sizes.txt"):
        n, na, nb, grp = map(int, row[:4])
        printed = float(row[4])
        est = orc.dim(n, na, nb) / grp
        digits = len(row[4].split("e")[0].replace(".", ""))
        assert abs(est - printed) <= 0.5 * 10 ** (math.floor(math.log10(printed)) - digits + 1)


def test_dim_overflow(orc):
    with pytest.raises(OverflowError):
        orc.dim(64, 32, 32)
    assert orc.dim(28, 7, 7) == math.comb(28, 7) ** 2
