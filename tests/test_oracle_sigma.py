"""Pins for the oracle's sigma = H psi (Sec. 2.2) and truncation (Eq. 11)."""
import numpy as np
import pytest

import gen


def _cfg0(orc):
    return orc.System.from_dict(gen.config_system(0))


def test_sigma_equals_dense_product(orc):
    """Against the dense H of the (8o, 4a/4b) space: values within rounding of
    the per-entry magnitude A_k = sum |H_kD c_D|, support = entries that got a
    non-zero product."""
    S = _cfg0(orc)
    H = orc.dense_h(S)
    rng = np.random.default_rng(1)
    r = np.sort(rng.choice(4900, size=700, replace=False)).astype(np.uint64)
    c = rng.normal(size=r.size)
    sr, sv, sa, nel = orc.sigma(S, r, c)
    assert nel == r.size * (orc.n_connected(8, 4, 4) + 1)
    x = np.zeros(4900)
    x[r.astype(np.int64)] = c
    dense = H @ x
    prod_nz = (np.abs(H[:, r.astype(np.int64)]) * np.abs(c)).sum(axis=1)
    support = np.nonzero(prod_nz > 0)[0]
    assert np.array_equal(sr.astype(np.int64), support)
    assert np.all(np.abs(sv - dense[support]) <= 1e-13 * sa + 1e-300)
    assert np.allclose(sa, prod_nz[support], rtol=1e-13, atol=0)
    assert np.all(np.abs(sv) <= sa * (1 + 1e-15))


def test_sigma_element_screen_against_dense(orc):
    """Heat-bath style selection (Sec. 4 outlook): with eps_element the
    products |H_kD c_D| < eps are not generated.  Against the dense H: sigma_k
    = sum over the kept products, support = rows with a kept product; eps = 0
    is the exact sigma."""
    S = _cfg0(orc)
    H = orc.dense_h(S)
    rng = np.random.default_rng(2)
    r = np.sort(rng.choice(4900, size=600, replace=False)).astype(np.uint64)
    c = rng.normal(size=r.size) * np.exp(rng.uniform(-8, 0, size=r.size))
    P = H[:, r.astype(np.int64)] * c  # every product H_kD c_D
    for eps in (0.0, 1e-4, 1e-2):
        keep = (P != 0.0) & ~(np.abs(P) < eps)
        want = np.where(keep, P, 0.0).sum(axis=1)
        absw = np.where(keep, np.abs(P), 0.0).sum(axis=1)
        support = np.nonzero(keep.any(axis=1))[0]
        sr, sv, sa, _ = orc.sigma(S, r, c, eps_element=eps)
        assert np.array_equal(sr.astype(np.int64), support)
        assert np.all(np.abs(sv - want[support]) <= 1e-13 * absw[support])
        if eps > 0:  # the screen removed products
            assert 0 < np.count_nonzero(keep) < np.count_nonzero(P)


def test_sigma_pull_equals_push_bitwise(orc):
    """Each pulled entry sums the same products in the same order as the
    list-sort-merge, so the two agree bit for bit."""
    d = gen.config_system(2)
    S = orc.System.from_dict(d)
    a, b, lev = gen.near_aufbau_dets(28, 7, 7, 40, seed=5)
    r = np.sort(orc.det_rank(28, 7, a, b))
    c = gen.level_coefs(np.zeros(r.size), seed=6)
    sr, sv, sa, _ = orc.sigma(S, r, c)
    rng = np.random.default_rng(2)
    pick = rng.choice(sr.size, size=200, replace=False)
    val, asum, pres = orc.sigma_entries(S, r, c, sr[pick])
    assert pres.all()
    assert np.array_equal(val.view(np.uint64), sv[pick].view(np.uint64))
    assert np.array_equal(asum.view(np.uint64), sa[pick].view(np.uint64))
    # a target that nothing reaches is absent
    far = orc.det_rank(28, 7, np.array([0xFE00000], dtype=np.uint64),
                       np.array([0xFE00000], dtype=np.uint64))
    v, _, p = orc.sigma_entries(S, r, c, far)
    assert not p[0] and v[0] == 0.0


def test_sigma_hubbard_drops_zero_products(orc):
    """Hubbard ring: of the 1818 enumerated excitations only hops along the
    ring give non-zero elements; zero products are not entries."""
    d = gen.config_system(1)
    S = orc.System.from_dict(d)
    sr, sv, sa, nel = orc.sigma(S, np.array([0], dtype=np.uint64), np.array([1.0]))
    assert nel == 1819
    # aufbau determinant (sites 0..5 filled in both spins): one hop per spin
    # leaves the block at each end, 2 per spin, plus the diagonal (6 doubly
    # occupied sites, U = 4 each)
    assert sr.size == 5
    assert sv[0] == pytest.approx(24.0)


def test_topk_brute_force(orc):
    rng = np.random.default_rng(3)
    for trial in range(40):
        m = int(rng.integers(1, 300))
        r = np.sort(rng.choice(10 ** 6, size=m, replace=False)).astype(np.uint64)
        # many exact ties and zeros
        c = rng.choice([0.0, 0.5, -0.5, 0.25, 1.0, -1.0, 2.0], size=m) * \
            (1 + (rng.random(m) < 0.3) * rng.random(m))
        k = int(rng.integers(0, m + 5))
        got = orc.topk_indices(r, c, k)
        cand = [i for i in range(m) if c[i] != 0.0]
        cand.sort(key=lambda i: (-abs(c[i]), int(r[i])))
        want = np.sort(np.array(cand[:k], dtype=np.int64))
        assert np.array_equal(got, want)
        rr, cc = orc.truncate_topk(r, c, k)
        assert np.all(np.diff(rr.astype(np.int64)) > 0)
        if cc.size:
            assert abs(np.dot(cc, cc) - 1.0) < 1e-14
