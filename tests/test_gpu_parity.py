"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Bars: bit-exact for ranks, excitation sets and retained index sets; sigma
within 1e-11 of the per-entry magnitude A_k = sum_D |H_kD c_D|; energies
within 1e-9 Ha.
"""
import numpy as np
import pytest

import gen

from conftest import bits_from_string, read_golden

pytestmark = pytest.mark.gpu

SIGMA_TOL = 1e-11


@pytest.fixture(scope="module")
def sf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2312_01846_gb300 as sf
    sf.lib()
    return sf


def _systems(sf, orc, d):
    return sf.System.from_dict(d), orc.System.from_dict(d)


def _vector(orc, sf, gsys, d, count, seed, max_level=2):
    """A near-aufbau vector: ranks from both sides must agree bit for bit."""
    a, b, lev = gen.near_aufbau_dets(d["n"], d["na"], d["nb"], count, seed, max_level=max_level)
    r_or = orc.det_rank(d["n"], d["nb"], a, b)
    r_gpu = sf.to_u64(sf.sfci_rank(gsys, a, b))
    assert np.array_equal(r_or, r_gpu)
    order = np.argsort(r_or)
    c = gen.level_coefs(lev, seed + 1)
    return r_or[order], c[order]


def _check_sigma(sf, orc, gsys, osys, r, c, eps=0.0):
    gr, gv = sf.sfci_sigma(gsys, r, c, eps_screen=eps)
    orank, oval, oabs, _ = orc.sigma(osys, r, c)
    if eps > 0:
        keep = ~(np.abs(oval) < eps)
        gr_u = sf.to_u64(gr)
        # entries within rounding of the screen threshold may fall either way
        near = np.abs(np.abs(oval) - eps) <= SIGMA_TOL * oabs
        must = keep & ~near
        assert np.all(np.isin(orank[must], gr_u))
        assert np.all(np.isin(gr_u, orank[keep | near]))
        return
    assert np.array_equal(sf.to_u64(gr), orank)
    err = np.abs(gv.cpu().numpy() - oval)
    assert np.all(err <= SIGMA_TOL * oabs), err.max()
    return gr, gv, orank, oval, oabs


# ------------------------------------------------------------------ Eq. 12

@pytest.mark.parametrize("cfg", [0, 1])
def test_unrank_rank_exhaustive(sf, orc, cfg):
    d = gen.config_system(cfg)
    gsys = sf.System.from_dict(d)
    r = np.arange(gsys.dim, dtype=np.uint64)
    a, b = sf.sfci_unrank(gsys, r)
    oa, ob = orc.det_unrank(d["n"], d["na"], d["nb"], r)
    assert np.array_equal(sf.to_u64(a), oa) and np.array_equal(sf.to_u64(b), ob)
    assert np.array_equal(sf.to_u64(sf.sfci_rank(gsys, a, b)), r)


def test_table1_order_on_gpu(sf):
    """Table 1: unrank(i) on the GPU is the i-th determinant of the g-chain."""
    chain = [bits_from_string(row[0]) for row in read_golden("table1_gchain_6o3e.txt")]
    gsys = sf.System(6, 3, 0, np.zeros((6, 6)), np.zeros((6,) * 4))
    a, b = sf.sfci_unrank(gsys, np.arange(20, dtype=np.uint64))
    assert sf.to_u64(a).tolist() == chain
    assert sf.to_u64(sf.sfci_rank(gsys, a, b)).tolist() == list(range(20))


def test_rank_sampled_large_spaces(sf, orc):
    for (n, na, nb) in [(28, 7, 7), (64, 5, 3), (40, 12, 11)]:
        gsys = sf.System(n, na, nb, np.zeros((n, n)), np.zeros((n,) * 4))
        rng = np.random.default_rng(n)
        r = np.unique(rng.integers(0, gsys.dim, size=5000, dtype=np.uint64))
        r[-1] = gsys.dim - 1
        a, b = sf.sfci_unrank(gsys, r)
        oa, ob = orc.det_unrank(n, na, nb, r)
        assert np.array_equal(sf.to_u64(a), oa) and np.array_equal(sf.to_u64(b), ob)
        assert np.array_equal(sf.to_u64(sf.sfci_rank(gsys, a, b)), r)
        gsys.close()


def test_rank_rejects_bad_input(sf):
    gsys = sf.System(8, 4, 4, np.zeros((8, 8)), np.zeros((8,) * 4))
    with pytest.raises(sf.SfciError) as e:
        sf.sfci_rank(gsys, np.array([0b111], dtype=np.uint64), np.array([0b1111], dtype=np.uint64))
    assert e.value.status == sf.SFCI_E_INVALID
    with pytest.raises(sf.SfciError) as e:
        sf.sfci_unrank(gsys, np.array([4900], dtype=np.uint64))
    assert e.value.status == sf.SFCI_E_INVALID


# ----------------------------------------------------- excitations, elements

@pytest.mark.parametrize("cfg,count", [(0, 4900), (2, 40), (1, 300)])
def test_excitations_bit_exact(sf, orc, cfg, count):
    d = gen.config_system(cfg)
    gsys, osys = _systems(sf, orc, d)
    n, na, nb = d["n"], d["na"], d["nb"]
    if count >= gsys.dim:
        r = np.arange(gsys.dim, dtype=np.uint64)
    else:
        r, _ = _vector(orc, sf, gsys, d, count, seed=21)
    src, tgt, elem = sf.sfci_debug_excitations(gsys, r)
    src = src.cpu().numpy()
    tgt = sf.to_u64(tgt)
    elem = elem.cpu().numpy()
    per = orc.n_connected(n, na, nb) + 1
    assert src.size == r.size * per
    sa, sb = orc.det_unrank(n, na, nb, r)
    want_t = np.empty(r.size * per, dtype=np.uint64)
    for s in range(r.size):
        ca, cb = orc.connected(n, na, nb, sa[s], sb[s])
        want_t[s * per] = r[s]
        want_t[s * per + 1:(s + 1) * per] = orc.det_rank(n, nb, ca, cb)
    assert np.array_equal(src, np.repeat(np.arange(r.size), per))
    for s in range(r.size):
        g = np.sort(tgt[s * per:(s + 1) * per])
        w = np.sort(want_t[s * per:(s + 1) * per])
        assert np.array_equal(g, w), f"excitation set of source {s} differs"
    ta, tb = orc.det_unrank(n, na, nb, tgt)
    ref = orc.hmat_batch(osys, np.repeat(sa, per), np.repeat(sb, per), ta, tb)
    diff = np.abs(elem - ref)
    assert np.all(diff <= 1e-14 * np.maximum(1.0, np.abs(ref))), diff.max()
    bitwise = np.mean(elem.view(np.uint64) == ref.view(np.uint64))
    print(f"cfg{cfg}: {src.size} elements, bitwise-equal fraction {bitwise:.6f}")


# ------------------------------------------------------------------ sigma

def test_sigma_cfg0_full_vector(sf, orc):
    d = gen.config_system(0)
    gsys, osys = _systems(sf, orc, d)
    rng = np.random.default_rng(3)
    r = np.arange(gsys.dim, dtype=np.uint64)
    c = rng.normal(size=r.size)
    _check_sigma(sf, orc, gsys, osys, r, c)


@pytest.mark.parametrize("count", [1, 31, 33, 257, 1000])
def test_sigma_cfg0_ragged(sf, orc, count):
    d = gen.config_system(0)
    gsys, osys = _systems(sf, orc, d)
    rng = np.random.default_rng(count)
    r = np.sort(rng.choice(gsys.dim, size=count, replace=False)).astype(np.uint64)
    c = rng.normal(size=count)
    _check_sigma(sf, orc, gsys, osys, r, c)


def test_sigma_cfg2_near_aufbau(sf, orc):
    d = gen.config_system(2)
    gsys, osys = _systems(sf, orc, d)
    r, c = _vector(orc, sf, gsys, d, 150, seed=5)
    _check_sigma(sf, orc, gsys, osys, r, c)


def test_sigma_hubbard(sf, orc):
    d = gen.config_system(1)
    gsys, osys = _systems(sf, orc, d)
    r, c = _vector(orc, sf, gsys, d, 2000, seed=8, max_level=3)
    out = _check_sigma(sf, orc, gsys, osys, r, c)
    # only ring hops and the diagonal are non-zero
    assert out[0].numel() <= r.size * 25


def test_sigma_screen(sf, orc):
    d = gen.config_system(0)
    gsys, osys = _systems(sf, orc, d)
    rng = np.random.default_rng(9)
    r = np.sort(rng.choice(gsys.dim, size=600, replace=False)).astype(np.uint64)
    c = rng.normal(size=r.size) * 1e-2
    _check_sigma(sf, orc, gsys, osys, r, c, eps=5e-3)


def test_sigma_edge_cases(sf, orc):
    d = gen.config_system(0)
    gsys, osys = _systems(sf, orc, d)
    gr, gv = sf.sfci_sigma(gsys, np.zeros(0, dtype=np.uint64), np.zeros(0))
    assert gr.numel() == 0
    # all-zero coefficients: no element is generated
    gr, gv = sf.sfci_sigma(gsys, np.array([0, 5], dtype=np.uint64), np.zeros(2))
    assert gr.numel() == 0
    # the last determinant of the space
    _check_sigma(sf, orc, gsys, osys, np.array([gsys.dim - 1], dtype=np.uint64), np.array([0.7]))
    with pytest.raises(sf.SfciError) as e:
        sf.sfci_sigma(gsys, np.array([5, 3], dtype=np.uint64), np.ones(2))
    assert e.value.status == sf.SFCI_E_INVALID
    with pytest.raises(sf.SfciError) as e:
        sf.sfci_sigma(gsys, np.array([gsys.dim], dtype=np.uint64), np.ones(1))
    assert e.value.status == sf.SFCI_E_INVALID


def test_sigma_capacity_is_reported(sf):
    import ctypes as C
    import torch
    d = gen.config_system(0)
    gsys = sf.System.from_dict(d)
    r = torch.arange(100, dtype=torch.int64, device="cuda")
    c = torch.ones(100, dtype=torch.float64, device="cuda")
    cap = 50
    ws = torch.empty(sf.sigma_workspace_bytes(gsys, 100, cap), dtype=torch.uint8, device="cuda")
    orank = torch.empty(cap, dtype=torch.int64, device="cuda")
    ocoef = torch.empty(cap, dtype=torch.float64, device="cuda")
    n = C.c_int64()
    st = sf.lib().sfci_sigma(gsys.handle, sf._ptr(r), sf._ptr(c), 100, 0.0, sf._ptr(orank),
                             sf._ptr(ocoef), cap, C.byref(n), sf._ptr(ws), ws.numel(),
                             sf._stream())
    assert st == sf.SFCI_E_CAPACITY and n.value > cap
    gr, _ = sf.sfci_sigma(gsys, r, c)
    assert n.value == gr.numel() or n.value > 2 * cap


# ---------------------------------------------------------------- top-k

@pytest.mark.parametrize("n,k", [(0, 5), (1, 1), (7, 3), (1000, 100), (100000, 4321),
                                 ((1 << 20) + 3, 100000), (5000, 5000), (5000, 0)])
def test_topk_bit_exact(sf, orc, n, k):
    rng = np.random.default_rng(n + k)
    r = rng.choice(1 << 40, size=n, replace=False).astype(np.uint64) if n else np.zeros(0, np.uint64)
    # many exact ties, exact zeros, both signs, and a wide exponent range
    c = rng.choice([0.0, 1.0, -1.0, 0.5, 2.0, -3e-7, 1e-300], size=n) * \
        np.where(rng.random(n) < 0.5, 1.0, rng.random(n))
    gr, gv = sf.sfci_truncate_topk(r, c, k, normalize=True)
    wr, wv = orc.truncate_topk(r, c, k)
    assert np.array_equal(sf.to_u64(gr), wr)
    if wv.size:
        assert np.allclose(gv.cpu().numpy(), wv, rtol=1e-15, atol=0)
    gr2, gv2 = sf.sfci_truncate_topk(r, c, k, normalize=False)
    idx = orc.topk_indices(r, c, k)
    o = np.argsort(r[idx])
    assert np.array_equal(gv2.cpu().numpy().view(np.uint64), c[idx][o].view(np.uint64))


# ---------------------------------------------------------------- Lanczos

def _gpu_lanczos(sf, gsys, n_keep, n_lanczos, n_iter, eps=0.0, init=None):
    r0 = np.array([0], dtype=np.uint64) if init is None else init[0]
    c0 = np.array([1.0]) if init is None else init[1]
    lz = sf.Lanczos(gsys, r0, c0, n_keep, n_lanczos, max_iter=n_iter, eps_screen=eps)
    infos = [lz.step() for _ in range(n_iter)]
    lz.close()
    return infos


def test_lanczos_untruncated_cfg0(sf, orc):
    d = gen.config_system(0)
    gsys, osys = _systems(sf, orc, d)
    g = _gpu_lanczos(sf, gsys, 4900, 10, 30)
    o = orc.sfci(osys, np.array([0], dtype=np.uint64), np.array([1.0]), 4900, 10, 30)
    eg = [s["lambda_min"] for s in g if s["cycle_end"]]
    eo = [s["lambda"] for s in o if s["lambda"] is not None]
    assert len(eg) == len(eo) == 3
    assert np.max(np.abs(np.array(eg) - np.array(eo))) < 1e-9
    # per step a_i agrees too
    ag = [s["a"] for s in g]
    ao = [s["a"] for s in o]
    assert np.max(np.abs(np.array(ag) - np.array(ao))) < 1e-9


def test_lanczos_truncated_no_spin_symmetry(sf, orc):
    """4 alpha / 3 beta electrons: no spin-flip symmetry, so no exact ties at
    the truncation boundary; the truncated runs agree to 1e-9 Ha."""
    d = dict(gen.molecular_integrals(8, 16, seed=50), n=8, na=4, nb=3)
    gsys, osys = _systems(sf, orc, d)
    g = _gpu_lanczos(sf, gsys, 300, 10, 30)
    o = orc.sfci(osys, np.array([0], dtype=np.uint64), np.array([1.0]), 300, 10, 30)
    eg = np.array([s["lambda_min"] for s in g if s["cycle_end"]])
    eo = np.array([s["lambda"] for s in o if s["lambda"] is not None])
    print("truncated 4a/3b energies gpu-oracle:", eg - eo)
    assert eg.size == eo.size == 3
    assert np.max(np.abs(eg - eo)) < 1e-9
    # no ties at the cut: every step keeps the same number of entries and a_i
    # agrees step by step
    kept_g = [s["n_kept"] for s in g if not s["cycle_end"]]
    kept_o = [s["n_kept"] for s in o if "n_kept" in s]
    assert kept_g == kept_o
    ag = np.array([s["a"] for s in g])
    ao = np.array([s["a"] for s in o])
    assert np.max(np.abs(ag - ao)) < 1e-9


def test_sigma_sums_exact_and_repeatable(sf, orc):
    """Every sigma entry is the exactly rounded sum of its products
    fl(<D'|H|D> c_D): checked with rational arithmetic on sampled entries, and
    two calls agree bit for bit."""
    from fractions import Fraction
    d = gen.config_system(0)
    gsys, osys = _systems(sf, orc, d)
    rng = np.random.default_rng(12)
    r = np.sort(rng.choice(gsys.dim, size=700, replace=False)).astype(np.uint64)
    c = rng.normal(size=r.size) * np.exp(rng.normal(size=r.size))
    gr1, gv1 = sf.sfci_sigma(gsys, r, c)
    gr2, gv2 = sf.sfci_sigma(gsys, r, c)
    k1, v1 = sf.to_u64(gr1), gv1.cpu().numpy()
    assert np.array_equal(k1, sf.to_u64(gr2))
    assert np.array_equal(v1.view(np.uint64), gv2.cpu().numpy().view(np.uint64))
    src, tgt, elem = sf.sfci_debug_excitations(gsys, r)
    src = src.cpu().numpy()
    tgt = sf.to_u64(tgt)
    prod = elem.cpu().numpy() * c[src]          # the float64 products (one rounding each)
    keep = prod != 0.0
    tgt, prod = tgt[keep], prod[keep]
    order = np.argsort(tgt, kind="stable")
    tgt, prod = tgt[order], prod[order]
    uk, start = np.unique(tgt, return_index=True)
    assert np.array_equal(uk, k1)
    ends = np.append(start[1:], tgt.size)
    for i in rng.choice(uk.size, size=min(300, uk.size), replace=False):
        exact = sum((Fraction(float(x)) for x in prod[start[i]:ends[i]]), Fraction(0))
        assert float(exact) == v1[i], (i, float(exact), v1[i])
