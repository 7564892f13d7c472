"""GPU density matrices (sfci_rdm12) and the autograd adjoint, against the oracle.

The energy of a fixed vector is linear in h and (pq|rs), so central finite
differences along any direction are exact up to rounding; the gradients from
the RDMs must match them, and the RDMs themselves must match the oracle's
operator-application RDMs element by element.
"""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2312_01846_gb300 as sf
    sf.lib()
    return sf


def _rand_vec(orc, dimv, m, seed):
    rng = np.random.default_rng(seed)
    r = np.sort(rng.choice(dimv, size=m, replace=False)).astype(np.uint64)
    return r, rng.normal(size=m)


@pytest.mark.parametrize("n,na,nb,m", [(6, 3, 2, 90), (8, 4, 4, 300), (5, 1, 3, 40), (7, 0, 3, 30)])
def test_rdm_matches_oracle(sf, orc, n, na, nb, m):
    d = gen.molecular_integrals(n, 4, seed=n * 10 + na)
    gsys = sf.System(n, na, nb, d["h"], d["g"])
    osys = orc.System(n, na, nb, d["h"], d["g"])
    r, c = _rand_vec(orc, gsys.dim, min(m, gsys.dim), seed=n + m)
    g1, g2, nrm = sf.sfci_rdm12(gsys, r, c)
    o1, o2 = orc.rdm12(osys, r, c)
    assert abs(nrm - np.dot(c, c)) < 1e-12 * np.dot(c, c)
    assert np.allclose(g1.cpu().numpy(), o1, rtol=0, atol=1e-12 * max(1, np.abs(o1).max()))
    assert np.allclose(g2.cpu().numpy(), o2, rtol=0, atol=1e-12 * max(1, np.abs(o2).max()))


def _oracle_energy(orc, osys, r, c):
    """<psi|H|psi> / <psi|psi> with sigma pulled entry by entry on psi's support."""
    val, _, _ = orc.sigma_entries(osys, r, c, r)
    return float(np.dot(c, val) / np.dot(c, c))


def test_rdm_cfg4_energy_and_finite_differences(sf, orc):
    import torch
    d = gen.config_system(4)
    n = d["n"]
    gsys, osys = sf.System.from_dict(d), orc.System.from_dict(d)
    a, b, lev = gen.near_aufbau_dets(n, 5, 5, 4000, seed=41)
    r = orc.det_rank(n, 5, a, b)
    o = np.argsort(r)
    r, c = r[o], gen.level_coefs(lev, 42)[o]
    g1, g2, nrm = sf.sfci_rdm12(gsys, r, c)
    g1n, g2n = g1.cpu().numpy(), g2.cpu().numpy()
    N = 10
    assert abs(np.trace(g1n) - N * nrm) < 1e-10 * nrm
    assert abs(np.einsum("pprr->", g2n) - N * (N - 1) * nrm) < 1e-9 * nrm
    e_rdm = (np.einsum("pq,pq->", d["h"], g1n) + 0.5 * np.einsum("pqrs,pqrs->", d["g"], g2n)) / nrm
    e_or = _oracle_energy(orc, osys, r, c)
    assert abs(e_rdm - e_or) < 1e-9
    # autograd gradients vs central differences of the oracle energy, step 1e-5,
    # along symmetric directions (h and the 8-fold symmetric g)
    h_t = torch.tensor(d["h"], device="cuda", requires_grad=True)
    g_t = torch.tensor(d["g"], device="cuda", requires_grad=True)
    e = sf.RayleighEnergy.apply(h_t, g_t, gsys, r, c, 0.0)
    assert abs(e.item() - e_or) < 1e-9  # the library's contraction (sfci_rdm_energy)
    e.backward()
    gh, gg = h_t.grad.cpu().numpy(), g_t.grad.cpu().numpy()
    rng = np.random.default_rng(43)
    for trial in range(2):
        dh = rng.normal(size=(n, n))
        dh = dh + dh.T
        dB = rng.normal(size=(2, n, n))
        dB = dB + np.transpose(dB, (0, 2, 1))
        dg = gen.factor_to_eri(dB)
        step = 1e-5
        ep = _oracle_energy(orc, orc.System(n, 5, 5, d["h"] + step * dh, d["g"] + step * dg), r, c)
        em = _oracle_energy(orc, orc.System(n, 5, 5, d["h"] - step * dh, d["g"] - step * dg), r, c)
        fd = (ep - em) / (2 * step)
        ad = np.sum(gh * dh) + np.sum(gg * dg)
        assert abs(fd - ad) < 1e-6 * max(1.0, abs(fd)), (fd, ad)


def test_factor_gradient_on_sfci_vector(sf):
    """cfg4 workload: a sparse vector from a GPU SFCI run, dE/dB through
    g = sum_L B^L (x) B^L by autograd, against central differences of the
    sigma-based energy <psi|H psi>/<psi|psi> (a different kernel path)."""
    import torch
    d = gen.config_system(4)
    n = d["n"]
    gsys = sf.System.from_dict(d)
    lz = sf.Lanczos(gsys, np.array([0], dtype=np.uint64), np.array([1.0]), 300_000, 10)
    for _ in range(12):
        lz.step()
    r, c = lz.vector()
    lz.close()
    assert r.numel() > 100_000
    B = torch.tensor(d["B"], device="cuda", requires_grad=True)
    h_t = torch.tensor(d["h"], device="cuda", requires_grad=True)
    g_t = torch.einsum("lpq,lrs->pqrs", B, B)
    e = sf.RayleighEnergy.apply(h_t, g_t, gsys, r, c, 0.0)
    e.backward()
    gB = B.grad.cpu().numpy()

    def e_sigma(Bnp):
        g = gen.factor_to_eri(Bnp)
        s2 = sf.System(n, 5, 5, d["h"], g)
        sr, sv = sf.sfci_sigma(s2, r, c, out_cap=40_000_000)
        idx = torch.searchsorted(sr, r)
        idx = idx.clamp(max=sr.numel() - 1)
        hit = sr[idx] == r
        num = (c[hit] * sv[idx[hit]]).sum().item()
        s2.close()
        return num / (c * c).sum().item()

    rng = np.random.default_rng(44)
    for (l, p, q) in [(0, 0, 0), (3, 2, 7), (63, 19, 4)]:
        step = 1e-5
        Bp = d["B"].copy()
        Bm = d["B"].copy()
        for (x, y) in {(p, q), (q, p)}:
            Bp[l, x, y] += step
            Bm[l, x, y] -= step
        fd = (e_sigma(Bp) - e_sigma(Bm)) / (2 * step)
        ad = gB[l, p, q] + (gB[l, q, p] if p != q else 0.0)
        assert abs(fd - ad) < 1e-6 * max(1.0, abs(fd)), (l, p, q, fd, ad)
    _ = rng
