"""SFCI_FP32_ELEMENTS against the float64 oracle.

In this mode singles and doubles are evaluated from float32 copies of h and g
with float32 sums; the diagonal, the product with c_D, the accumulation of
sigma, the dots and the eigensolve stay float64.  The bars follow from float32
rounding (u = 2^-24):

- an off-diagonal element is a float32 sum of K <= 1 + N + max(na, nb)
  float32-rounded terms, so |e32 - e64| <= (K + 1) u sum|terms|
  <= (K + 1) u (max|h| + (K - 1) max|g|) =: eps_e;
- the diagonal is the float64 value, bit for bit, and every target index is
  the same integer as in float64;
- sigma: |s32_k - s64_k| <= eps_e sum_D |c_D| + 1e-11 A_k;
- energies: for any vector x, |<x|H32|x> - <x|H64|x>| <= ||H32 - H64||_2 <x|x>,
  with ||X||_2 <= sqrt(||X||_1 ||X||_inf) from the element differences.
"""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def sf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2312_01846_gb300 as sf
    sf.lib()
    return sf


def _eps_e(d):
    na, nb = d["na"], d["nb"]
    K = 1 + na + nb + max(na, nb)
    return (K + 1) * U32 * (np.abs(d["h"]).max() + (K - 1) * np.abs(d["g"]).max())


def _near_aufbau(orc, d, count, seed):
    a, b, lev = gen.near_aufbau_dets(d["n"], d["na"], d["nb"], count, seed, max_level=2)
    r = orc.det_rank(d["n"], d["nb"], a, b)
    o = np.argsort(r)
    return r[o], gen.level_coefs(lev, seed + 1)[o]


@pytest.mark.parametrize("cfg,count", [(0, 4900), (2, 40), (1, 300)])
def test_fp32_elements_within_bound(sf, orc, cfg, count):
    d = gen.config_system(cfg)
    g32 = sf.System.from_dict(d, flags=sf.SFCI_FP32_ELEMENTS)
    osys = orc.System.from_dict(d)
    n, na, nb = d["n"], d["na"], d["nb"]
    r = np.arange(g32.dim, dtype=np.uint64) if count >= g32.dim else _near_aufbau(orc, d, count, 61)[0]
    src, tgt, elem = sf.sfci_debug_excitations(g32, r)
    src, tgt, elem = src.cpu().numpy(), sf.to_u64(tgt), elem.cpu().numpy()
    per = g32.n_conn + 1
    sa, sb = orc.det_unrank(n, na, nb, r)
    ta, tb = orc.det_unrank(n, na, nb, tgt)
    ref = orc.hmat_batch(osys, np.repeat(sa, per), np.repeat(sb, per), ta, tb)
    diag = tgt == r[src]
    assert diag.sum() == r.size
    # the diagonal is float64: identical to the oracle's ordered sum
    assert np.array_equal(elem[diag].view(np.uint64), ref[diag].view(np.uint64))
    err = np.abs(elem - ref)[~diag]
    bound = _eps_e(d)
    print(f"cfg{cfg}: max |e32 - e64| = {err.max():.3e}, bound {bound:.3e}")
    assert np.all(err <= bound)


@pytest.mark.parametrize("cfg,count", [(0, 4900), (2, 40)])
def test_fp32_sigma_within_bound(sf, orc, cfg, count):
    d = gen.config_system(cfg)
    g32 = sf.System.from_dict(d, flags=sf.SFCI_FP32_ELEMENTS)
    osys = orc.System.from_dict(d)
    if count >= g32.dim:
        r = np.arange(g32.dim, dtype=np.uint64)
        c = np.random.default_rng(62).normal(size=r.size)
    else:
        r, c = _near_aufbau(orc, d, count, 63)
    gr, gv = sf.sfci_sigma(g32, r, c)
    orank, oval, oabs, _ = orc.sigma(osys, r, c)
    assert np.array_equal(sf.to_u64(gr), orank)
    err = np.abs(gv.cpu().numpy() - oval)
    tol = _eps_e(d) * np.abs(c).sum() + 1e-11 * oabs
    print(f"cfg{cfg}: max sigma error {err.max():.3e}")
    assert np.all(err <= tol)


def _sparse_dot_sigma(sf, sys, r, c):
    """<psi|H|psi> through sfci_sigma: sigma on psi's support, dotted with c."""
    import torch
    sr, sv = sf.sfci_sigma(sys, r, c)
    rd = torch.from_numpy(np.ascontiguousarray(r).view(np.int64)).cuda()
    idx = torch.searchsorted(sr, rd).clamp(max=sr.numel() - 1)
    hit = sr[idx] == rd
    cd = torch.from_numpy(np.ascontiguousarray(c)).cuda()
    return float((cd[hit] * sv[idx[hit]]).sum().item())


def test_fp32_rayleigh_quotient_bound_cfg0(sf, orc):
    """For any vector x, |<x|H32|x> - <x|H64|x>| <= ||H32 - H64||_2 <x|x>.
    The float32-element solver's vector after 40 untruncated steps: its
    float32 and float64 Rayleigh quotients obey that bound, the float64 one
    lies above the lowest eigenvalue, and the solver's lambda_min tracks the
    float64 solver's at every cycle end."""
    import scipy.sparse as sp
    d = gen.config_system(0)
    g32 = sf.System.from_dict(d, flags=sf.SFCI_FP32_ELEMENTS)
    g64 = sf.System.from_dict(d)
    osys = orc.System.from_dict(d)
    r = np.arange(g32.dim, dtype=np.uint64)
    s32, t32, e32 = sf.sfci_debug_excitations(g32, r)
    s64, t64, e64 = sf.sfci_debug_excitations(g64, r)
    assert np.array_equal(t32.cpu().numpy(), t64.cpu().numpy())
    X = sp.coo_matrix(((e32 - e64).cpu().numpy(), (sf.to_u64(t32).astype(np.int64), s32.cpu().numpy())),
                      shape=(g32.dim, g32.dim)).tocsr()
    absX = abs(X)
    norm2 = float(np.sqrt(absX.sum(axis=0).max() * absX.sum(axis=1).max()))
    lams = {}
    for name, g in (("f32", g32), ("f64", g64)):
        lz = sf.Lanczos(g, np.array([0], dtype=np.uint64), np.array([1.0]), 4900, 10, max_iter=40)
        lams[name] = [i["lambda_min"] for i in (lz.step() for _ in range(40)) if i["cycle_end"]]
        if name == "f32":
            vr, vc = lz.vector()
            vr, vc = sf.to_u64(vr), vc.cpu().numpy()
        lz.close()
    nrm = float(np.dot(vc, vc))
    rho32 = _sparse_dot_sigma(sf, g32, vr, vc) / nrm
    rho64 = _sparse_dot_sigma(sf, g64, vr, vc) / nrm
    e_min = float(np.linalg.eigvalsh(orc.dense_h(osys))[0])
    dl = np.array(lams["f32"]) - np.array(lams["f64"])
    print(f"||dH||_2 <= {norm2:.3e}; rho32 - rho64 = {rho32 - rho64:.3e}; "
          f"lambda32 - lambda64 per cycle: {dl}")
    assert abs(rho32 - rho64) <= norm2 + 1e-12 * abs(rho64)
    assert rho64 >= e_min - 1e-9
    assert np.all(np.abs(dl) <= 2 * norm2)
