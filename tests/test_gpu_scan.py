"""Batched scan (sfci_scan_*): instances stepped together must give what each
instance gives on its own, and, untruncated, what the oracle gives.

The scan only changes where and when each instance's kernels run (its own
stream, a worker thread); the arithmetic is the solver's, with exact sigma
sums, so the scan repeats the one-at-a-time run.  Energies agree to 1e-9 Ha
untruncated and, truncated, to 1e-8 Ha over the cycles compared (the bars
leave room for the float64 dots).
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


def _lams(infos):
    return [i["lambda_min"] for i in infos if i["cycle_end"]]


def _small_instances():
    """Uneven full-space instances: (n, na, nb, seed) with dim <= 4900."""
    out = []
    for (n, na, nb, seed) in [(8, 4, 4, 0), (7, 3, 2, 71), (8, 3, 3, 72), (6, 2, 3, 73), (9, 2, 2, 74)]:
        d = gen.molecular_integrals(n, 8, seed=seed)
        out.append(dict(d, n=n, na=na, nb=nb))
    return out


def test_scan_untruncated_matches_single_and_oracle(sf, orc):
    ds = _small_instances()
    systems = [sf.System.from_dict(d) for d in ds]
    n_iter = 20
    inst = [(s, np.array([0], dtype=np.uint64), np.array([1.0]), s.dim) for s in systems]
    sc = sf.Scan(inst, n_lanczos=10, max_iter=n_iter, workers=3)
    steps = [sc.step() for _ in range(n_iter)]
    sc.close()
    for k, (d, s) in enumerate(zip(ds, systems)):
        lam_scan = _lams([st[k] for st in steps])
        lz = sf.Lanczos(s, np.array([0], dtype=np.uint64), np.array([1.0]), s.dim, 10, max_iter=n_iter)
        lam_one = _lams([lz.step() for _ in range(n_iter)])
        lz.close()
        assert len(lam_scan) == len(lam_one) == 2
        assert np.max(np.abs(np.array(lam_scan) - np.array(lam_one))) < 1e-9
        if k == 0:
            o = orc.sfci(orc.System.from_dict(d), np.array([0], dtype=np.uint64), np.array([1.0]),
                         s.dim, 10, n_iter)
            lam_or = [x["lambda"] for x in o if x["lambda"] is not None]
            assert np.max(np.abs(np.array(lam_scan) - np.array(lam_or))) < 1e-9


def test_scan_truncated_uneven_instances(sf):
    """Three uneven instances with reduced caps, integrals interpolated between
    two seeded sets as in the batched-scan generator, scan vs one at a time.
    n_alpha != n_beta: with equal counts, spin-flip partners have exactly equal
    |c|, and which partner survives a cut at such a tie depends on rounding, so
    truncated runs could not be compared entry for entry."""
    A = gen.molecular_integrals(12, 16, seed=31)
    Bs = gen.molecular_integrals(12, 16, seed=32)
    pick = []
    for (n, na, nb, lam) in [(10, 4, 3, 0.0), (12, 5, 4, 0.5), (9, 3, 2, 1.0)]:
        h = (1 - lam) * A["h"] + lam * Bs["h"]
        g = (1 - lam) * A["g"] + lam * Bs["g"]
        pick.append(dict(h=np.ascontiguousarray(h[:n, :n]), g=np.ascontiguousarray(g[:n, :n, :n, :n]),
                         e_core=0.0, n=n, na=na, nb=nb))
    caps = [3000, 1500, 2500]
    systems = [sf.System.from_dict(d) for d in pick]
    n_iter = 20
    inst = [(s, np.array([0], dtype=np.uint64), np.array([1.0]), c) for s, c in zip(systems, caps)]
    sc = sf.Scan(inst, n_lanczos=10, max_iter=n_iter)
    steps = [sc.step() for _ in range(n_iter)]
    vec = [sc.vector(k) for k in range(3)]
    sc.close()
    for k, s in enumerate(systems):
        infos_scan = [st[k] for st in steps]
        assert all(x["n_in"] <= caps[k] for x in infos_scan)
        lz = sf.Lanczos(s, np.array([0], dtype=np.uint64), np.array([1.0]), caps[k], 10, max_iter=n_iter)
        lam_one = _lams([lz.step() for _ in range(n_iter)])
        lz.close()
        lam_scan = _lams(infos_scan)
        print(f"instance {k}: n={pick[k]['n']} {pick[k]['na']}a{pick[k]['nb']}b cap={caps[k]} "
              f"scan-single {np.array(lam_scan) - np.array(lam_one)}")
        assert np.max(np.abs(np.array(lam_scan) - np.array(lam_one))) < 1e-8
        r, c = vec[k]
        assert r.numel() <= caps[k] and abs(float((c * c).sum()) - 1.0) < 1e-12


def test_scan_all_instances_replayed_by_oracle(sf, orc):
    """The 32-instance batched-scan workload (n 16-24, 5a5b-8a8b, integrals
    interpolated between two seeded sets) with the caps reduced 2000-fold
    (5-100 determinants, so the oracle keeps up): every step of every instance,
    stepped together by sfci_scan, is replayed by the oracle on that
    instance's own vectors, as in test_gpu_replay (sigma, T and S columns,
    a_i, b_i, the kept set up to the cut, cycle-end energies within 1e-9 Ha)."""
    from test_gpu_replay import Replay
    ds = gen.batched_scan_instances()
    caps = [max(30, d["cap"] // 2000) for d in ds]
    systems = [sf.System.from_dict(d) for d in ds]
    n_lanczos, n_iter = 4, 8
    inst = [(s, np.array([0], dtype=np.uint64), np.array([1.0]), c) for s, c in zip(systems, caps)]
    sc = sf.Scan(inst, n_lanczos=n_lanczos, max_iter=n_iter)

    def vec(k):
        r, c = sc.vector(k)
        return sf.to_u64(r).copy(), c.cpu().numpy().copy()

    reps = [Replay(orc, orc.System.from_dict(d), vec(k), caps[k], n_lanczos, f"instance {k}")
            for k, d in enumerate(ds)]
    for _ in range(n_iter):
        infos = sc.step()
        for k, rp in enumerate(reps):
            Tg, Sg = sc.matrices(k)
            rp.step(infos[k], Tg, Sg, vec(k))
    sc.close()
    for s in systems:
        s.close()
    assert all(rp.n_cycles == 2 for rp in reps)
    print("cycle-end energies per instance:", [rp.energies for rp in reps])
    print("kept-set differences at the cut:", [rp.n_diff for rp in reps])
