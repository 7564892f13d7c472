"""Memory passes of the bucketed sigma: the same Lanczos run with everything in
one pass, with the merge buckets spread over several passes (a small device
budget), and with an overflow list too short for a pass (so passes are split
into pieces and emitted again) must give the same numbers.

Each sigma entry is an exact fixed-point sum rounded once, and the kept set is
the exact top N_d with ties to the smaller rank, so neither the pass layout nor
the order in which elements arrive changes sigma; the coefficients a, b and
the energies agree to 1e-12 relative (the dots are FP64 reductions).
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


def _run(sf, gsys, n_keep, steps, **kw):
    lz = sf.Lanczos(gsys, np.array([0], dtype=np.uint64), np.array([1.0]), n_keep, 10, **kw)
    infos = [lz.step() for _ in range(steps)]
    r, c = lz.vector()
    lz.close()
    return infos, sf.to_u64(r), c.cpu().numpy()


def test_passes_and_splits_change_nothing(sf):
    d = gen.config_system(2)
    gsys = sf.System.from_dict(d)
    n_keep, steps = 20_000, 12
    one, r1, c1 = _run(sf, gsys, n_keep, steps)
    assert max(i["n_passes"] for i in one) == 1
    # element regions of the full-size steps are ~10 GB: a 3 GB budget needs passes
    multi, r2, c2 = _run(sf, gsys, n_keep, steps, mem_budget=3 << 30)
    p2 = [i["n_passes"] for i in multi]
    ovf = [i["n_overflow"] for i in multi]
    print("passes (budget)", p2)
    print("overflow of the largest pass", ovf)
    # a list limit of about a third of the largest pass's overflow: the passes
    # that overflow most are split into a few pieces
    lim = max(int(np.log2(max(ovf) / 3.0)), 10)
    split, r3, c3 = _run(sf, gsys, n_keep, steps, mem_budget=3 << 30, ovf_max_log2=lim)
    p3 = [i["n_passes"] for i in split]
    print(f"passes (budget + overflow list of 2^{lim})", p3)
    assert max(p2) >= 3
    assert any(b > a for a, b in zip(p2, p3))  # some pass was split
    for other in (multi, split):
        for key in ("a", "b"):
            x = np.array([i[key] for i in one])
            y = np.array([i[key] for i in other])
            assert np.max(np.abs(x - y) / np.maximum(np.abs(x), 1e-300)) < 1e-12, key
        lx = np.array([i["lambda_min"] for i in one if i["cycle_end"]])
        ly = np.array([i["lambda_min"] for i in other if i["cycle_end"]])
        assert lx.size == ly.size == 1
        assert np.max(np.abs(lx - ly)) < 1e-12 * np.max(np.abs(lx))
    for r, c in ((r2, c2), (r3, c3)):
        assert np.array_equal(r, r1)
        assert np.allclose(c, c1, rtol=1e-12, atol=0)


def test_overflow_limit_too_small_is_reported(sf):
    """A list limit that no split can satisfy ends the step with SFCI_E_CAPACITY
    and a message naming the overflow list."""
    d = gen.config_system(2)
    gsys = sf.System.from_dict(d)
    lz = sf.Lanczos(gsys, np.array([0], dtype=np.uint64), np.array([1.0]), 20_000, 10,
                    mem_budget=3 << 30, ovf_max_log2=1)
    with pytest.raises(sf.SfciError) as ei:
        for _ in range(6):
            lz.step()
    lz.close()
    assert ei.value.status == sf.SFCI_E_CAPACITY
    assert "overflow list" in str(ei.value)


def test_big_bucket_fallback_is_exact(sf):
    """The automatic bucket size's fallback, forced: with
    SFCI_LZ_FALLBACK_STRESS every sigma first tries 2048-element buckets in
    1024-slot tables.  From the aufbau determinant most of sigma's entries are
    distinct, so buckets with more than 1024 of them do not fit and those
    sigmas are redone with 1024-element buckets (info["bucket_redo"]).  The
    run must equal, bit for bit, a run with 1024-element buckets throughout
    (exact sums, exact top-N_d)."""
    d = gen.config_system(2)
    gsys = sf.System.from_dict(d)
    n_keep, steps = 20_000, 12
    ref, r1, c1 = _run(sf, gsys, n_keep, steps, bucket_elems=1024)
    big, r2, c2 = _run(sf, gsys, n_keep, steps, flags=sf.SFCI_LZ_FALLBACK_STRESS)
    redo = [i["bucket_redo"] for i in big]
    print("sigmas redone with 1024-element buckets per step:", redo)
    assert sum(redo) >= 1
    assert all(i["bucket_redo"] == 0 for i in ref)
    for key in ("a", "b", "lambda_min", "n_sigma", "n_kept"):
        assert [i[key] for i in ref] == [i[key] for i in big], key
    assert np.array_equal(r1, r2)
    assert np.array_equal(c1.view(np.uint64), c2.view(np.uint64))
