"""Alpha-alpha doubles by runs of sources that share alpha.

The sources of sigma are sorted by rank, alpha-major, so determinants with one
alpha string are consecutive.  When a sigma pass leaves rows to other passes,
or the runs average two sources or more, the alpha-alpha doubles are emitted
by a kernel of their own that takes each run's excitations once and pairs
them with the run's beta strings; otherwise the main emit kernel emits them
per source.  Both must give sigma exactly (Eqs. 10-11).  Three input vectors
of the 20-orbital 5a/5b system:
  - runs of 40, 7, 3 and 1 determinants in one pass (run kernel, windows with
    L = 32 and ragged runs), replayed step by step by the oracle (sigma, T
    and S columns, a, b, the kept set);
  - the same vector under a small device budget, so sigma takes several
    passes (run kernel, rows of other passes skipped): the same a, b, counts
    and kept vectors as the one-pass run (every sigma entry is an exact sum
    rounded once);
  - one determinant per alpha string in one pass (per-source path), replayed.
The step info's run count must equal the count of rank // C(n, n_beta) changes.
"""
import numpy as np
import pytest

import gen
from test_gpu_replay import Replay, _vec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2312_01846_gb300 as sf
    sf.lib()
    return sf


def _runs(rank, cb):
    a = rank // np.uint64(cb)
    return int(1 + np.count_nonzero(a[1:] != a[:-1])) if a.size else 0


def _vector(d, layout, seed):
    """Ranks with the given (alpha count, run length) layout, alpha strings and
    beta columns drawn at random (seeded), coefficients uniform in +-[0.1, 1]."""
    from math import comb
    rng = np.random.default_rng(seed)
    ca, cb = comb(d["n"], d["na"]), comb(d["n"], d["nb"])
    n_alpha = sum(k for k, _ in layout)
    alphas = rng.choice(ca, size=n_alpha, replace=False)
    ranks, pos = [], 0
    for k, length in layout:
        for a in alphas[pos:pos + k]:
            cols = rng.choice(cb, size=length, replace=False)
            ranks.append(np.uint64(a) * np.uint64(cb) + cols.astype(np.uint64))
        pos += k
    r = np.unique(np.concatenate(ranks))
    c = rng.uniform(0.1, 1.0, r.size) * rng.choice([-1.0, 1.0], r.size)
    return r, c, cb


def _run(sf, orc, d, r, c, n_keep, steps, label, replay=True, **kw):
    """step infos and the vector after each step; each step replayed by the
    oracle when replay is set"""
    gsys, osys = sf.System.from_dict(d), orc.System.from_dict(d)
    lz = sf.Lanczos(gsys, r, c, n_keep, 10, **kw)
    rp = Replay(orc, osys, _vec(sf, lz), n_keep, 10, label) if replay else None
    infos, vecs = [], []
    for _ in range(steps):
        info = lz.step()
        vecs.append(_vec(sf, lz))
        if rp is not None:
            Tg, Sg = lz.matrices()
            rp.step(info, Tg, Sg, vecs[-1])
        infos.append(info)
    lz.close()
    gsys.close()
    return infos, vecs


def test_runs_one_pass_and_passes(sf, orc):
    d = gen.config_system(4)
    r, c, cb = _vector(d, [(30, 40), (40, 7), (60, 3), (300, 1)], seed=11)
    n_keep = 2500
    assert r.size < n_keep  # w_0 is the whole input, normalised
    steps = 3
    one, v_one = _run(sf, orc, d, r, c, n_keep, steps, "runs, one pass")
    assert one[0]["n_passes"] == 1
    assert one[0]["n_alpha_runs"] == _runs(r, cb)
    assert r.size >= 2 * one[0]["n_alpha_runs"]  # the run kernel's case
    # a budget that needs several passes: 0.6, 0.45 or 0.3 of the first sigma's
    # regions, plus room for sigma's stream buffer and the overflow lists
    regions = one[0]["regions_gb"] * 1e9
    multi = None
    for frac in (0.6, 0.45, 0.3):
        try:
            multi, v_multi = _run(sf, orc, d, r, c, n_keep, steps, f"runs, budget {frac}", replay=False,
                                  mem_budget=int(regions * frac) + (96 << 20), ovf_max_log2=18)
        except sf.SfciError:
            continue
        if multi[0]["n_passes"] >= 2:
            break
    assert multi is not None and multi[0]["n_passes"] >= 2, "no budget gave several passes"
    print("passes per step:", [i["n_passes"] for i in multi])
    for key in ("a", "b", "n_sigma", "n_kept"):
        x = np.array([i[key] for i in one], dtype=float)
        y = np.array([i[key] for i in multi], dtype=float)
        assert np.allclose(x, y, rtol=1e-12, atol=0), key
    for (r1, c1), (r2, c2) in zip(v_one, v_multi):
        assert np.array_equal(r1, r2)
        assert np.allclose(c1, c2, rtol=1e-12, atol=0)


def test_one_source_per_alpha(sf, orc):
    d = gen.config_system(4)
    r, c, cb = _vector(d, [(800, 1)], seed=12)
    infos, _ = _run(sf, orc, d, r, c, 2500, 2, "one source per alpha")
    assert infos[0]["n_passes"] == 1
    assert infos[0]["n_alpha_runs"] == r.size == _runs(r, cb)
