"""Bucketed sigma with more alpha strings than the row map holds (C(36, 9) =
9.4e7 > 2^26): buckets by a hash of the full rank with equal regions, no
alpha-row plan.  A truncated Lanczos run against the oracle's, from the
aufbau determinant.

The sigma sums are exact (fixed point) on the GPU and ascending-source FP64
sums in the oracle; both round to the same doubles up to the oracle's own
sequential rounding, so the energies and the coefficients a_i agree to 1e-9.
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


def test_hash_buckets_against_oracle(sf, orc):
    d = dict(gen.molecular_integrals(36, 8, seed=61), n=36, na=9, nb=8)
    g, o = sf.System.from_dict(d), orc.System.from_dict(d)
    n_keep, n_lanczos, n_iter = 50, 4, 8
    lz = sf.Lanczos(g, np.array([0], dtype=np.uint64), np.array([1.0]), n_keep, n_lanczos, max_iter=n_iter)
    infos = [lz.step() for _ in range(n_iter)]
    lz.close()
    st = orc.sfci(o, np.array([0], dtype=np.uint64), np.array([1.0]), n_keep, n_lanczos, n_iter)
    a_g = np.array([i["a"] for i in infos])
    a_o = np.array([s["a"] for s in st])
    l_g = np.array([i["lambda_min"] for i in infos if i["cycle_end"]])
    l_o = np.array([s["lambda"] for s in st if s["lambda"] is not None])
    print("elements per step", [i["n_elements"] for i in infos])
    print("lambda gpu - oracle", l_g - l_o)
    assert max(i["n_buckets_log2"] for i in infos) >= 4
    assert l_g.size == l_o.size == 2
    assert np.max(np.abs(a_g - a_o)) < 1e-9
    assert np.max(np.abs(l_g - l_o)) < 1e-9
