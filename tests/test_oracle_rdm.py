"""Pins for the oracle's one- and two-particle density matrices."""
import numpy as np

import gen


def test_rdm_traces_and_energy(orc):
    n, na, nb = 6, 3, 2
    d = gen.molecular_integrals(n, 5, seed=11)
    S = orc.System(n, na, nb, d["h"], d["g"], e_core=0.3)
    dimv = orc.dim(n, na, nb)
    rng = np.random.default_rng(12)
    r = np.sort(rng.choice(dimv, size=90, replace=False)).astype(np.uint64)
    c = rng.normal(size=r.size)
    g1, g2 = orc.rdm12(S, r, c)
    nn = float(np.dot(c, c))
    N = na + nb
    assert abs(np.trace(g1) - N * nn) < 1e-11
    assert abs(np.einsum("pprr->", g2) - N * (N - 1) * nn) < 1e-10
    assert np.allclose(g1, g1.T, atol=1e-12)
    # <psi|H|psi> from the dense matrix
    H = orc.dense_h(S)
    x = np.zeros(dimv)
    x[r.astype(np.int64)] = c
    e_ref = x @ H @ x
    e_rdm = 0.3 * nn + np.einsum("pq,pq->", d["h"], g1) + 0.5 * np.einsum("pqrs,pqrs->", d["g"], g2)
    assert abs(e_ref - e_rdm) < 1e-10 * max(1.0, abs(e_ref))
