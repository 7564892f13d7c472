"""Pins for the oracle's one- and two-particle density matrices."""
import itertools

import numpy as np
import pytest

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


def _jw_apply(ops, state):
    """Apply (spin_orbital, is_creator) operators right to left to an
    occupation-number state (spin orbitals alpha 0..n-1, then beta 0..n-1,
    Jordan-Wigner order); returns (sign, state), sign 0 when it vanishes."""
    sign = 1
    for so, dag in reversed(ops):
        if ((state >> so) & 1) == dag:
            return 0, 0
        if bin(state & ((1 << so) - 1)).count("1") & 1:
            sign = -sign
        state ^= 1 << so
    return sign, state


@pytest.mark.parametrize("n,na,nb,seed", [(3, 2, 1, 21), (4, 2, 2, 22), (4, 3, 1, 23), (4, 1, 2, 24)])
def test_rdm_elements_equal_operator_expectations(orc, n, na, nb, seed):
    """Every element of the oracle's gamma and Gamma against the definition
    gamma_pq = sum_s <psi|a+_ps a_qs|psi>, Gamma_pqrs = sum_st <psi|a+_ps a+_rt
    a_st a_qs|psi>, evaluated by applying the operators to each determinant of
    a random psi in second quantisation (no Slater-Condon rules, no symmetry
    of the indices assumed).  A transposed pair (pq) or (rs), or Gamma_pqrs
    stored at [p, r, q, s], fails here."""
    d = gen.molecular_integrals(n, 2, seed=seed)
    S = orc.System(n, na, nb, d["h"], d["g"])
    dimv = orc.dim(n, na, nb)
    rng = np.random.default_rng(seed)
    m = min(dimv, 12)
    r = np.sort(rng.choice(dimv, size=m, replace=False)).astype(np.uint64)
    c = rng.normal(size=m)
    g1, g2 = orc.rdm12(S, r, c)
    a, b = orc.det_unrank(n, na, nb, r)
    psi = {int(x) | (int(y) << n): float(v) for x, y, v in zip(a, b, c)}
    ref1 = np.zeros((n, n))
    ref2 = np.zeros((n, n, n, n))
    for fock, v in psi.items():
        for s_ in range(2):
            for p in range(n):
                for q in range(n):
                    sg, out = _jw_apply([(s_ * n + p, 1), (s_ * n + q, 0)], fock)
                    if sg:
                        ref1[p, q] += psi.get(out, 0.0) * sg * v
        for s_ in range(2):
            for t_ in range(2):
                for p, q, rr, ss in itertools.product(range(n), repeat=4):
                    ops = [(s_ * n + p, 1), (t_ * n + rr, 1), (t_ * n + ss, 0), (s_ * n + q, 0)]
                    sg, out = _jw_apply(ops, fock)
                    if sg:
                        ref2[p, q, rr, ss] += psi.get(out, 0.0) * sg * v
    assert np.max(np.abs(g1 - ref1)) < 1e-12
    assert np.max(np.abs(g2 - ref2)) < 1e-12
    # the pin distinguishes the orientations: a random psi breaks the
    # symmetries that would hide a swapped index pair
    assert np.max(np.abs(ref2 - ref2.transpose(1, 0, 2, 3))) > 1e-3
    assert np.max(np.abs(ref2 - ref2.transpose(0, 2, 1, 3))) > 1e-3
