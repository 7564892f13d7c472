"""Pins for the oracle's excitation enumeration and Slater-Condon elements.

The independent reference is the Hamiltonian written in second quantisation,
H = e_core + sum_pq h_pq sum_s a+_ps a_qs
           + 1/2 sum_pqrs (pq|rs) sum_st a+_ps a+_rt a_st a_qs,
applied operator by operator to occupation-number states with Jordan-Wigner
signs (spin orbitals ordered alpha 0..n-1, then beta 0..n-1), plus closed-form
spectra of small model systems.
"""
import itertools

import numpy as np
import pytest

import gen


def _sector(n, na, nb):
    A = [sum(1 << p for p in c) for c in itertools.combinations(range(n), na)]
    B = [sum(1 << p for p in c) for c in itertools.combinations(range(n), nb)]
    return [(a, b) for a in A for b in B]


def _apply(ops, state):
    """Apply (spin_orbital, is_creator) operators right to left."""
    sign = 1
    for so, dag in reversed(ops):
        occ = (state >> so) & 1
        if occ == dag:
            return 0, 0
        if bin(state & ((1 << so) - 1)).count("1") & 1:
            sign = -sign
        state ^= 1 << so
    return sign, state


def _second_quantised_column(n, h, g, e_core, a, b):
    """H |a, b> as {fock_state: amplitude}."""
    s0 = a | (b << n)
    out = {s0: e_core}
    for sp in range(2):
        for p in range(n):
            for q in range(n):
                if h[p, q] == 0.0:
                    continue
                sg, st = _apply([(sp * n + p, 1), (sp * n + q, 0)], s0)
                if sg:
                    out[st] = out.get(st, 0.0) + sg * h[p, q]
    for sp in range(2):
        for tp in range(2):
            for p, q, r, s in itertools.product(range(n), repeat=4):
                v = g[p, q, r, s]
                if v == 0.0:
                    continue
                ops = [(sp * n + p, 1), (tp * n + r, 1), (tp * n + s, 0), (sp * n + q, 0)]
                sg, st = _apply(ops, s0)
                if sg:
                    out[st] = out.get(st, 0.0) + 0.5 * sg * v
    return out


@pytest.mark.parametrize("n", [2, 3, 4])
def test_slater_condon_equals_second_quantisation(orc, n):
    d = gen.molecular_integrals(n, 3, seed=40 + n)
    h, g = d["h"], d["g"]
    e_core = 0.731
    for na in range(n + 1):
        for nb in range(n + 1):
            S = orc.System(n, na, nb, h, g, e_core)
            dets = _sector(n, na, nb)
            for (a, b) in dets:
                col = _second_quantised_column(n, h, g, e_core, a, b)
                for (x, y) in dets:
                    ref = col.get(x | (y << n), 0.0)
                    got = orc.hmat(S, (a, b), (x, y))
                    assert abs(got - ref) <= 1e-12 * (1.0 + abs(ref)), (na, nb, a, b, x, y)


@pytest.mark.parametrize("n,na,nb", [(4, 2, 2), (5, 2, 3), (6, 3, 3), (6, 1, 4), (7, 3, 2)])
def test_connected_set_is_brute_force(orc, n, na, nb):
    """connected(D) = {D' != D with the same counts and at most two electrons
    moved}, i.e. popcount(a ^ a') + popcount(b ^ b') <= 4; the count is
    na va + nb vb + C(na,2)C(va,2) + C(nb,2)C(vb,2) + na va nb vb."""
    dets = _sector(n, na, nb)
    va, vb = n - na, n - nb
    from math import comb
    want = na * va + nb * vb + comb(na, 2) * comb(va, 2) + comb(nb, 2) * comb(vb, 2) \
        + na * va * nb * vb
    assert orc.n_connected(n, na, nb) == want
    rng = np.random.default_rng(7)
    for k in rng.choice(len(dets), size=min(12, len(dets)), replace=False):
        a, b = dets[k]
        oa, ob = orc.connected(n, na, nb, a, b)
        got = set(zip(oa.tolist(), ob.tolist()))
        assert len(got) == want
        brute = {(x, y) for (x, y) in dets
                 if (x, y) != (a, b) and bin(x ^ a).count("1") + bin(y ^ b).count("1") <= 4}
        assert got == brute


def test_hamiltonian_hermitian_cfg0(orc):
    S = orc.System.from_dict(gen.config_system(0))
    H = orc.dense_h(S)
    assert H.shape == (4900, 4900)
    scale = np.abs(H).max()
    assert np.max(np.abs(H - H.T)) <= 1e-13 * scale
    # an element beyond double excitations vanishes
    r = orc.det_unrank(8, 4, 4, np.array([0, 4899], dtype=np.uint64))
    assert H[4899, 0] == 0.0 and (bin(int(r[0][1]) ^ int(r[0][0])).count("1") == 8)


def test_two_site_hubbard_closed_form(orc):
    """Two sites, one up and one down electron: E0 = (U - sqrt(U^2 + 16 t^2))/2."""
    for t, U in [(1.0, 4.0), (0.5, 1.0), (1.3, 0.0), (1.0, 10.0)]:
        d = gen.two_site_hubbard(t, U)
        S = orc.System(2, 1, 1, d["h"], d["g"])
        e0 = orc.fci_ground_energy(S)
        assert abs(e0 - 0.5 * (U - np.sqrt(U * U + 16 * t * t))) < 1e-12


def test_two_orbital_minimal_basis_spectrum(orc):
    """Two orbitals of opposite symmetry (h_12 = 0, (11|12) = (22|12) = 0), one
    up and one down electron: the four levels are
    (E1 + E2)/2 +- sqrt((E2 - E1)^2/4 + K^2) and h11 + h22 + J +- K, with
    E1 = 2 h11 + (11|11), E2 = 2 h22 + (22|22), J = (11|22), K = (12|12)."""
    h11, h22, J11, J22, J, K = -1.25, -0.47, 0.67, 0.70, 0.66, 0.18
    h = np.diag([h11, h22])
    g = np.zeros((2, 2, 2, 2))
    g[0, 0, 0, 0] = J11
    g[1, 1, 1, 1] = J22
    g[0, 0, 1, 1] = g[1, 1, 0, 0] = J
    for idx in [(0, 1, 0, 1), (1, 0, 1, 0), (0, 1, 1, 0), (1, 0, 0, 1)]:
        g[idx] = K
    S = orc.System(2, 1, 1, h, g)
    ev = np.sort(np.linalg.eigvalsh(orc.dense_h(S)))
    E1, E2 = 2 * h11 + J11, 2 * h22 + J22
    rad = np.sqrt(0.25 * (E2 - E1) ** 2 + K * K)
    want = np.sort([0.5 * (E1 + E2) - rad, 0.5 * (E1 + E2) + rad,
                    h11 + h22 + J - K, h11 + h22 + J + K])
    assert np.allclose(ev, want, atol=1e-13, rtol=0)


@pytest.mark.parametrize("n,na,nb", [(6, 3, 3), (7, 2, 4), (8, 4, 4)])
def test_no_interaction_is_orbital_sum(orc, n, na, nb):
    """g = 0: E0 = sum of the lowest na plus the lowest nb eigenvalues of h."""
    d = gen.molecular_integrals(n, 2, seed=n)
    S = orc.System(n, na, nb, d["h"], np.zeros((n,) * 4), e_core=0.25)
    eps = np.linalg.eigvalsh(d["h"])
    assert abs(orc.fci_ground_energy(S) - (eps[:na].sum() + eps[:nb].sum() + 0.25)) < 1e-11


def test_hubbard_ring_free_fermions(orc):
    """A ring at U = 0: levels -2 t cos(2 pi m / L); 8 sites, 4 up 4 down."""
    d = gen.hubbard_ring(8, 1.0, 0.0)
    S = orc.System(8, 4, 4, d["h"], d["g"])
    lev = np.sort(-2.0 * np.cos(2 * np.pi * np.arange(8) / 8))
    assert abs(orc.fci_ground_energy(S) - 2 * lev[:4].sum()) < 1e-11
    # and the 12-site closed form quoted for the 12-site workload at U = 0
    lev12 = np.sort(-2.0 * np.cos(2 * np.pi * np.arange(12) / 12))
    assert abs(2 * lev12[:6].sum() - (-14.9282032)) < 1e-7


def test_dense_solver_cross_check(orc):
    """cfg0: numpy's dense eigensolver and scipy's Lanczos (ARPACK) agree."""
    from scipy.sparse.linalg import eigsh
    S = orc.System.from_dict(gen.config_system(0))
    H = orc.dense_h(S)
    e_dense = np.linalg.eigvalsh(H)[0]
    e_lz = eigsh(H, k=1, which="SA", tol=1e-12)[0][0]
    assert abs(e_dense - e_lz) < 1e-9
