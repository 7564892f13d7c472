"""Pins for the oracle's truncated Lanczos (Sec. 2.1, Eqs. 5-11)."""
import numpy as np
import pytest

import gen


@pytest.fixture(scope="module")
def cfg0(orc):
    S = orc.System.from_dict(gen.config_system(0))
    w, V = np.linalg.eigh(orc.dense_h(S))
    return S, w, V


def _lams(steps):
    return [s["lambda"] for s in steps if s["lambda"] is not None]


def test_untruncated_first_cycle_is_lanczos(orc, cfg0):
    """With N_d >= dim and no screen the basis is the Lanczos basis of Eqs. 1-6:
    S = 1 and T tridiagonal (Eq. 7) up to rounding."""
    S, w, V = cfg0
    st = orc.sfci(S, np.array([0], dtype=np.uint64), np.array([1.0]), 4900, 8, 8)
    T, Sm = st[-1]["T"], st[-1]["S"]
    assert np.max(np.abs(Sm - np.eye(8))) < 1e-9
    far = np.abs(np.triu(T, 2))
    assert far.max() < 1e-8 * np.abs(T).max()
    assert np.all(np.abs(np.diag(T, 1)) > 1e-6)


def test_untruncated_converges_to_exact_sector_energy(orc, cfg0):
    """N_d >= dim: SFCI is restarted Lanczos and converges to the lowest
    eigenvalue whose eigenvector overlaps the start determinant (the random
    exchange integrals make the absolute ground state high-spin, outside the
    closed-shell start's sector)."""
    S, w, V = cfg0
    k = int(np.argmax(np.abs(V[0]) > 1e-8))
    e_sector = w[k]
    st = orc.sfci(S, np.array([0], dtype=np.uint64), np.array([1.0]), 4900, 10, 80)
    lam = _lams(st)
    assert abs(lam[-1] - e_sector) < 1e-9
    assert all(l >= w[0] - 1e-10 for l in lam)
    assert all(b <= a + 1e-10 for a, b in zip(lam, lam[1:]))


def test_truncated_is_variational_and_improves(orc, cfg0):
    """Rayleigh-Ritz in the span of the truncated vectors: every lambda and
    every cycle's <w_0|H|w_0> lies above the exact ground state; a larger N_d
    ends lower (Table 3's trend); Psi is not truncated (Table 3: |phi_0| > N_d)."""
    S, w, V = cfg0
    final = {}
    for nd in (60, 600):
        st = orc.sfci(S, np.array([0], dtype=np.uint64), np.array([1.0]), nd, 10, 40)
        lam = _lams(st)
        assert all(l >= w[0] - 1e-10 for l in lam)
        for s in st:
            if s["lambda"] is not None:
                assert s["T"][0, 0] >= w[0] - 1e-10
                assert s["psi_size"] > nd
            assert s["n_in"] <= nd
        final[nd] = lam[-1]
    assert final[600] < final[60]


def test_screen_drops_small_entries(orc):
    r = np.array([1, 5, 9, 12], dtype=np.uint64)
    v = np.array([1e-6, -3e-5, 5e-5, -2.0])
    rr, vv = orc.screen(r, v, 5e-5)
    assert rr.tolist() == [9, 12] and vv.tolist() == [5e-5, -2.0]
    rr, vv = orc.screen(r, v, 0.0)
    assert rr.size == 4


def test_generalised_eigensolver(orc):
    rng = np.random.default_rng(4)
    A = rng.normal(size=(6, 6))
    T = A + A.T
    B = rng.normal(size=(6, 6))
    Sm = B @ B.T + 6 * np.eye(6)
    lam, x = orc.gen_eig_lowest(T, Sm)
    from scipy.linalg import eigh
    assert abs(lam - eigh(T, Sm, eigvals_only=True)[0]) < 1e-12
    assert np.allclose(T @ x, lam * (Sm @ x), atol=1e-10)
