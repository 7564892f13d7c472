"""Seeded synthetic inputs for the sparse-FCI sigma = H psi path.

Both the CPU oracle and the CUDA library are fed from here, so that the two
sides read identical bits.  The module holds none of the method's arithmetic:
it draws integrals, writes the Hubbard ring as integrals, and samples
occupation strings and coefficients.  Ranking, excitation, matrix elements and
every other step of the method live on each side separately.

Conventions shared with the callers (they are input formats, not method):
  * orbital p (0-based) of a spin string is bit p of a uint64;
  * ``h`` is an (n, n) float64 array, ``g`` an (n, n, n, n) float64 array with
    g[p, q, r, s] = (pq|rs) in chemists' notation, real orbitals, 8-fold
    symmetric (the paper takes these integrals from an external program,
    Sec. 3; no molecular integrals are available here, so seeded synthetic ones
    of the same shapes stand in for them).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "molecular_integrals",
    "hubbard_ring",
    "two_site_hubbard",
    "config_system",
    "near_aufbau_dets",
    "random_dets",
    "level_coefs",
    "batched_scan_instances",
]


def _symmetric_gaussian(rng, n, sd, with_diag):
    """Symmetric (n, n) matrix: upper triangle drawn N(0, sd), then mirrored."""
    m = np.zeros((n, n))
    iu = np.triu_indices(n, 0 if with_diag else 1)
    m[iu] = rng.normal(0.0, sd, size=len(iu[0]))
    m = m + m.T - np.diag(np.diag(m))
    return m


def molecular_integrals(n: int, n_factors: int, seed: int, diag=None,
                        sd_offdiag: float = 0.1, sd_factor: float = 0.3,
                        cluster_diag: bool = False):
    """Synthetic molecular integrals.

    h: symmetric, off-diagonal N(0, sd_offdiag); diagonal ``linspace(-2, 1, n)``
    (ascending, so the lowest-occupation determinant is the aufbau one) or, with
    ``cluster_diag``, two near-degenerate clusters: n/2 values U[-2.0, -1.9] and
    n - n/2 values U[0.9, 1.0], each sorted.
    g: (pq|rs) = sum_L B^L_pq B^L_rs with B^L symmetric, entries N(0, sd_factor):
    8-fold symmetric and positive semidefinite as an (n^2, n^2) matrix.
    Returns dict(h, g, B, e_core).
    """
    rng = np.random.default_rng(seed)
    if cluster_diag:
        lo = np.sort(rng.uniform(-2.0, -1.9, size=n // 2))
        hi = np.sort(rng.uniform(0.9, 1.0, size=n - n // 2))
        diag = np.concatenate([lo, hi])
    elif diag is None:
        diag = np.linspace(-2.0, 1.0, n)
    h = _symmetric_gaussian(rng, n, sd_offdiag, with_diag=False)
    h[np.diag_indices(n)] = np.asarray(diag, dtype=np.float64)
    B = np.stack([_symmetric_gaussian(rng, n, sd_factor, with_diag=True)
                  for _ in range(n_factors)])
    g = factor_to_eri(B)
    return {"h": np.ascontiguousarray(h), "g": g, "B": B, "e_core": 0.0}


def factor_to_eri(B):
    """(pq|rs) = sum_L B[L,p,q] B[L,r,s], summed over L in ascending order."""
    L, n, _ = B.shape
    flat = B.reshape(L, n * n)
    g = np.zeros((n * n, n * n))
    for l in range(L):
        g += np.outer(flat[l], flat[l])
    return np.ascontiguousarray(g.reshape(n, n, n, n))


def hubbard_ring(n_sites: int, t: float = 1.0, U: float = 4.0):
    """1D Hubbard ring as integrals: h[i, i+-1 mod n] = -t, (pp|pp) = U, else 0."""
    n = n_sites
    h = np.zeros((n, n))
    for i in range(n):
        h[i, (i + 1) % n] = -t
        h[(i + 1) % n, i] = -t
    g = np.zeros((n, n, n, n))
    for p in range(n):
        g[p, p, p, p] = U
    return {"h": h, "g": g, "e_core": 0.0}


def two_site_hubbard(t: float, U: float):
    """Two sites joined by one bond (not a ring: a single hopping -t)."""
    h = np.array([[0.0, -t], [-t, 0.0]])
    g = np.zeros((2, 2, 2, 2))
    g[0, 0, 0, 0] = U
    g[1, 1, 1, 1] = U
    return {"h": h, "g": g, "e_core": 0.0}


def config_system(cfg: int):
    """The five workloads (integrals and electron counts).

    0: n=8, 4a/4b, L=16 factors (seed 0), diagonal -2..+1.
    1: 12-site Hubbard ring, 6a/6b, t=1, U=4.
    2: n=28, 7a/7b, L=200 (seed 2), two near-degenerate diagonal clusters
       (a stretched-bond stand-in shaped like the paper's (26-28 orbital,
       8-18 electron) molecules).
    4: n=20, 5a/5b, L=64 (seed 4).
    (3, the batched scan, is built by ``batched_scan_instances``.)
    """
    if cfg == 0:
        d = molecular_integrals(8, 16, seed=0)
        return dict(d, n=8, na=4, nb=4)
    if cfg == 1:
        d = hubbard_ring(12, 1.0, 4.0)
        return dict(d, n=12, na=6, nb=6)
    if cfg == 2:
        d = molecular_integrals(28, 200, seed=2, cluster_diag=True)
        return dict(d, n=28, na=7, nb=7)
    if cfg == 4:
        d = molecular_integrals(20, 64, seed=4)
        return dict(d, n=20, na=5, nb=5)
    raise ValueError(f"no single-system workload {cfg}")


def batched_scan_instances(count: int = 32, seed: int = 3, n_max: int = 24,
                           n_factors: int = 16):
    """A geometry-like scan: ``count`` instances with uneven sizes.

    Two integral sets A (seed 31) and B (seed 32) at n_max orbitals; instance i
    uses (1 - lam) A + lam B with lam = i / (count - 1), restricted to its leading
    n x n (and n^4) block.  n ~ U{16..24}, na = nb ~ U{5..8}, vector cap
    log-uniform in [1e4, 2e5].
    """
    rng = np.random.default_rng(seed)
    A = molecular_integrals(n_max, n_factors, seed=31)
    Bs = molecular_integrals(n_max, n_factors, seed=32)
    out = []
    for i in range(count):
        lam = i / max(count - 1, 1)
        n = int(rng.integers(16, n_max + 1))
        ne = int(rng.integers(5, 9))
        cap = int(round(np.exp(rng.uniform(np.log(1e4), np.log(2e5)))))
        h = (1.0 - lam) * A["h"] + lam * Bs["h"]
        g = (1.0 - lam) * A["g"] + lam * Bs["g"]
        out.append({
            "h": np.ascontiguousarray(h[:n, :n]),
            "g": np.ascontiguousarray(g[:n, :n, :n, :n]),
            "e_core": 0.0, "n": n, "na": ne, "nb": ne, "cap": cap, "lam": lam,
        })
    return out


# ---------------------------------------------------------------- determinants

def _excite(rng, n, m, k, size):
    """``size`` spin strings made from the aufbau string (orbitals 0..m-1) by
    moving k electrons to randomly chosen empty orbitals."""
    base = np.uint64((1 << m) - 1) if m < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    out = np.full(size, base, dtype=np.uint64)
    if k == 0 or size == 0:
        return out
    holes = np.argsort(rng.random((size, m)), axis=1)[:, :k]
    parts = m + np.argsort(rng.random((size, n - m)), axis=1)[:, :k]
    one = np.uint64(1)
    for c in range(k):
        out ^= one << holes[:, c].astype(np.uint64)
        out ^= one << parts[:, c].astype(np.uint64)
    return out


def near_aufbau_dets(n: int, na: int, nb: int, count: int, seed: int,
                     max_level: int = 2, include_aufbau: bool = True):
    """``count`` distinct determinants (alpha, beta) near the aufbau one.

    Each spin string is excited k times with k drawn from {0..max_level}
    (weights favouring low k), the shape of a truncated Lanczos vector that
    grew from the lowest-occupation determinant.  Returns (alpha, beta, level)
    as uint64, uint64, int arrays (unsorted, unique pairs).
    """
    rng = np.random.default_rng(seed)
    kmax_a = min(max_level, na, n - na)
    kmax_b = min(max_level, nb, n - nb)
    seen = set()
    A, Bv, K = [], [], []
    if include_aufbau:
        a0 = (1 << na) - 1
        b0 = (1 << nb) - 1
        seen.add((a0, b0))
        A.append(a0), Bv.append(b0), K.append(0)
    wa = np.array([3.0 ** -k for k in range(kmax_a + 1)]) * \
        np.array([1.0] + [float(k) for k in range(1, kmax_a + 1)])
    wb = np.array([3.0 ** -k for k in range(kmax_b + 1)]) * \
        np.array([1.0] + [float(k) for k in range(1, kmax_b + 1)])
    wa /= wa.sum()
    wb /= wb.sum()
    guard = 0
    while len(A) < count:
        guard += 1
        if guard > 200:
            raise ValueError("space too small for the requested count")
        m = max(2 * (count - len(A)), 1024)
        ka = rng.choice(kmax_a + 1, size=m, p=wa)
        kb = rng.choice(kmax_b + 1, size=m, p=wb)
        sa = np.empty(m, dtype=np.uint64)
        sb = np.empty(m, dtype=np.uint64)
        for k in range(kmax_a + 1):
            sel = np.nonzero(ka == k)[0]
            sa[sel] = _excite(rng, n, na, k, len(sel))
        for k in range(kmax_b + 1):
            sel = np.nonzero(kb == k)[0]
            sb[sel] = _excite(rng, n, nb, k, len(sel))
        for x, y, k in zip(sa.tolist(), sb.tolist(), (ka + kb).tolist()):
            if (x, y) in seen:
                continue
            seen.add((x, y))
            A.append(x), Bv.append(y), K.append(k)
            if len(A) == count:
                break
    return (np.array(A, dtype=np.uint64), np.array(Bv, dtype=np.uint64),
            np.array(K, dtype=np.int64))


def random_dets(n: int, na: int, nb: int, count: int, seed: int):
    """``count`` distinct determinants drawn uniformly from the whole space."""
    rng = np.random.default_rng(seed)
    seen = set()
    A, Bv = [], []
    one = np.uint64(1)
    guard = 0
    while len(A) < count:
        guard += 1
        if guard > 200:
            raise ValueError("space too small for the requested count")
        m = max(2 * (count - len(A)), 256)
        pa = np.argsort(rng.random((m, n)), axis=1)[:, :na]
        pb = np.argsort(rng.random((m, n)), axis=1)[:, :nb]
        sa = np.zeros(m, dtype=np.uint64)
        sb = np.zeros(m, dtype=np.uint64)
        for c in range(na):
            sa |= one << pa[:, c].astype(np.uint64)
        for c in range(nb):
            sb |= one << pb[:, c].astype(np.uint64)
        for x, y in zip(sa.tolist(), sb.tolist()):
            if (x, y) in seen:
                continue
            seen.add((x, y))
            A.append(x), Bv.append(y)
            if len(A) == count:
                break
    return np.array(A, dtype=np.uint64), np.array(Bv, dtype=np.uint64)


def level_coefs(level, seed: int, decay: float = 1.5):
    """Coefficients whose magnitude decays with excitation level, random sign."""
    rng = np.random.default_rng(seed)
    level = np.asarray(level)
    mag = np.exp(-decay * level) * rng.uniform(0.2, 1.0, size=level.shape)
    sign = np.where(rng.random(level.shape) < 0.5, -1.0, 1.0)
    return mag * sign
