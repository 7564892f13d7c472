"""CPU oracle for the sparse-FCI sigma = H psi path.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` import this package.  It
shares no code with the CUDA library and never calls it.

The heavy per-determinant steps (Eq. 12 ranking, excitation enumeration,
Slater-Condon elements, sigma by list-sort-merge) are plain C in
``sfci_oracle.c``; this module binds them and states the rest with numpy:

  * ``truncate_topk``   Eq. 11: keep the N_d largest |c| (ties to the smaller
                        index, exact zeros never kept), normalise;
  * ``sfci``            the truncated Lanczos of Sec. 2.1 (Eq. 10, Eq. 11),
                        the generalised problem T x = lambda S x with
                        S_ij = <w_i|w_j>, restart after N_L vectors and the
                        halting test;
  * ``fci_ground_energy`` dense diagonalisation of a small space.

Where the paper is silent or garbled the readings are:
  * b_i = <w_{i-1}| sigma_i> (Eq. 10 read literally; Eq. 6's sqrt form is the
    norm of the unnormalised vector);
  * a cycle holds N_L vectors w_0..w_{N_L-1}, so N_L sigma applications per
    cycle, and the iteration count N_I counts sigma applications;
  * T_ji = <w_j|sigma_i> for j <= i, mirrored;  E = lowest generalised
    eigenvalue, by canonical orthogonalisation of S (eigenvalues below
    1e-12 * max dropped);
  * the epsilon screen drops |sigma_k| < eps after the merge, before the dots.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_u64p = C.POINTER(C.c_uint64)
_f64p = C.POINTER(C.c_double)
_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)


class _Sys(C.Structure):
    _fields_ = [("n", C.c_int), ("na", C.c_int), ("nb", C.c_int),
                ("e_core", C.c_double), ("h", _f64p), ("g", _f64p)]


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = C.CDLL(path)
        L.or_binom.restype = C.c_uint64
        L.or_binom.argtypes = [C.c_int, C.c_int]
        L.or_string_rank.restype = C.c_uint64
        L.or_string_rank.argtypes = [C.c_uint64, C.c_int]
        L.or_string_unrank.restype = C.c_uint64
        L.or_string_unrank.argtypes = [C.c_uint64, C.c_int, C.c_int]
        L.or_string_successor.restype = C.c_int
        L.or_string_successor.argtypes = [C.c_uint64, C.c_int, _u64p]
        L.or_dim.restype = C.c_int
        L.or_dim.argtypes = [C.c_int, C.c_int, C.c_int, _u64p]
        L.or_det_rank.restype = C.c_uint64
        L.or_det_rank.argtypes = [C.c_int, C.c_int, C.c_uint64, C.c_uint64]
        L.or_det_rank_batch.restype = None
        L.or_det_rank_batch.argtypes = [C.c_int, C.c_int, _u64p, _u64p, _u64p, C.c_int64]
        L.or_det_unrank_batch.restype = None
        L.or_det_unrank_batch.argtypes = [C.c_int, C.c_int, C.c_int, _u64p, _u64p,
                                          _u64p, C.c_int64]
        L.or_hmat.restype = C.c_double
        L.or_hmat.argtypes = [C.POINTER(_Sys), C.c_uint64, C.c_uint64, C.c_uint64,
                              C.c_uint64]
        L.or_hmat_batch.restype = None
        L.or_hmat_batch.argtypes = [C.POINTER(_Sys), _u64p, _u64p, _u64p, _u64p, _f64p, C.c_int64]
        L.or_n_connected.restype = C.c_int64
        L.or_n_connected.argtypes = [C.c_int, C.c_int, C.c_int]
        L.or_connected.restype = C.c_int64
        L.or_connected.argtypes = [C.c_int, C.c_uint64, C.c_uint64, _u64p, _u64p]
        L.or_sigma.restype = C.c_int64
        L.or_sigma.argtypes = [C.POINTER(_Sys), _u64p, _f64p, C.c_int64, _u64p, _f64p,
                               _f64p, C.c_int64, _i64p, C.c_int, C.c_double]
        L.or_sigma_entries.restype = None
        L.or_sigma_entries.argtypes = [C.POINTER(_Sys), _u64p, _f64p, C.c_int64, _u64p,
                                       C.c_int64, _f64p, _f64p, _i32p, C.c_int]
        L.or_dense_h.restype = C.c_int
        L.or_dense_h.argtypes = [C.POINTER(_Sys), _f64p, C.c_int64]
        L.or_rdm12.restype = C.c_int
        L.or_rdm12.argtypes = [C.POINTER(_Sys), _u64p, _f64p, C.c_int64, _f64p, _f64p]
        L.or_max_threads.restype = C.c_int
        _LIB = L
    return _LIB


def _p(a, t):
    return a.ctypes.data_as(t)


def n_threads():
    return max(1, os.cpu_count() or 1)


# ---------------------------------------------------------------- system

class System:
    """Integrals and electron counts (h: n x n, g: n^4 chemists' order)."""

    def __init__(self, n, na, nb, h, g, e_core=0.0):
        self.n, self.na, self.nb = int(n), int(na), int(nb)
        self.h = np.ascontiguousarray(h, dtype=np.float64).reshape(n, n)
        self.g = np.ascontiguousarray(g, dtype=np.float64).reshape(n, n, n, n)
        self.e_core = float(e_core)
        self._s = _Sys(self.n, self.na, self.nb, self.e_core, _p(self.h, _f64p),
                       _p(self.g, _f64p))

    @classmethod
    def from_dict(cls, d):
        return cls(d["n"], d["na"], d["nb"], d["h"], d["g"], d.get("e_core", 0.0))

    @property
    def ref(self):
        return C.byref(self._s)

    @property
    def dim(self):
        return dim(self.n, self.na, self.nb)


# ------------------------------------------------------------ Eq. 12 etc.

def binom(n, k):
    return int(lib().or_binom(n, k))


def string_rank(s, n):
    return int(lib().or_string_rank(int(s), n))


def string_unrank(r, n, m):
    return int(lib().or_string_unrank(int(r), n, m))


def string_successor(s, n):
    out = C.c_uint64(0)
    ok = lib().or_string_successor(int(s), n, C.byref(out))
    return int(out.value) if ok else None


def dim(n, na, nb):
    out = C.c_uint64(0)
    if lib().or_dim(n, na, nb, C.byref(out)) != 0:
        raise OverflowError("C(n,na)*C(n,nb) does not fit in 64 bits")
    return int(out.value)


def det_rank(n, nb, alpha, beta):
    a = np.ascontiguousarray(alpha, dtype=np.uint64)
    b = np.ascontiguousarray(beta, dtype=np.uint64)
    out = np.empty(a.shape, dtype=np.uint64)
    lib().or_det_rank_batch(n, nb, _p(a, _u64p), _p(b, _u64p), _p(out, _u64p), a.size)
    return out


def det_unrank(n, na, nb, rank):
    r = np.ascontiguousarray(rank, dtype=np.uint64)
    a = np.empty(r.shape, dtype=np.uint64)
    b = np.empty(r.shape, dtype=np.uint64)
    lib().or_det_unrank_batch(n, na, nb, _p(r, _u64p), _p(a, _u64p), _p(b, _u64p), r.size)
    return a, b


def n_connected(n, na, nb):
    return int(lib().or_n_connected(n, na, nb))


def connected(n, na, nb, alpha, beta):
    m = n_connected(n, na, nb)
    oa = np.empty(m, dtype=np.uint64)
    ob = np.empty(m, dtype=np.uint64)
    c = lib().or_connected(n, int(alpha), int(beta), _p(oa, _u64p), _p(ob, _u64p))
    assert c == m
    return oa, ob


def hmat(sys: System, src, tgt):
    """<tgt|H|src> with src = (alpha, beta), tgt = (alpha, beta)."""
    return float(lib().or_hmat(sys.ref, int(src[0]), int(src[1]), int(tgt[0]), int(tgt[1])))


def hmat_batch(sys: System, src_a, src_b, tgt_a, tgt_b):
    """<tgt|H|src> for arrays of determinants."""
    a = [np.ascontiguousarray(x, dtype=np.uint64) for x in (src_a, src_b, tgt_a, tgt_b)]
    out = np.empty(a[0].size)
    lib().or_hmat_batch(sys.ref, *[_p(x, _u64p) for x in a], _p(out, _f64p), a[0].size)
    return out


def dense_h(sys: System):
    d = sys.dim
    if d > 20000:
        raise ValueError("dense H is for small spaces only")
    H = np.empty((d, d))
    lib().or_dense_h(sys.ref, _p(H, _f64p), d)
    return H


def fci_ground_energy(sys: System):
    """Lowest eigenvalue of the dense H (numpy's symmetric eigensolver)."""
    return float(np.linalg.eigvalsh(dense_h(sys))[0])


# ---------------------------------------------------------------- sigma

def sigma(sys: System, rank, coef, threads=None, eps_element=0.0):
    """sigma = H psi by list-sort-merge.  Returns (rank, value, abs_sum,
    n_elements) with ranks ascending; abs_sum[k] = sum_D |<k|H|D> c_D|.
    eps_element > 0: intermediate elements with |<k|H|D> c_D| < eps_element are
    not generated (heat-bath style selection, Sec. 4 outlook)."""
    r = np.ascontiguousarray(rank, dtype=np.uint64)
    c = np.ascontiguousarray(coef, dtype=np.float64)
    nt = threads or n_threads()
    cap = max(16, r.size * 8)
    while True:
        orank = np.empty(cap, dtype=np.uint64)
        oval = np.empty(cap)
        oabs = np.empty(cap)
        nel = C.c_int64(0)
        m = lib().or_sigma(sys.ref, _p(r, _u64p), _p(c, _f64p), r.size, _p(orank, _u64p),
                           _p(oval, _f64p), _p(oabs, _f64p), cap, C.byref(nel), nt,
                           float(eps_element))
        if m < 0:
            raise MemoryError("oracle sigma: out of memory")
        if m <= cap:
            return orank[:m], oval[:m], oabs[:m], int(nel.value)
        cap = m


def sigma_entries(sys: System, rank, coef, targets, threads=None):
    """sigma_k for the given targets, each pulled one by one.  Returns
    (value, abs_sum, present)."""
    r = np.ascontiguousarray(rank, dtype=np.uint64)
    c = np.ascontiguousarray(coef, dtype=np.float64)
    t = np.ascontiguousarray(targets, dtype=np.uint64)
    val = np.empty(t.size)
    asum = np.empty(t.size)
    pres = np.empty(t.size, dtype=np.int32)
    lib().or_sigma_entries(sys.ref, _p(r, _u64p), _p(c, _f64p), r.size, _p(t, _u64p), t.size,
                           _p(val, _f64p), _p(asum, _f64p), _p(pres, _i32p),
                           threads or n_threads())
    return val, asum, pres.astype(bool)


def screen(rank, val, eps):
    """Drop |sigma_k| < eps (the paper's epsilon threshold, Sec. 3)."""
    if eps <= 0.0:
        return rank, val
    keep = ~(np.abs(val) < eps)
    return rank[keep], val[keep]


# ----------------------------------------------------------- truncation

def topk_indices(rank, coef, k):
    """Indices of the entries Eq. 11 keeps: the k largest |c|; equal |c| go to
    the smaller rank; exact zeros are never kept."""
    rank = np.asarray(rank, dtype=np.uint64)
    coef = np.asarray(coef, dtype=np.float64)
    nz = np.nonzero(coef != 0.0)[0]
    order = np.lexsort((rank[nz], -np.abs(coef[nz])))
    return np.sort(nz[order[:k]])


def truncate_topk(rank, coef, k, normalize=True):
    """Eq. 11: w' = the k largest-magnitude entries, w = w' / sqrt(<w'|w'>).
    Output ascending by rank."""
    rank = np.asarray(rank, dtype=np.uint64)
    coef = np.asarray(coef, dtype=np.float64)
    idx = topk_indices(rank, coef, k)
    r = rank[idx]
    c = coef[idx].copy()
    order = np.argsort(r, kind="stable")
    r, c = r[order], c[order]
    if normalize and c.size:
        c = c / np.sqrt(np.dot(c, c))
    return r, c


# ---------------------------------------------------- sparse-vector algebra

def sparse_dot(ra, ca, rb, cb):
    """<a|b> over the common ranks (both ascending)."""
    if ra.size == 0 or rb.size == 0:
        return 0.0
    idx = np.searchsorted(rb, ra)
    idx_c = np.minimum(idx, rb.size - 1)
    hit = (idx < rb.size) & (rb[idx_c] == ra)
    return float(np.dot(ca[hit], cb[idx_c[hit]]))


def sparse_axpy_union(ra, ca, terms):
    """u = a + sum_t s_t * v_t on the union of supports, in the order given:
    u_k = ((a_k - s_1 v1_k) - s_2 v2_k) ...  terms = [(s, rv, cv), ...]."""
    allr = np.unique(np.concatenate([ra] + [t[1] for t in terms]))
    u = np.zeros(allr.size)
    pos = np.searchsorted(allr, ra)
    u[pos] = ca
    for s, rv, cv in terms:
        if rv.size == 0:
            continue
        pos = np.searchsorted(allr, rv)
        u[pos] = u[pos] - s * cv
    return allr, u


def gen_eig_lowest(T, S, drop=1e-12):
    """Lowest root of T x = lambda S x by canonical orthogonalisation."""
    s, U = np.linalg.eigh(S)
    keep = s > drop * s.max()
    X = U[:, keep] / np.sqrt(s[keep])
    Tp = X.T @ T @ X
    lam, y = np.linalg.eigh(0.5 * (Tp + Tp.T))
    return float(lam[0]), X @ y[:, 0]


def sfci(sys: System, init_rank, init_coef, n_keep, n_lanczos=10, n_iter=30,
         eps_screen=0.0, conv_tol=None, threads=None, record_vectors=False, eps_element=0.0):
    """The truncated Lanczos of Sec. 2.1.

    Each cycle starts from w_0 (truncated, normalised) and for i = 0..N_L-1:
      sigma_i = H w_i (screened);  T_ji = <w_j|sigma_i>, S_ji = <w_j|w_i>, j <= i;
      u = sigma_i - a_i w_i - b_i w_{i-1}, a_i = T_ii, b_i = T_{i-1,i}  (Eq. 10);
      w_{i+1} = normalise(top_{N_d}(u))  (Eq. 11).
    At the cycle end T x = lambda S x is solved; E = lambda_min; Psi =
    sum_j x_j w_j; w_0 <- normalise(top_{N_d}(Psi)) (restart).  Stops after
    n_iter sigma applications or when the energy drop is below conv_tol.
    Returns a list with one dict per sigma application.
    """
    wr, wc = truncate_topk(init_rank, init_coef, n_keep)
    steps = []
    it = 0
    cycle = 0
    e_prev = None
    while it < n_iter:
        W = [(wr, wc)]
        NL = n_lanczos
        T = np.zeros((NL, NL))
        Sm = np.zeros((NL, NL))
        for i in range(NL):
            sr, sv, _, nel = sigma(sys, W[i][0], W[i][1], threads, eps_element)
            sr, sv = screen(sr, sv, eps_screen)
            it += 1
            for j in range(i + 1):
                T[j, i] = sparse_dot(W[j][0], W[j][1], sr, sv)
                Sm[j, i] = sparse_dot(W[j][0], W[j][1], W[i][0], W[i][1])
            info = {"iter": it, "cycle": cycle, "i": i, "a": T[i, i],
                    "n_in": int(W[i][0].size), "n_sigma": int(sr.size),
                    "n_elements": nel, "converged": False, "lambda": None}
            steps.append(info)
            last = (i == NL - 1) or (it >= n_iter)
            if not last:
                a = T[i, i]
                b = T[i - 1, i] if i > 0 else 0.0
                terms = [(a, W[i][0], W[i][1])]
                if i > 0:
                    terms.append((b, W[i - 1][0], W[i - 1][1]))
                ur, uv = sparse_axpy_union(sr, sv, terms)
                unorm = np.sqrt(np.dot(uv, uv))
                info["u_norm"] = float(unorm)
                if unorm < 1e-14 * abs(a) or not np.any(uv != 0.0):
                    last = True
                else:
                    W.append(truncate_topk(ur, uv, n_keep))
                    info["n_kept"] = int(W[-1][0].size)
            if last:
                m = len(W)
                Tm = np.triu(T[:m, :m]) + np.triu(T[:m, :m], 1).T
                Smm = np.triu(Sm[:m, :m]) + np.triu(Sm[:m, :m], 1).T
                lam, x = gen_eig_lowest(Tm, Smm)
                pr = np.zeros(0, dtype=np.uint64)
                pv = np.zeros(0)
                # Psi = sum_j x_j w_j, accumulated in ascending j
                allr = np.unique(np.concatenate([w[0] for w in W]))
                acc = np.zeros(allr.size)
                for j, (r, c) in enumerate(W):
                    pos = np.searchsorted(allr, r)
                    acc[pos] = acc[pos] + x[j] * c
                pr, pv = allr, acc
                info["lambda"] = lam
                info["psi_size"] = int(np.count_nonzero(pv))
                info["T"] = Tm.copy()
                info["S"] = Smm.copy()
                info["x"] = x.copy()
                if record_vectors:
                    info["W"] = [(r.copy(), c.copy()) for r, c in W]
                wr, wc = truncate_topk(pr, pv, n_keep)
                if conv_tol is not None and e_prev is not None and e_prev - lam < conv_tol:
                    info["converged"] = True
                    return steps
                e_prev = lam
                cycle += 1
                break
            if record_vectors:
                info["W_next"] = (W[-1][0].copy(), W[-1][1].copy())
    return steps


# ---------------------------------------------------------------- RDMs

def rdm12(sys: System, rank, coef):
    """Spin-summed 1- and 2-RDMs of psi (not normalised), by operator
    application; gamma[p,q] = sum_s <a+_ps a_qs>, Gamma[p,q,r,s] =
    sum_{st} <a+_ps a+_rt a_st a_qs>.  Small psi only."""
    r = np.ascontiguousarray(rank, dtype=np.uint64)
    c = np.ascontiguousarray(coef, dtype=np.float64)
    n = sys.n
    g1 = np.empty((n, n))
    g2 = np.empty((n, n, n, n))
    lib().or_rdm12(sys.ref, _p(r, _u64p), _p(c, _f64p), r.size, _p(g1, _f64p), _p(g2, _f64p))
    return g1, g2
