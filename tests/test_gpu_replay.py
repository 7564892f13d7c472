"""Step-by-step replay of whole GPU solver runs by the oracle.

For every step of a GPU run the oracle takes the GPU's own basis vectors
(w_0 .. w_i of the current cycle) and recomputes what the step should have
produced from them (Sec. 2.1, Eqs. 10-11):
  - sigma_i = H w_i (list, sort, ordered sums), T_ji = <w_j|sigma_i> and
    S_ji = <w_j|w_i> for j <= i: the GPU's T and S columns within
    1e-11 sum_k |w_j,k| A_k (A_k = sum_D |H_kD c_D|) and 1e-13;
  - a_i, b_i the same way;
  - u = sigma_i - a_i w_i - b_i w_{i-1} and its exact top-N_d: the GPU's
    w_{i+1} keeps the same entries, except entries whose |u| lies within
    1e-11 A_k of the cut (rounding can order near-ties either way; at
    n_alpha = n_beta spin-flip partners tie exactly), and its values agree
    to 1e-11 A_k / ||u_kept|| on the common entries;
  - at a cycle end: lambda_min within 1e-9 Ha of the lowest root of the
    GPU's T, S (host eigensolver) and of the oracle's T, S (the oracle's dots
    on the GPU's vectors), and the restart vector w_0 = top_N_d(sum_j x_j w_j)
    with the same rule at the cut (up to the sign of the eigenvector).
Replaying on the GPU's vectors keeps the comparison local to one step: a
near-tie decided differently at one step does not make later steps diverge.
Workloads: 8 orbitals 4a/4b (closed shell) at N_d = 300, 30 steps; the
12-site Hubbard ring 6a/6b at N_d = 2e4, 40 steps from the aufbau determinant.
"""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu

TOL = 1e-11


@pytest.fixture(scope="module")
def sf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2312_01846_gb300 as sf
    sf.lib()
    return sf


def _vec(sf, lz):
    r, c = lz.vector()
    return sf.to_u64(r).copy(), c.cpu().numpy().copy()


def _on(r, c, keys):
    """values of the sparse vector (r, c) at keys (0 where absent)."""
    if r.size == 0:
        return np.zeros(keys.size)
    pos = np.minimum(np.searchsorted(r, keys), r.size - 1)
    return np.where(r[pos] == keys, c[pos], 0.0)


def _check_kept(gr, gc, ur, uv, tol, n_keep, orc, label, sign=1.0):
    """GPU's kept vector (gr, gc) against the exact top-N_d of u (ur, uv);
    tol[k] bounds the rounding of |u_k| on either side.  When u has more than
    N_d non-zero entries the cut is the N_d-th largest |u|; otherwise every
    non-zero entry is kept and the cut is 0 (an entry that cancels to zero in
    exact arithmetic may come out as exactly 0 on one side and as a rounding
    residue on the other).  Every kept-set difference must lie within
    tolerance of the cut.  Returns the number of differences."""
    kr, kv = orc.truncate_topk(ur, uv, n_keep)
    binding = kr.size == n_keep and np.count_nonzero(uv) > n_keep
    if binding:
        assert gr.size == kr.size, (label, gr.size, kr.size)
    else:
        assert gr.size <= n_keep, (label, gr.size)
    if kr.size == 0 and gr.size == 0:
        return 0
    pos_k = np.searchsorted(ur, kr)
    if binding:
        cut_at = np.argmin(np.abs(uv[pos_k]))
        cut, tol_cut = np.abs(uv[pos_k][cut_at]), tol[pos_k][cut_at]
    else:
        cut, tol_cut = 0.0, 0.0
    diff = np.setxor1d(gr, kr)
    if diff.size:
        pos = np.minimum(np.searchsorted(ur, diff), ur.size - 1)
        assert np.all(ur[pos] == diff), (label, "a kept GPU entry is not in u's support")
        near = np.abs(np.abs(uv[pos]) - cut) <= tol[pos] + tol_cut
        assert np.all(near), (label, diff[~near][:5], np.abs(uv[pos])[~near][:5], cut)
    common = np.intersect1d(gr, kr)
    nrm = np.sqrt(np.dot(uv[pos_k], uv[pos_k]))
    g = gc[np.searchsorted(gr, common)]
    o = kv[np.searchsorted(kr, common)]
    bound = tol[np.searchsorted(ur, common)] / nrm + 1e-12 * np.abs(o)
    err = np.abs(sign * g - o)
    assert np.all(err <= bound), (label, err.max(), (err / bound).max())
    return int(diff.size)


class Replay:
    """Oracle replay of one solver: feed it each step's info, the solver's T and
    S after the step (sfci_lanczos_matrices) and its next input vector."""

    def __init__(self, orc, osys, w0, n_keep, n_lanczos, label):
        self.orc, self.osys, self.n_keep, self.label = orc, osys, n_keep, label
        self.W = [w0]
        self.T_or = np.zeros((n_lanczos, n_lanczos))
        self.S_or = np.zeros((n_lanczos, n_lanczos))
        self.n_diff = self.n_cycles = self.steps = 0
        self.energies = []

    def step(self, info, Tg, Sg, nxt):
        orc, W, T_or, S_or, n_keep = self.orc, self.W, self.T_or, self.S_or, self.n_keep
        label, step = self.label, self.steps
        self.steps += 1
        i = info["index"]
        assert i == len(W) - 1
        wr, wc = W[i]
        sr, sv, sa, _ = orc.sigma(self.osys, wr, wc)
        for j in range(i + 1):
            rj, cj = W[j]
            t = float(np.dot(cj, _on(sr, sv, rj)))
            tb = float(np.dot(np.abs(cj), _on(sr, sa, rj)))
            T_or[j, i] = t
            S_or[j, i] = orc.sparse_dot(rj, cj, wr, wc)
            assert abs(Tg[j, i] - t) <= TOL * tb + 1e-15, (label, step, j, Tg[j, i], t, tb)
            assert abs(Sg[j, i] - S_or[j, i]) <= 1e-13, (label, step, j)
        a, b = T_or[i, i], (T_or[i - 1, i] if i > 0 else 0.0)
        assert info["a"] == Tg[i, i] and info["b"] == (Tg[i - 1, i] if i > 0 else 0.0)
        if not info["cycle_end"]:
            terms = [(a, wr, wc)] + ([(b, W[i - 1][0], W[i - 1][1])] if i > 0 else [])
            ur, uv = orc.sparse_axpy_union(sr, sv, terms)
            # |u_k| is known to 1e-11 of its terms' magnitudes, plus what the
            # GPU's a and b may differ by (1e-11 of their own terms) times w_k
            da = TOL * float(np.dot(np.abs(wc), _on(sr, sa, wr)))
            wi_u = np.abs(_on(wr, wc, ur))
            tol = TOL * (_on(sr, sa, ur) + abs(a) * wi_u) + da * wi_u
            if i > 0:
                rm, cm = W[i - 1]
                db = TOL * float(np.dot(np.abs(cm), _on(sr, sa, rm)))
                wm_u = np.abs(_on(rm, cm, ur))
                tol = tol + TOL * abs(b) * wm_u + db * wm_u
            self.n_diff += _check_kept(nxt[0], nxt[1], ur, uv, tol, n_keep, orc, f"{label} step {step}")
            W.append(nxt)
            return
        # cycle end: the generalised eigenproblem of this cycle
        m = i + 1
        sym = lambda X: np.triu(X[:m, :m]) + np.triu(X[:m, :m], 1).T  # noqa: E731
        lam_g, x_g = orc.gen_eig_lowest(sym(Tg), sym(Sg))
        lam_o, _ = orc.gen_eig_lowest(sym(T_or), sym(S_or))
        assert abs(info["lambda_min"] - lam_g) < 1e-9, (label, step, info["lambda_min"], lam_g)
        assert abs(info["lambda_min"] - lam_o) < 1e-9, (label, step, info["lambda_min"], lam_o)
        self.energies.append(info["lambda_min"])
        # restart vector: Psi = sum_j x_j w_j (ascending j), top N_d, normalised
        allr = np.unique(np.concatenate([w[0] for w in W]))
        acc = np.zeros(allr.size)
        asum = np.zeros(allr.size)
        for j, (rj, cj) in enumerate(W):
            pos = np.searchsorted(allr, rj)
            acc[pos] = acc[pos] + x_g[j] * cj
            asum[pos] = asum[pos] + np.abs(x_g[j] * cj)
        # the eigenvector's sign is free: match it on the largest entry
        big = np.argmax(np.abs(acc))
        g_big = _on(nxt[0], nxt[1], allr[big:big + 1])[0]
        sign = 1.0 if g_big * acc[big] >= 0 else -1.0
        # x is known to the two eigensolvers' rounding (Jacobi on the GPU's host
        # side, LAPACK here): 1e-10 of each entry's terms and 1e-12 of the largest
        tol = 1e-10 * asum + 1e-12 * np.abs(acc).max()
        self.n_diff += _check_kept(nxt[0], nxt[1], allr, acc, tol, n_keep, orc, f"{label} restart {step}", sign)
        self.W = [nxt]
        T_or[:] = 0.0
        S_or[:] = 0.0
        self.n_cycles += 1


def _replay(sf, orc, d, n_keep, n_lanczos, n_iter, label):
    gsys, osys = sf.System.from_dict(d), orc.System.from_dict(d)
    lz = sf.Lanczos(gsys, np.array([0], dtype=np.uint64), np.array([1.0]), n_keep, n_lanczos,
                    max_iter=n_iter)
    rp = Replay(orc, osys, _vec(sf, lz), n_keep, n_lanczos, label)
    for _ in range(n_iter):
        info = lz.step()
        Tg, Sg = lz.matrices()
        rp.step(info, Tg, Sg, _vec(sf, lz))
    lz.close()
    gsys.close()
    print(f"{label}: {n_iter} steps, {rp.n_cycles} cycle ends, energies {rp.energies}, "
          f"kept-set differences at the cut {rp.n_diff}")
    return rp.energies


def test_replay_closed_shell_cfg0(sf, orc):
    """8 orbitals, 4a/4b (spin-flip partners tie exactly), N_d = 300, 30 steps."""
    d = gen.config_system(0)
    e = _replay(sf, orc, d, 300, 10, 30, "cfg0 N_d=300")
    assert len(e) == 3


def test_replay_hubbard_ring_cfg1(sf, orc):
    """12-site Hubbard ring, 6a/6b, t = 1, U = 4, N_d = 2e4, N_L = 10, 40 steps
    from the aufbau determinant (rank 0)."""
    d = gen.config_system(1)
    e = _replay(sf, orc, d, 20_000, 10, 40, "Hubbard 12 sites N_d=2e4")
    assert len(e) == 4
