/*
 * Sparse-FCI oracle: a plain, slow CPU statement of what the sigma = H psi
 * path computes.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's CPU
 * baseline load this library.  It shares no code, header, table or helper
 * with the CUDA library, and the product path never calls it.
 *
 * Every function states one piece of the method in its most direct form:
 *   - binomial coefficients, C(n,k) = 0 for n < k (the note under Eq. 12);
 *   - the determinant <-> integer bijection h(D) = sum_i C(chi_i - 1, i)
 *     (Eq. 12), its inverse by the greedy combinatorial-number-system rule,
 *     and the paper's successor g (Sec. 2.2, Table 1);
 *   - the index of an (alpha, beta) determinant, alpha-major:
 *     rank = h(alpha) * C(n, n_beta) + h(beta)  (the paper buckets on the
 *     spin-up string only, Sec. 3);
 *   - Slater-Condon matrix elements by comparing two occupation lists, with the
 *     fermionic sign counted from the Jordan-Wigner ordering (alpha orbitals
 *     0..n-1, then beta orbitals 0..n-1);
 *   - sigma = H psi by listing every intermediate element (target, source,
 *     value) (Sec. 2.2), sorting by (target, source) and summing each target's
 *     run in ascending source order;
 *   - one sigma entry by pulling from the determinants connected to the target;
 *   - the dense Hamiltonian of a small space, and the one- and two-particle
 *     density matrices by applying creation/annihilation operators.
 *
 * Built with -O2 -ffp-contract=off so that no multiply-add is fused.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int n, na, nb;
    double e_core;
    const double *h; /* n*n, h[p*n+q] */
    const double *g; /* n^4, g[((p*n+q)*n+r)*n+s] = (pq|rs) */
} or_sys;

/* ------------------------------------------------------------ binomials */

static uint64_t BIN[65][65];

__attribute__((constructor)) static void or_binom_init(void)
{
    for (int n = 0; n <= 64; n++) {
        for (int k = 0; k <= 64; k++)
            BIN[n][k] = 0;
        BIN[n][0] = 1;
        for (int k = 1; k <= n; k++)
            BIN[n][k] = BIN[n - 1][k - 1] + BIN[n - 1][k];
    }
}

/* C(n, k), and 0 whenever n < k (Eq. 12's convention). */
uint64_t or_binom(int n, int k)
{
    if (n < 0 || k < 0 || n > 64 || k > 64 || n < k)
        return 0;
    return BIN[n][k];
}

/* -------------------------------------------------- Eq. 12 and its inverse */

/* h(D) = sum_{i=1..M} C(chi_i - 1, i), chi_1 < chi_2 < ... the occupied
 * orbitals counted from 1 (Eq. 12).  Orbital chi is bit chi-1 of s. */
uint64_t or_string_rank(uint64_t s, int n)
{
    uint64_t h = 0;
    int i = 0;
    for (int chi = 1; chi <= n; chi++) {
        if ((s >> (chi - 1)) & 1u) {
            i += 1;
            h += or_binom(chi - 1, i);
        }
    }
    return h;
}

/* Inverse of Eq. 12 (the paper does not print one): for i = M down to 1 take
 * the largest c with C(c, i) <= r; electron i sits on orbital c+1 (bit c);
 * subtract C(c, i). */
uint64_t or_string_unrank(uint64_t r, int n, int m)
{
    uint64_t s = 0;
    int top = n - 1;
    for (int i = m; i >= 1; i--) {
        int c = top;
        while (c >= 0 && or_binom(c, i) > r)
            c--;
        if (c < 0)
            return 0; /* unreachable for r < C(n, m) */
        s |= 1ull << c;
        r -= or_binom(c, i);
        top = c - 1;
    }
    return s;
}

/* The successor g of Sec. 2.2 (Table 1): scanning from orbital 1, find the
 * first occupied orbital whose right neighbour is empty; flush every occupied
 * orbital on its left to the far left, and swap the pair.  Returns 0 for the
 * final string (all occupied orbitals flushed right). */
int or_string_successor(uint64_t s, int n, uint64_t *next)
{
    int below = 0;
    for (int p = 0; p + 1 < n; p++) {
        if (!((s >> p) & 1u))
            continue;
        if (!((s >> (p + 1)) & 1u)) {
            uint64_t t = s & ~((1ull << (p + 1)) - 1ull); /* clear 0..p */
            if (below)
                t |= (1ull << below) - 1ull;
            t |= 1ull << (p + 1);
            *next = t;
            return 1;
        }
        below += 1;
    }
    return 0;
}

/* dim = C(n, na) * C(n, nb); returns -1 if it does not fit below 2^64 - 1. */
int or_dim(int n, int na, int nb, uint64_t *dim)
{
    if (n < 1 || n > 64 || na < 0 || nb < 0 || na > n || nb > n)
        return -1;
    uint64_t ca = or_binom(n, na), cb = or_binom(n, nb);
    if (cb != 0 && ca > (UINT64_MAX - 1) / cb)
        return -1;
    *dim = ca * cb;
    return 0;
}

/* alpha-major index of a determinant. */
uint64_t or_det_rank(int n, int nb, uint64_t a, uint64_t b)
{
    return or_string_rank(a, n) * or_binom(n, nb) + or_string_rank(b, n);
}

void or_det_unrank(int n, int na, int nb, uint64_t r, uint64_t *a, uint64_t *b)
{
    uint64_t cb = or_binom(n, nb);
    *a = or_string_unrank(r / cb, n, na);
    *b = or_string_unrank(r % cb, n, nb);
}

void or_det_rank_batch(int n, int nb, const uint64_t *a, const uint64_t *b,
                       uint64_t *out, int64_t count)
{
    for (int64_t i = 0; i < count; i++)
        out[i] = or_det_rank(n, nb, a[i], b[i]);
}

void or_det_unrank_batch(int n, int na, int nb, const uint64_t *r,
                         uint64_t *a, uint64_t *b, int64_t count)
{
    for (int64_t i = 0; i < count; i++)
        or_det_unrank(n, na, nb, r[i], &a[i], &b[i]);
}

/* ------------------------------------------------ fermionic sign, elements */

/* number of occupied spin orbitals with Jordan-Wigner index below so
 * (alpha orbital p has index p, beta orbital p has index n + p). */
static int occupied_below(uint64_t a, uint64_t b, int n, int so)
{
    int c = 0;
    for (int q = 0; q < so; q++)
        c += (q < n) ? (int)((a >> q) & 1u) : (int)((b >> (q - n)) & 1u);
    return c;
}

static void set_so(uint64_t *a, uint64_t *b, int n, int so, int on)
{
    uint64_t *w = so < n ? a : b;
    int p = so < n ? so : so - n;
    if (on)
        *w |= 1ull << p;
    else
        *w &= ~(1ull << p);
}

/* apply a^dagger_to a_from to the determinant, return the sign it picks up. */
static int apply_hop(uint64_t *a, uint64_t *b, int n, int from, int to)
{
    int sign = 1;
    if (occupied_below(*a, *b, n, from) & 1)
        sign = -sign;
    set_so(a, b, n, from, 0);
    if (occupied_below(*a, *b, n, to) & 1)
        sign = -sign;
    set_so(a, b, n, to, 1);
    return sign;
}

static int occ_list(uint64_t s, int n, int *occ)
{
    int m = 0;
    for (int p = 0; p < n; p++)
        if ((s >> p) & 1u)
            occ[m++] = p;
    return m;
}

static inline double H1(const or_sys *S, int p, int q) { return S->h[p * S->n + q]; }

static inline double G2(const or_sys *S, int p, int q, int r, int s)
{
    int n = S->n;
    return S->g[(((size_t)p * n + q) * n + r) * n + s];
}

static int lowest_bit(uint64_t x)
{
    for (int p = 0; p < 64; p++)
        if ((x >> p) & 1u)
            return p;
    return -1;
}

/* <D_src| H |D_src>: sum_k h_kk + 1/2 sum_{k,l} (kk|ll)
 *                    - 1/2 sum_{k,l same spin} (kl|lk) + e_core. */
static double diag_element(const or_sys *S, uint64_t a, uint64_t b)
{
    int n = S->n, oa[64], ob[64];
    int ma = occ_list(a, n, oa), mb = occ_list(b, n, ob);
    int all[128], m = 0;
    for (int k = 0; k < ma; k++)
        all[m++] = oa[k];
    for (int k = 0; k < mb; k++)
        all[m++] = ob[k];
    double one = 0.0, coul = 0.0, exch = 0.0;
    for (int k = 0; k < ma; k++)
        one += H1(S, oa[k], oa[k]);
    for (int k = 0; k < mb; k++)
        one += H1(S, ob[k], ob[k]);
    for (int k = 0; k < m; k++)
        for (int l = 0; l < m; l++)
            coul += G2(S, all[k], all[k], all[l], all[l]);
    for (int k = 0; k < ma; k++)
        for (int l = 0; l < ma; l++)
            exch += G2(S, oa[k], oa[l], oa[l], oa[k]);
    for (int k = 0; k < mb; k++)
        for (int l = 0; l < mb; l++)
            exch += G2(S, ob[k], ob[l], ob[l], ob[k]);
    return S->e_core + one + 0.5 * coul - 0.5 * exch;
}

/* <D_tgt| H |D_src> by comparing the two occupation lists.  Occupations in the
 * sums are those of the source.  Zero beyond double excitations or when the
 * electron counts differ. */
double or_hmat(const or_sys *S, uint64_t as, uint64_t bs, uint64_t at, uint64_t bt)
{
    int n = S->n;
    uint64_t ra = as & ~at, pa = at & ~as; /* alpha removed / added */
    uint64_t rb = bs & ~bt, pb = bt & ~bs;
    int ka = __builtin_popcountll(ra), kb = __builtin_popcountll(rb);
    if (__builtin_popcountll(pa) != ka || __builtin_popcountll(pb) != kb)
        return 0.0;
    if (ka + kb > 2)
        return 0.0;
    if (ka + kb == 0)
        return diag_element(S, as, bs);

    int oa[64], ob[64];
    int ma = occ_list(as, n, oa), mb = occ_list(bs, n, ob);
    uint64_t ca = as, cb = bs;

    if (ka + kb == 1) {
        int alpha = (ka == 1);
        int i = lowest_bit(alpha ? ra : rb), x = lowest_bit(alpha ? pa : pb);
        int off = alpha ? 0 : n;
        int sign = apply_hop(&ca, &cb, n, off + i, off + x);
        double v = H1(S, x, i);
        for (int k = 0; k < ma; k++)
            v += G2(S, x, i, oa[k], oa[k]);
        for (int k = 0; k < mb; k++)
            v += G2(S, x, i, ob[k], ob[k]);
        const int *os = alpha ? oa : ob;
        int ms = alpha ? ma : mb;
        for (int k = 0; k < ms; k++)
            v -= G2(S, x, os[k], os[k], i);
        return sign * v;
    }
    if (ka == 2 || kb == 2) {
        int alpha = (ka == 2);
        uint64_t r = alpha ? ra : rb, p = alpha ? pa : pb;
        int i = lowest_bit(r), j = lowest_bit(r & (r - 1));
        int x = lowest_bit(p), y = lowest_bit(p & (p - 1));
        int off = alpha ? 0 : n;
        int sign = apply_hop(&ca, &cb, n, off + i, off + x);
        sign *= apply_hop(&ca, &cb, n, off + j, off + y);
        return sign * (G2(S, x, i, y, j) - G2(S, x, j, y, i));
    }
    /* one alpha and one beta electron moved */
    {
        int i = lowest_bit(ra), x = lowest_bit(pa);
        int j = lowest_bit(rb), y = lowest_bit(pb);
        int sign = apply_hop(&ca, &cb, n, i, x);
        sign *= apply_hop(&ca, &cb, n, n + j, n + y);
        return sign * G2(S, x, i, y, j);
    }
}

void or_hmat_batch(const or_sys *S, const uint64_t *as, const uint64_t *bs, const uint64_t *at,
                   const uint64_t *bt, double *out, int64_t count)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < count; i++)
        out[i] = or_hmat(S, as[i], bs[i], at[i], bt[i]);
}

/* ---------------------------------------------------------- enumeration */

/* Number of determinants connected to one determinant by a single or double
 * excitation. */
int64_t or_n_connected(int n, int na, int nb)
{
    int64_t va = n - na, vb = n - nb;
    int64_t sa = (int64_t)na * va, sb = (int64_t)nb * vb;
    int64_t daa = (int64_t)or_binom(na, 2) * (int64_t)or_binom((int)va, 2);
    int64_t dbb = (int64_t)or_binom(nb, 2) * (int64_t)or_binom((int)vb, 2);
    return sa + sb + daa + dbb + sa * sb;
}

/* All determinants reached from (a, b) by one or two electron moves, in a fixed
 * order: alpha singles, beta singles, alpha-alpha doubles, beta-beta doubles,
 * alpha-beta doubles (Sec. 4.3, outlook: all single and double excitations). */
int64_t or_connected(int n, uint64_t a, uint64_t b, uint64_t *oa_out, uint64_t *ob_out)
{
    int oa[64], va[64], ob[64], vb[64];
    int ma = 0, mva = 0, mb = 0, mvb = 0;
    for (int p = 0; p < n; p++) {
        if ((a >> p) & 1u) oa[ma++] = p; else va[mva++] = p;
        if ((b >> p) & 1u) ob[mb++] = p; else vb[mvb++] = p;
    }
    int64_t c = 0;
    for (int i = 0; i < ma; i++)
        for (int x = 0; x < mva; x++) {
            oa_out[c] = a ^ (1ull << oa[i]) ^ (1ull << va[x]);
            ob_out[c++] = b;
        }
    for (int i = 0; i < mb; i++)
        for (int x = 0; x < mvb; x++) {
            oa_out[c] = a;
            ob_out[c++] = b ^ (1ull << ob[i]) ^ (1ull << vb[x]);
        }
    for (int i = 0; i < ma; i++)
        for (int j = i + 1; j < ma; j++)
            for (int x = 0; x < mva; x++)
                for (int y = x + 1; y < mva; y++) {
                    oa_out[c] = a ^ (1ull << oa[i]) ^ (1ull << oa[j]) ^ (1ull << va[x]) ^ (1ull << va[y]);
                    ob_out[c++] = b;
                }
    for (int i = 0; i < mb; i++)
        for (int j = i + 1; j < mb; j++)
            for (int x = 0; x < mvb; x++)
                for (int y = x + 1; y < mvb; y++) {
                    oa_out[c] = a;
                    ob_out[c++] = b ^ (1ull << ob[i]) ^ (1ull << ob[j]) ^ (1ull << vb[x]) ^ (1ull << vb[y]);
                }
    for (int i = 0; i < ma; i++)
        for (int x = 0; x < mva; x++)
            for (int j = 0; j < mb; j++)
                for (int y = 0; y < mvb; y++) {
                    oa_out[c] = a ^ (1ull << oa[i]) ^ (1ull << va[x]);
                    ob_out[c++] = b ^ (1ull << ob[j]) ^ (1ull << vb[y]);
                }
    return c;
}

/* ---------------------------------------------------------------- sigma */

typedef struct {
    uint64_t tgt;
    int64_t src;
    double v;
} or_elem;

static int cmp_elem(const void *x, const void *y)
{
    const or_elem *p = (const or_elem *)x, *q = (const or_elem *)y;
    if (p->tgt != q->tgt)
        return p->tgt < q->tgt ? -1 : 1;
    if (p->src != q->src)
        return p->src < q->src ? -1 : 1;
    return 0;
}

/* sigma = H psi (Sec. 2.2).  Step 1: every input entry (D, c_D) generates its
 * intermediate elements (rank(D'), <D'|H|D> c_D) for D' = D and every D'
 * connected to D; products that are exactly zero are not generated, nor, with
 * eps_elem > 0, products with |<D'|H|D> c_D| < eps_elem (the heat-bath style
 * selection the outlook of Sec. 4 proposes; eps_elem = 0 is the exact sigma).
 * Step 2:
 * the elements are sorted by (target, source) and each target's run is summed
 * in ascending source order.  out_abs receives sum |element| per target.
 * Returns the number of distinct targets (entries beyond cap are not
 * written), or -1 if memory runs out.  *n_elements receives the number of
 * connected elements enumerated (diagonal included). */
int64_t or_sigma(const or_sys *S, const uint64_t *in_rank, const double *in_coef,
                 int64_t n_in, uint64_t *out_rank, double *out_val, double *out_abs,
                 int64_t cap, int64_t *n_elements, int n_threads, double eps_elem)
{
    int n = S->n, na = S->na, nb = S->nb;
    int64_t per = or_n_connected(n, na, nb) + 1;
    int64_t total = per * n_in;
    or_elem *el = (or_elem *)malloc(sizeof(or_elem) * (size_t)(total > 0 ? total : 1));
    if (!el)
        return -1;
    if (n_threads < 1)
        n_threads = 1;
#pragma omp parallel num_threads(n_threads)
    {
        uint64_t *ta = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)per);
        uint64_t *tb = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)per);
#pragma omp for schedule(dynamic, 16)
        for (int64_t s = 0; s < n_in; s++) {
            uint64_t a, b;
            or_det_unrank(n, na, nb, in_rank[s], &a, &b);
            ta[0] = a;
            tb[0] = b;
            int64_t m = 1 + or_connected(n, a, b, ta + 1, tb + 1);
            for (int64_t e = 0; e < m; e++) {
                double v = or_hmat(S, a, b, ta[e], tb[e]) * in_coef[s];
                or_elem *o = &el[s * per + e];
                o->tgt = (v != 0.0 && !(fabs(v) < eps_elem)) ? or_det_rank(n, nb, ta[e], tb[e]) : UINT64_MAX;
                o->src = s;
                o->v = v;
            }
        }
        free(ta);
        free(tb);
    }
    int64_t kept = 0;
    for (int64_t e = 0; e < total; e++)
        if (el[e].tgt != UINT64_MAX)
            el[kept++] = el[e];
    if (n_elements)
        *n_elements = total;
    qsort(el, (size_t)kept, sizeof(or_elem), cmp_elem);
    int64_t m = 0;
    for (int64_t e = 0; e < kept;) {
        uint64_t t = el[e].tgt;
        double sum = 0.0, asum = 0.0;
        while (e < kept && el[e].tgt == t) {
            sum += el[e].v;
            asum += fabs(el[e].v);
            e++;
        }
        if (m < cap) {
            out_rank[m] = t;
            out_val[m] = sum;
            if (out_abs)
                out_abs[m] = asum;
        }
        m++;
    }
    free(el);
    return m;
}

static int64_t find_rank(const uint64_t *r, int64_t n, uint64_t key)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (r[mid] < key)
            lo = mid + 1;
        else
            hi = mid;
    }
    return (lo < n && r[lo] == key) ? lo : -1;
}

static int cmp_pair(const void *x, const void *y)
{
    const or_elem *p = (const or_elem *)x, *q = (const or_elem *)y;
    return (p->src > q->src) - (p->src < q->src);
}

/* One entry sigma_k, pulled: every determinant D in {k} and connected to k
 * that the (ascending, unique) input holds contributes <k|H|D> c_D, summed in
 * ascending source order (the same terms and order as or_sigma).  Returns the
 * value; *present = 1 if at least one non-zero product arrived. */
double or_sigma_entry(const or_sys *S, const uint64_t *in_rank, const double *in_coef,
                      int64_t n_in, uint64_t target, double *abs_sum, int *present)
{
    int n = S->n, na = S->na, nb = S->nb;
    int64_t per = or_n_connected(n, na, nb) + 1;
    uint64_t *ta = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)per);
    uint64_t *tb = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)per);
    or_elem *pr = (or_elem *)malloc(sizeof(or_elem) * (size_t)per);
    uint64_t ka, kb;
    or_det_unrank(n, na, nb, target, &ka, &kb);
    ta[0] = ka;
    tb[0] = kb;
    int64_t m = 1 + or_connected(n, ka, kb, ta + 1, tb + 1), np = 0;
    for (int64_t e = 0; e < m; e++) {
        int64_t s = find_rank(in_rank, n_in, or_det_rank(n, nb, ta[e], tb[e]));
        if (s < 0)
            continue;
        double v = or_hmat(S, ta[e], tb[e], ka, kb) * in_coef[s];
        if (v == 0.0)
            continue;
        pr[np].src = s;
        pr[np].v = v;
        pr[np].tgt = target;
        np++;
    }
    qsort(pr, (size_t)np, sizeof(or_elem), cmp_pair);
    double sum = 0.0, asum = 0.0;
    for (int64_t e = 0; e < np; e++) {
        sum += pr[e].v;
        asum += fabs(pr[e].v);
    }
    if (abs_sum)
        *abs_sum = asum;
    if (present)
        *present = np > 0;
    free(ta);
    free(tb);
    free(pr);
    return sum;
}

void or_sigma_entries(const or_sys *S, const uint64_t *in_rank, const double *in_coef,
                      int64_t n_in, const uint64_t *targets, int64_t n_t,
                      double *val, double *abs_sum, int32_t *present, int n_threads)
{
    if (n_threads < 1)
        n_threads = 1;
#pragma omp parallel for num_threads(n_threads) schedule(dynamic, 4)
    for (int64_t t = 0; t < n_t; t++) {
        int pres = 0;
        val[t] = or_sigma_entry(S, in_rank, in_coef, n_in, targets[t], &abs_sum[t], &pres);
        present[t] = pres;
    }
}

/* Dense H of the whole space (small spaces only): H[t*dim + s] = <t|H|s>. */
int or_dense_h(const or_sys *S, double *H, int64_t dim)
{
    int n = S->n, na = S->na, nb = S->nb;
    uint64_t *A = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)dim);
    uint64_t *B = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)dim);
    if (!A || !B)
        return -1;
    for (int64_t r = 0; r < dim; r++)
        or_det_unrank(n, na, nb, (uint64_t)r, &A[r], &B[r]);
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t t = 0; t < dim; t++)
        for (int64_t s = 0; s < dim; s++)
            H[t * dim + s] = or_hmat(S, A[s], B[s], A[t], B[t]);
    free(A);
    free(B);
    return 0;
}

/* ---------------------------------------------------------------- RDMs */

/* apply a_so (on = 0) or a^dagger_so (on = 1); returns 0 if the result
 * vanishes, else the sign. */
static int apply_op(uint64_t *a, uint64_t *b, int n, int so, int on)
{
    uint64_t w = so < n ? *a : *b;
    int p = so < n ? so : so - n;
    int occ = (int)((w >> p) & 1u);
    if (occ == on)
        return 0;
    int sign = (occupied_below(*a, *b, n, so) & 1) ? -1 : 1;
    set_so(a, b, n, so, on);
    return sign;
}

/* Spin-summed density matrices of psi (not normalised):
 *   rdm1[p*n+q]          = sum_sigma     <psi| a+_{p s} a_{q s} |psi>
 *   rdm2[((p*n+q)*n+r)*n+s] = sum_{s,t} <psi| a+_{p s} a+_{r t} a_{s t} a_{q s} |psi>
 * by applying the operators right to left to every determinant of psi and
 * looking the result up in psi.  O(|psi| N^2 (2n)^2): small cases only. */
int or_rdm12(const or_sys *S, const uint64_t *rank, const double *coef, int64_t m,
             double *rdm1, double *rdm2)
{
    int n = S->n, na = S->na, nb = S->nb;
    size_t n2 = (size_t)n * n, n4 = n2 * n2;
    memset(rdm1, 0, sizeof(double) * n2);
    memset(rdm2, 0, sizeof(double) * n4);
    for (int64_t d = 0; d < m; d++) {
        uint64_t a0, b0;
        or_det_unrank(n, na, nb, rank[d], &a0, &b0);
        for (int sg = 0; sg < 2; sg++)
            for (int p = 0; p < n; p++)
                for (int q = 0; q < n; q++) {
                    uint64_t a = a0, b = b0;
                    int s1 = apply_op(&a, &b, n, sg * n + q, 0);
                    if (!s1) continue;
                    int s2 = apply_op(&a, &b, n, sg * n + p, 1);
                    if (!s2) continue;
                    int64_t e = find_rank(rank, m, or_det_rank(n, nb, a, b));
                    if (e < 0) continue;
                    rdm1[p * n + q] += s1 * s2 * coef[e] * coef[d];
                }
        for (int sg = 0; sg < 2; sg++)
            for (int tg = 0; tg < 2; tg++)
                for (int q = 0; q < n; q++)
                    for (int s = 0; s < n; s++) {
                        uint64_t a1 = a0, b1 = b0;
                        int s1 = apply_op(&a1, &b1, n, sg * n + q, 0);
                        if (!s1) continue;
                        int s2 = apply_op(&a1, &b1, n, tg * n + s, 0);
                        if (!s2) continue;
                        for (int r = 0; r < n; r++) {
                            uint64_t a2 = a1, b2 = b1;
                            int s3 = apply_op(&a2, &b2, n, tg * n + r, 1);
                            if (!s3) continue;
                            for (int p = 0; p < n; p++) {
                                uint64_t a = a2, b = b2;
                                int s4 = apply_op(&a, &b, n, sg * n + p, 1);
                                if (!s4) continue;
                                int64_t e = find_rank(rank, m, or_det_rank(n, nb, a, b));
                                if (e < 0) continue;
                                rdm2[(((size_t)p * n + q) * n + r) * n + s] +=
                                    s1 * s2 * s3 * s4 * coef[e] * coef[d];
                            }
                        }
                    }
    }
    return 0;
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
